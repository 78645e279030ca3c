// Batched execution of many small parametric circuits in one persistent kernel launch,
// replayed from a CUDA graph: for every (circuit, observable) pair the energy
// E = <psi|H|psi> and the adjoint gradient dE/dtheta (reverse sweep of Sec. 4.4 parametric
// circuits, rotation convention exp(+i theta P / 2) of the paper's gate table), complex64
// storage with compensated FP32 products summed in FP64.
//
// Layout of the work:
//  * One CTA of 1024 threads per SM claims circuits through an atomic counter, longest first
//    (the host sorts by estimated cost); nothing waits on another CTA.
//  * A circuit's gates are split on the host into passes. Each pass owns a window of at most
//    13 "local" qubits and holds gates acting only inside it; a gate joins the earliest pass
//    after every pass that touched its qubits and that still has room, so the passes applied in
//    order reproduce the circuit (gates outside a window commute with it). A pass is applied to
//    the state one chunk of 2^13 amplitudes at a time (the chunk fixes the other qubits), each
//    chunk staged in shared memory, so a whole pass costs one read and one write of the state.
//  * n <= 13: the whole state (and lambda) stays in shared memory for the entire circuit.
//  * Forward sweep; lambda = H psi and E = Re <psi|lambda>; reverse sweep over passes and gates:
//    at a rotation exp(i theta P/2) the gradient is -Im <lambda|P|psi>, then the gate is
//    un-applied from psi and lambda.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kBT = 512;               // threads per CTA: 16 warps
constexpr int kWarps = kBT / 32;
constexpr int kLocal = 13;             // qubits per chunk
constexpr int kChunk = 1 << kLocal;    // 16 warps x 32 lanes x 16 registers
constexpr int kRegBits = 4;
constexpr int kRegs = 1 << kRegBits;
constexpr int kMaxStageParams = 32;
constexpr int kClasses = 5;            // groups of 16, 8, 4, 2, 1 warps
constexpr int kMaxBatchQubits = 24;

enum BKind : uint8_t { BK_RX = 0, BK_RY = 1, BK_RZ = 2, BK_CZ = 3, BK_CNOT = 4, BK_H = 5, BK_X = 6, BK_Y = 7, BK_Z = 8 };

// one gate in the local coordinates of its pass
struct BGate {
    uint8_t kind;
    uint8_t a;      // local bit of the target
    uint8_t b;      // local bit of the second qubit (CZ) or of the control (CNOT)
    uint8_t ja;     // register bit holding the target (non-diagonal gates)
    int32_t slot;   // angle slot (rotations), -1 otherwise
    int32_t grad;   // gradient index (parametric rotations), -1 otherwise
};

// gates whose non-diagonal actions stay inside the register sub-cube spanned by act[]
struct BStage {
    int32_t g0, g1;
    int32_t nact;
    int32_t nparam;
    uint8_t act[4];
};

struct BPass {
    int32_t s0, s1;               // stage range
    uint32_t tab_lo[128];         // local index bits 0..6 -> address bits
    uint32_t tab_hi[64];          // local index bits 7..12 -> address bits
    uint32_t nonlocal;            // qubits outside the window (fixed per chunk)
    int32_t nlocal;
};

struct BTerm {
    uint32_t xmask, zmask;
    double coef;
    int32_t nY, pad;
};

struct BItem {
    int32_t n;
    int32_t p0, p1;               // pass range
    int32_t t0, t1;               // observable term range
    int32_t angle0;               // first angle slot
    int32_t grad0, ngrad;         // gradient outputs
};

struct BatchDev {
    const BItem* items;
    const int32_t* order;         // items grouped by class, longest first within a class
    const BPass* passes;
    const BStage* stages;
    const BGate* gates;
    const BTerm* terms;
    const float2* cs;             // (cos, sin) of theta/2 per angle slot
    float2* ws;                   // per-CTA workspace: psi and lambda, 2^maxn each (chunked circuits)
    uint64_t ws_stride;
    double* energy;
    double* grad;
    unsigned int* counters;       // one work counter per class
    int32_t cls_begin[kClasses + 1];
};

// group barrier: the CTA, a named barrier over the group's warps, or the warp
__device__ __forceinline__ void gbar(int G, int w0) {
    if (G == kWarps) {
        __syncthreads();
    } else if (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + w0), "r"(G * 32) : "memory");
    }
}

// shared-memory position of local index l: the low four bits are XOR-folded with the higher
// ones so that lanes spread over the banks whichever bits are in registers
__device__ __forceinline__ uint32_t swz(uint32_t l) { return l ^ ((l >> 4) & 15u) ^ ((l >> 8) & 15u); }

__device__ __forceinline__ uint32_t chunk_addr(const BPass& P, uint32_t base, uint32_t l) {
    return base | P.tab_lo[l & 127] | P.tab_hi[l >> 7];
}

__device__ __forceinline__ uint32_t chunk_base(uint32_t nonlocal, uint32_t c) {
    uint32_t r = 0, m = nonlocal;
    while (m) {
        const uint32_t bit = m & (0u - m);
        if (c & 1u) r |= bit;
        c >>= 1;
        m ^= bit;
    }
    return r;
}

// chunk transfers between global memory and the shared-memory slice (chunked circuits run on
// the whole CTA: 512 threads x 16 amplitudes); every load is issued before the first store
__device__ __noinline__ void chunk_load(const BPass& P, uint32_t base, const float2* __restrict__ g, float2* s,
                                           int tg) {
    float2 t[kRegs];
#pragma unroll
    for (int j = 0; j < kRegs; j++) t[j] = g[chunk_addr(P, base, uint32_t(tg + j * kBT))];
#pragma unroll
    for (int j = 0; j < kRegs; j++) s[uint32_t(tg + j * kBT) ^ ((uint32_t(tg + j * kBT) >> 4) & 15u) ^
                                      ((uint32_t(tg + j * kBT) >> 8) & 15u)] = t[j];
}
__device__ __noinline__ void chunk_store(const BPass& P, uint32_t base, float2* __restrict__ g, const float2* s,
                                            int tg) {
    float2 t[kRegs];
#pragma unroll
    for (int j = 0; j < kRegs; j++) {
        const uint32_t l = uint32_t(tg + j * kBT);
        t[j] = s[l ^ ((l >> 4) & 15u) ^ ((l >> 8) & 15u)];
    }
#pragma unroll
    for (int j = 0; j < kRegs; j++) g[chunk_addr(P, base, uint32_t(tg + j * kBT))] = t[j];
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// 2x2 complex matrix of a non-diagonal single-qubit gate (or of its adjoint)
struct M2 {
    float2 m00, m01, m10, m11;
};
__device__ __forceinline__ M2 gate_m2(uint8_t kind, float c, float sn) {
    M2 m;
    switch (kind) {
        case BK_RX:  // [[c, i s], [i s, c]]
            m.m00 = make_float2(c, 0.f); m.m01 = make_float2(0.f, sn);
            m.m10 = make_float2(0.f, sn); m.m11 = make_float2(c, 0.f);
            break;
        case BK_RY:  // [[c, s], [-s, c]]
            m.m00 = make_float2(c, 0.f); m.m01 = make_float2(sn, 0.f);
            m.m10 = make_float2(-sn, 0.f); m.m11 = make_float2(c, 0.f);
            break;
        case BK_H: {
            const float h = 0.70710678118654752f;
            m.m00 = make_float2(h, 0.f); m.m01 = make_float2(h, 0.f);
            m.m10 = make_float2(h, 0.f); m.m11 = make_float2(-h, 0.f);
            break;
        }
        case BK_X:
            m.m00 = make_float2(0.f, 0.f); m.m01 = make_float2(1.f, 0.f);
            m.m10 = make_float2(1.f, 0.f); m.m11 = make_float2(0.f, 0.f);
            break;
        default:  // Y = [[0, -i], [i, 0]]
            m.m00 = make_float2(0.f, 0.f); m.m01 = make_float2(0.f, -1.f);
            m.m10 = make_float2(0.f, 1.f); m.m11 = make_float2(0.f, 0.f);
            break;
    }
    return m;
}

__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

// 2x2 update of the register pairs (r, r | 2^J)
template <int J>
__device__ __forceinline__ void pairs_1q(float2 (&v)[kRegs], int R, const M2& m) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        if (r >= R) continue;
        const int r1 = r | (1 << J);
        const float2 u = v[r], w = v[r1];
        v[r] = cfma2(m.m01, w, cfma2(m.m00, u, make_float2(0.f, 0.f)));
        v[r1] = cfma2(m.m11, w, cfma2(m.m10, u, make_float2(0.f, 0.f)));
    }
}

// local index of register r of this thread: the thread's base (its bits outside the register
// sub-cube) plus the active bits selected by r
struct LocalMap {
    uint32_t base;
    uint32_t am[kRegBits];
    __device__ __forceinline__ uint32_t at(int r) const {
        uint32_t o = base;
#pragma unroll
        for (int j = 0; j < kRegBits; j++)
            if ((r >> j) & 1) o |= am[j];
        return o;
    }
};

template <int J>
__device__ __forceinline__ void pairs_cnot(float2 (&v)[kRegs], const LocalMap& li, int R, int cb) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        if (r >= R) continue;
        const int r1 = r | (1 << J);
        if ((li.at(r) >> cb) & 1) {
            const float2 u = v[r];
            v[r] = v[r1];
            v[r1] = u;
        }
    }
}

// apply g (or its adjoint) to the registers
__device__ __forceinline__ void apply_reg(float2 (&v)[kRegs], const LocalMap& li, int R, const BGate& g,
                                          float2 cs, bool adjoint) {
    const float c = cs.x, sn = adjoint ? -cs.y : cs.y;
    switch (g.kind) {
        case BK_RZ: {  // diag(c + i s, c - i s)
#pragma unroll
            for (int r = 0; r < kRegs; r++)
                if (r < R) v[r] = cmulf(make_float2(c, ((li.at(r) >> g.a) & 1) ? -sn : sn), v[r]);
            break;
        }
        case BK_Z: {
#pragma unroll
            for (int r = 0; r < kRegs; r++)
                if (r < R && ((li.at(r) >> g.a) & 1)) v[r] = make_float2(-v[r].x, -v[r].y);
            break;
        }
        case BK_CZ: {
#pragma unroll
            for (int r = 0; r < kRegs; r++)
                if (r < R && ((li.at(r) >> g.a) & 1) && ((li.at(r) >> g.b) & 1)) v[r] = make_float2(-v[r].x, -v[r].y);
            break;
        }
        case BK_CNOT:
            switch (g.ja) {
                case 0: pairs_cnot<0>(v, li, R, g.b); break;
                case 1: pairs_cnot<1>(v, li, R, g.b); break;
                case 2: pairs_cnot<2>(v, li, R, g.b); break;
                default: pairs_cnot<3>(v, li, R, g.b); break;
            }
            break;
        default: {
            const M2 m = gate_m2(g.kind, c, sn);
            switch (g.ja) {
                case 0: pairs_1q<0>(v, R, m); break;
                case 1: pairs_1q<1>(v, R, m); break;
                case 2: pairs_1q<2>(v, R, m); break;
                default: pairs_1q<3>(v, R, m); break;
            }
            break;
        }
    }
}

// Im sum conj(lam) (P psi) over this thread's registers, P the axis of rotation g
template <int J>
__device__ __forceinline__ void grad_pairs(const float2 (&p)[kRegs], const float2 (&l)[kRegs], int R, uint8_t kind,
                                           DFAcc& im) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        if (r >= R) continue;
        const int r1 = r | (1 << J);
        const float2 a = p[r], b = p[r1], la = l[r], lb = l[r1];
        float2 p0, p1;  // X -> (b, a); Y -> (-i b, i a)
        if (kind == BK_RX) { p0 = b; p1 = a; }
        else { p0 = make_float2(b.y, -b.x); p1 = make_float2(-a.y, a.x); }
        df_add_prod(im, la.x, p0.y);
        df_add_prod(im, -la.y, p0.x);
        df_add_prod(im, lb.x, p1.y);
        df_add_prod(im, -lb.y, p1.x);
    }
}

__device__ __forceinline__ double grad_reg(const float2 (&p)[kRegs], const float2 (&l)[kRegs], const LocalMap& li,
                                           int R, const BGate& g) {
    DFAcc im;
    df_zero(im);
    if (g.kind == BK_RZ) {  // Z: (a, -b) by the target bit
#pragma unroll
        for (int r = 0; r < kRegs; r++) {
            if (r >= R) continue;
            const float sg = ((li.at(r) >> g.a) & 1) ? -1.f : 1.f;
            df_add_prod(im, l[r].x, sg * p[r].y);
            df_add_prod(im, -l[r].y, sg * p[r].x);
        }
    } else {
        switch (g.ja) {
            case 0: grad_pairs<0>(p, l, R, g.kind, im); break;
            case 1: grad_pairs<1>(p, l, R, g.kind, im); break;
            case 2: grad_pairs<2>(p, l, R, g.kind, im); break;
            default: grad_pairs<3>(p, l, R, g.kind, im); break;
        }
    }
    return df_value(im);
}

// local-index map of thread tg in stage S of a window of nl local bits
__device__ __forceinline__ LocalMap stage_map(const BStage& S, int nl, int tg) {
    LocalMap m;
    uint32_t actmask = 0;
#pragma unroll
    for (int j = 0; j < kRegBits; j++) {
        m.am[j] = j < S.nact ? (1u << S.act[j]) : 0u;
        actmask |= m.am[j];
    }
    uint32_t base = 0, t = uint32_t(tg);
    for (int b = 0; b < nl; b++) {
        if ((actmask >> b) & 1) continue;
        if (t & 1u) base |= 1u << b;
        t >>= 1;
    }
    m.base = base;
    return m;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBT, 1) k_batch(const BatchDev B) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* smem_p = reinterpret_cast<float2*>(smem);
    float2* smem_l = smem_p + kChunk;
    __shared__ double red[2][kMaxStageParams][kWarps];  // gradient partials per stage parity
    __shared__ double redE[kWarps];
    __shared__ int s_claim[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* gpsi = B.ws + uint64_t(blockIdx.x) * 2 * B.ws_stride;
    float2* glam = gpsi + B.ws_stride;
    int parity = 0;
    for (int cls = 0; cls < kClasses; cls++) {
        const int G = kWarps >> cls;
        const int w0 = (warp / G) * G;
        const int tg = threadIdx.x - w0 * 32;
        const int nthr = G * 32;
        float2* sp = smem_p + w0 * 32 * kRegs;
        float2* sl = smem_l + w0 * 32 * kRegs;
        const int count = B.cls_begin[cls + 1] - B.cls_begin[cls];
        while (true) {
            if (tg == 0) s_claim[w0] = int(atomicAdd(&B.counters[cls], 1u));
            gbar(G, w0);
            const int k = s_claim[w0];
            gbar(G, w0);
            if (k >= count) break;
            const int item = B.order[B.cls_begin[cls] + k];
            const BItem it = B.items[item];
            const int nl = it.n < kLocal ? it.n : kLocal;
            const bool resident = it.n <= kLocal;
            const uint32_t size = 1u << nl;
            const uint32_t N = 1u << it.n;
            const int R = 1 << (nl < kRegBits ? nl : kRegBits);
            const int T = int(size) / R;  // threads holding registers
            const float2* cs = B.cs + it.angle0;
            for (int j = tg; j < it.ngrad; j += nthr) B.grad[it.grad0 + j] = 0.0;
            // ---------------- forward sweep
            for (int p = it.p0; p < it.p1; p++) {
                const BPass& P = B.passes[p];
                const uint32_t nch = resident ? 1u : (N >> kLocal);
                for (uint32_t c = 0; c < nch; c++) {
                    const uint32_t base = resident ? 0u : chunk_base(P.nonlocal, c);
                    if (p == it.p0) {
                        for (uint32_t l = tg; l < size; l += nthr)
                            sp[swz(l)] = make_float2((base == 0 && l == 0) ? 1.f : 0.f, 0.f);
                    } else if (!resident) {
                        chunk_load(P, base, gpsi, sp, tg);
                    }
                    gbar(G, w0);
                    for (int s = P.s0; s < P.s1; s++) {
                        const BStage S = B.stages[s];
                        if (tg < T) {
                            const LocalMap li = stage_map(S, nl, tg);
                            float2 v[kRegs];
#pragma unroll
                            for (int r = 0; r < kRegs; r++)
                                if (r < R) v[r] = sp[swz(li.at(r))];
                            for (int gi = S.g0; gi < S.g1; gi++) {
                                const BGate g = B.gates[gi];
                                apply_reg(v, li, R, g, g.slot >= 0 ? cs[g.slot] : make_float2(1.f, 0.f), false);
                            }
#pragma unroll
                            for (int r = 0; r < kRegs; r++)
                                if (r < R) sp[swz(li.at(r))] = v[r];
                        }
                        gbar(G, w0);
                    }
                    if (!resident) {
                        chunk_store(P, base, gpsi, sp, tg);
                        gbar(G, w0);
                    }
                }
            }
            // ---------------- lambda = H psi and E = Re <psi|lambda>
            {
                DFAcc e;
                df_zero(e);
                constexpr int U = 2;
                for (uint32_t y0 = tg; y0 < N; y0 += U * nthr) {
                    float2 src[U][4];
                    float2 ps[U];
                    const int nt = it.t1 - it.t0;
#pragma unroll
                    for (int k = 0; k < U; k++) {
                        const uint32_t y = y0 + k * nthr;
                        if (y >= N) continue;
                        ps[k] = resident ? sp[swz(y)] : gpsi[y];
#pragma unroll
                        for (int t = 0; t < 4; t++)
                            if (t < nt) {
                                const uint32_t y2 = y ^ B.terms[it.t0 + t].xmask;
                                src[k][t] = resident ? sp[swz(y2)] : gpsi[y2];
                            }
                    }
#pragma unroll
                    for (int k = 0; k < U; k++) {
                        const uint32_t y = y0 + k * nthr;
                        if (y >= N) continue;
                        double re = 0.0, im = 0.0;
                        for (int t = it.t0; t < it.t1; t++) {
                            const BTerm Tm = B.terms[t];
                            const uint32_t y2 = y ^ Tm.xmask;
                            float2 v = (t - it.t0 < 4) ? src[k][min(t - it.t0, 3)] : (resident ? sp[swz(y2)] : gpsi[y2]);
                            v = mul_ipow(v, Tm.nY + 2 * (__popc(y2 & Tm.zmask) & 1));
                            re = fma(Tm.coef, double(v.x), re);
                            im = fma(Tm.coef, double(v.y), im);
                        }
                        const float2 lam = make_float2(float(re), float(im));
                        if (resident) sl[swz(y)] = lam; else glam[y] = lam;
                        df_add_prod(e, ps[k].x, lam.x);
                        df_add_prod(e, ps[k].y, lam.y);
                    }
                }
                const double ew = warp_sum(df_value(e));
                if (lane == 0) redE[warp] = ew;
                gbar(G, w0);
                if (tg == 0) {
                    double E = 0.0;
                    for (int w = w0; w < w0 + G; w++) E += redE[w];
                    B.energy[item] = E;
                }
                gbar(G, w0);
            }
            // ---------------- reverse sweep: gradient, then un-apply, gate by gate
            for (int p = it.p1 - 1; p >= it.p0; p--) {
                const BPass& P = B.passes[p];
                const uint32_t nch = resident ? 1u : (N >> kLocal);
                for (uint32_t c = 0; c < nch; c++) {
                    const uint32_t base = resident ? 0u : chunk_base(P.nonlocal, c);
                    if (!resident) {
                        chunk_load(P, base, gpsi, sp, tg);
                        chunk_load(P, base, glam, sl, tg);
                        gbar(G, w0);
                    }
                    for (int s = P.s1 - 1; s >= P.s0; s--) {
                        const BStage S = B.stages[s];
                        // every lane reaches the warp reductions; lanes beyond T hold no amplitudes
                        const bool active = tg < T;
                        LocalMap li;
                        float2 v[kRegs], u[kRegs];
                        if (active) {
                            li = stage_map(S, nl, tg);
#pragma unroll
                            for (int r = 0; r < kRegs; r++)
                                if (r < R) {
                                    v[r] = sp[swz(li.at(r))];
                                    u[r] = sl[swz(li.at(r))];
                                }
                        }
                        int slot = 0;
                        for (int gi = S.g1 - 1; gi >= S.g0; gi--) {
                            const BGate g = B.gates[gi];
                            const float2 c2 = g.slot >= 0 ? cs[g.slot] : make_float2(1.f, 0.f);
                            if (g.grad >= 0) {
                                const double gw = warp_sum(active ? grad_reg(v, u, li, R, g) : 0.0);
                                if (lane == 0) red[parity][slot][warp] = gw;
                                slot++;
                            }
                            if (active) {
                                apply_reg(v, li, R, g, c2, true);
                                apply_reg(u, li, R, g, c2, true);
                            }
                        }
                        if (active) {
#pragma unroll
                            for (int r = 0; r < kRegs; r++)
                                if (r < R) {
                                    sp[swz(li.at(r))] = v[r];
                                    sl[swz(li.at(r))] = u[r];
                                }
                        }
                        gbar(G, w0);
                        if (tg < S.nparam) {
                            // this thread owns the tg-th parametric gate of the stage (reverse order)
                            int slot = 0, gidx = -1;
                            for (int gi = S.g1 - 1; gi >= S.g0; gi--) {
                                const BGate g = B.gates[gi];
                                if (g.grad >= 0) {
                                    if (slot == tg) { gidx = g.grad; break; }
                                    slot++;
                                }
                            }
                            double sum = 0.0;
                            for (int w = w0; w < w0 + G; w++) sum += red[parity][tg][w];
                            // dE/dtheta = -Im <lambda|P|psi>
                            B.grad[it.grad0 + gidx] -= sum;
                        }
                        parity ^= 1;
                    }
                    if (!resident) {
                        chunk_store(P, base, gpsi, sp, tg);
                        chunk_store(P, base, glam, sl, tg);
                        gbar(G, w0);
                    }
                }
            }
        }
    }
}

// (cos, sin) of theta/2 for every angle slot
__global__ void k_angles(const double* __restrict__ theta, float2* __restrict__ cs, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double s, c;
        sincos(0.5 * theta[i], &s, &c);
        cs[i] = make_float2(float(c), float(s));
    }
}

}  // namespace

}  // namespace qs

// ------------------------------------------------------------------ host side
struct qs_batch {
    int count = 0;
    int total_grads = 0;
    int total_angles = 0;
    int max_n = 0;
    std::vector<qs::BItem> items;
    std::vector<int32_t> order;
    std::vector<qs::BPass> passes;
    std::vector<qs::BStage> stages;
    std::vector<qs::BGate> gates;
    std::vector<qs::BTerm> terms;
    std::vector<int32_t> angle_param;   // angle slot -> parameter index of its circuit (or -1)
    std::vector<double> angle_fixed;    // angle slot -> fixed angle (when not parametric)
    std::vector<int32_t> angle_item;    // angle slot -> item
    std::vector<int32_t> param0;        // item -> first parameter in the caller's theta array
    std::vector<int32_t> grad_of_item;  // item -> grad0
    // device buffers
    void* d_items = nullptr;
    void* d_order = nullptr;
    void* d_passes = nullptr;
    void* d_stages = nullptr;
    void* d_gates = nullptr;
    void* d_terms = nullptr;
    double* d_theta = nullptr;
    float2* d_cs = nullptr;
    float2* d_ws = nullptr;
    double* d_energy = nullptr;
    double* d_grad = nullptr;
    unsigned int* d_counter = nullptr;
    double* h_theta = nullptr;   // pinned
    double* h_energy = nullptr;  // pinned
    double* h_grad = nullptr;    // pinned
    int cls_begin[qs::kClasses + 1] = {};
    int grid = 0;
    size_t smem = 0;
    uint64_t ws_stride = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    int device = 0;
};

namespace qs {
namespace {

// split one circuit into passes over windows of <= kLocal qubits
void plan_passes(const qs_circuit& c, const std::vector<BGate>& gl, const std::vector<uint32_t>& gmask,
                 qs_batch& b, BItem& it) {
    const int n = c.n;
    const int win = std::min(n, kLocal);
    struct P {
        uint32_t mask = 0;
        std::vector<int> gates;
    };
    std::vector<P> ps;
    std::vector<int> last(n, -1);
    const uint32_t low = (1u << std::min(5, win)) - 1u;  // keep the 5 lowest qubits local: 256-byte runs
    for (size_t i = 0; i < gl.size(); i++) {
        const uint32_t m = gmask[i];
        int dep = -1;
        for (int q = 0; q < n; q++)
            if ((m >> q) & 1) dep = std::max(dep, last[q]);
        int chosen = -1;
        for (int p = std::max(dep, 0); p < int(ps.size()); p++) {
            if (p < dep) continue;
            if (__builtin_popcount(ps[p].mask | m | low) <= win) {
                chosen = p;
                break;
            }
        }
        if (chosen < 0) {
            ps.emplace_back();
            chosen = int(ps.size()) - 1;
        }
        ps[chosen].mask |= m;
        ps[chosen].gates.push_back(int(i));
        for (int q = 0; q < n; q++)
            if ((m >> q) & 1) last[q] = chosen;
    }
    if (ps.empty()) ps.emplace_back();
    it.p0 = int(b.passes.size());
    for (auto& p : ps) {
        // window: the pass's qubits, the lowest qubits, then fill with the lowest unused ones
        uint32_t w = p.mask | low;
        for (int q = 0; q < n && __builtin_popcount(w) < win; q++) w |= 1u << q;
        std::vector<int> lq;
        for (int q = 0; q < n; q++)
            if ((w >> q) & 1) lq.push_back(q);
        BPass bp;
        std::memset(&bp, 0, sizeof(bp));
        bp.nlocal = int(lq.size());
        bp.nonlocal = ((n >= 32) ? 0xffffffffu : ((1u << n) - 1u)) & ~w;
        for (int l = 0; l < 128; l++) {
            uint32_t a = 0;
            for (int j = 0; j < 7 && j < int(lq.size()); j++)
                if ((l >> j) & 1) a |= 1u << lq[j];
            bp.tab_lo[l] = a;
        }
        for (int h = 0; h < 64; h++) {
            uint32_t a = 0;
            for (int j = 0; j < 6 && 7 + j < int(lq.size()); j++)
                if ((h >> j) & 1) a |= 1u << lq[7 + j];
            bp.tab_hi[h] = a;
        }
        auto local = [&](int q) { return uint8_t(std::find(lq.begin(), lq.end(), q) - lq.begin()); };
        // stages: runs of gates whose non-diagonal targets fit a sub-cube of kRegBits local bits
        // held in registers (diagonal gates act on any bit), at most kMaxStageParams rotations
        const int nl = int(lq.size());
        const int na = std::min(kRegBits, nl);
        bp.s0 = int(b.stages.size());
        std::vector<BGate> cur;
        std::vector<int> act;
        int nparam = 0;
        auto close_stage = [&]() {
            if (cur.empty()) return;
            for (int q = 0; q < nl && int(act.size()) < na; q++)
                if (std::find(act.begin(), act.end(), q) == act.end()) act.push_back(q);
            BStage st;
            std::memset(&st, 0, sizeof(st));
            st.g0 = int(b.gates.size());
            st.nact = na;
            st.nparam = nparam;
            for (int j = 0; j < na; j++) st.act[j] = uint8_t(act[j]);
            for (BGate g : cur) {
                if (g.kind != BK_RZ && g.kind != BK_Z && g.kind != BK_CZ)
                    g.ja = uint8_t(std::find(act.begin(), act.end(), int(g.a)) - act.begin());
                b.gates.push_back(g);
            }
            st.g1 = int(b.gates.size());
            b.stages.push_back(st);
            cur.clear();
            act.clear();
            nparam = 0;
        };
        for (int gi : p.gates) {
            BGate g = gl[gi];
            g.a = local(g.a);
            if (g.kind == BK_CZ || g.kind == BK_CNOT) g.b = local(g.b);
            const bool diag = g.kind == BK_RZ || g.kind == BK_Z || g.kind == BK_CZ;
            const int par = g.grad >= 0 ? 1 : 0;
            bool fits = nparam + par <= kMaxStageParams;
            if (!diag && std::find(act.begin(), act.end(), int(g.a)) == act.end() && int(act.size()) >= na)
                fits = false;
            if (!fits) close_stage();
            if (!diag && std::find(act.begin(), act.end(), int(g.a)) == act.end()) act.push_back(g.a);
            cur.push_back(g);
            nparam += par;
        }
        close_stage();
        bp.s1 = int(b.stages.size());
        b.passes.push_back(bp);
    }
    it.p1 = int(b.passes.size());
}

void free_batch(qs_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    void* dev[] = {b->d_items, b->d_order, b->d_passes, b->d_stages, b->d_gates, b->d_terms, b->d_theta,
                   b->d_cs, b->d_ws, b->d_energy, b->d_grad, b->d_counter};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (b->h_theta) cudaFreeHost(b->h_theta);
    if (b->h_energy) cudaFreeHost(b->h_energy);
    if (b->h_grad) cudaFreeHost(b->h_grad);
}

template <typename T>
void upload(void** d, const std::vector<T>& h) {
    const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    QS_TRY_CUDA(cudaMalloc(d, bytes));
    if (!h.empty()) QS_TRY_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// enqueue one batch evaluation on `st` (used directly and under graph capture)
void enqueue(qs_batch* b, cudaStream_t st) {
    QS_TRY_CUDA(cudaMemcpyAsync(b->d_theta, b->h_theta, sizeof(double) * std::max(1, b->total_angles),
                                cudaMemcpyHostToDevice, st));
    k_angles<<<std::max(1, std::min(1024, (b->total_angles + 255) / 256)), 256, 0, st>>>(b->d_theta, b->d_cs,
                                                                                          b->total_angles);
    QS_TRY_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int) * kClasses, st));
    BatchDev B;
    B.items = static_cast<const BItem*>(b->d_items);
    B.order = static_cast<const int32_t*>(b->d_order);
    B.passes = static_cast<const BPass*>(b->d_passes);
    B.stages = static_cast<const BStage*>(b->d_stages);
    B.gates = static_cast<const BGate*>(b->d_gates);
    B.terms = static_cast<const BTerm*>(b->d_terms);
    B.cs = b->d_cs;
    B.ws = b->d_ws;
    B.ws_stride = b->ws_stride;
    B.energy = b->d_energy;
    B.grad = b->d_grad;
    B.counters = b->d_counter;
    for (int c = 0; c <= kClasses; c++) B.cls_begin[c] = b->cls_begin[c];
    k_batch<<<b->grid, kBT, b->smem, st>>>(B);
    QS_TRY_CUDA(cudaGetLastError());
    QS_TRY_CUDA(cudaMemcpyAsync(b->h_energy, b->d_energy, sizeof(double) * std::max(1, b->count),
                                cudaMemcpyDeviceToHost, st));
    QS_TRY_CUDA(cudaMemcpyAsync(b->h_grad, b->d_grad, sizeof(double) * std::max(1, b->total_grads),
                                cudaMemcpyDeviceToHost, st));
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" {

#define BATCH_BEGIN \
    try {           \
        clear_error();
#define BATCH_END                                \
    }                                            \
    catch (const Error& e) {                     \
        set_error(e.msg);                        \
        return e.code;                           \
    }                                            \
    catch (const std::bad_alloc&) {              \
        set_error("host allocation failed");     \
        return QS_ERR_OOM;                       \
    }                                            \
    catch (const std::exception& e) {            \
        set_error(e.what());                     \
        return QS_ERR_CUDA;                      \
    }                                            \
    return QS_OK;

qs_status qs_batch_create(const qs_circuit* circuits, const qs_pauli_obs* observables, int count, qs_dtype dt,
                          qs_batch** out) {
    BATCH_BEGIN
    QS_REQUIRE(out != nullptr, "null output");
    *out = nullptr;
    QS_REQUIRE(count >= 1, "batch needs at least one circuit");
    QS_REQUIRE(circuits != nullptr && observables != nullptr, "null circuits or observables");
    if (dt != QS_C64) throw Error{QS_ERR_UNSUPPORTED, "batched execution runs complex64 states"};
    std::unique_ptr<qs_batch> b(new qs_batch());
    b->count = count;
    std::vector<double> cost(count);
    int param_base = 0;
    for (int k = 0; k < count; k++) {
        const qs_circuit& c = circuits[k];
        const qs_pauli_obs& o = observables[k];
        QS_REQUIRE(c.n >= 1 && c.n <= kMaxBatchQubits, "batched circuits have 1..24 qubits");
        QS_REQUIRE(c.n_gates >= 0 && (c.n_gates == 0 || c.gates), "null gate array");
        QS_REQUIRE(c.n_params >= 0, "negative parameter count");
        b->max_n = std::max(b->max_n, c.n);
        BItem it;
        std::memset(&it, 0, sizeof(it));
        it.n = c.n;
        it.angle0 = b->total_angles;
        it.grad0 = b->total_grads;
        it.ngrad = c.n_params;
        b->param0.push_back(param_base);
        std::vector<BGate> gl;
        std::vector<uint32_t> gm;
        int slots = 0;
        for (int i = 0; i < c.n_gates; i++) {
            const qs_gate& g = c.gates[i];
            check_qubits(c.n, g.targets, g.m, g.controls, g.mc);
            BGate bg;
            std::memset(&bg, 0, sizeof(bg));
            bg.slot = -1;
            bg.grad = -1;
            bg.a = uint8_t(g.targets[0]);
            uint32_t m = 1u << g.targets[0];
            QS_REQUIRE(g.kind == QS_GATE_NAMED, "batched circuits take named gates only");
            switch (g.named) {
                case QS_NAMED_RX:
                case QS_NAMED_RY:
                case QS_NAMED_RZ:
                    QS_REQUIRE(g.mc == 0 && g.m == 1, "batched rotations act on one qubit, uncontrolled");
                    bg.kind = g.named == QS_NAMED_RX ? BK_RX : g.named == QS_NAMED_RY ? BK_RY : BK_RZ;
                    bg.slot = slots++;
                    b->angle_item.push_back(k);
                    if (g.param_index >= 0) {
                        QS_REQUIRE(g.param_index < c.n_params, "param_index out of range");
                        bg.grad = g.param_index;
                        b->angle_param.push_back(g.param_index);
                        b->angle_fixed.push_back(0.0);
                    } else {
                        b->angle_param.push_back(-1);
                        b->angle_fixed.push_back(g.params[0]);
                    }
                    break;
                case QS_NAMED_CZ:
                    QS_REQUIRE(g.m == 2 && g.mc == 0, "CZ acts on two targets");
                    bg.kind = BK_CZ;
                    bg.b = uint8_t(g.targets[1]);
                    m |= 1u << g.targets[1];
                    break;
                case QS_NAMED_CNOT:
                    QS_REQUIRE(g.m == 1 && g.mc == 1 && g.control_values[0] == 1, "CNOT has one control (value 1)");
                    bg.kind = BK_CNOT;
                    bg.b = uint8_t(g.controls[0]);
                    m |= 1u << g.controls[0];
                    break;
                case QS_NAMED_H: bg.kind = BK_H; break;
                case QS_NAMED_X: bg.kind = BK_X; break;
                case QS_NAMED_Y: bg.kind = BK_Y; break;
                case QS_NAMED_Z: bg.kind = BK_Z; break;
                default: throw Error{QS_ERR_UNSUPPORTED, "batched circuits take RX RY RZ CZ CNOT H X Y Z"};
            }
            if (g.named != QS_NAMED_CNOT) QS_REQUIRE(g.mc == 0, "only CNOT may carry a control in a batch");
            gl.push_back(bg);
            gm.push_back(m);
        }
        plan_passes(c, gl, gm, *b, it);
        // observable terms
        QS_REQUIRE(o.n_terms >= 0 && (o.n_terms == 0 || (o.coef && o.x_mask && o.z_mask)), "bad observable");
        it.t0 = int(b->terms.size());
        const uint64_t lim = (1ull << c.n) - 1;
        for (int t = 0; t < o.n_terms; t++) {
            QS_REQUIRE((o.x_mask[t] & ~lim) == 0 && (o.z_mask[t] & ~lim) == 0, "Pauli term acts on a qubit >= n");
            BTerm T;
            T.xmask = uint32_t(o.x_mask[t]);
            T.zmask = uint32_t(o.z_mask[t]);
            T.coef = o.coef[t];
            T.nY = __builtin_popcount(T.xmask & T.zmask);
            T.pad = 0;
            b->terms.push_back(T);
        }
        it.t1 = int(b->terms.size());
        b->total_angles += slots;
        b->total_grads += c.n_params;
        param_base += c.n_params;
        const double passes = double(it.p1 - it.p0);
        cost[k] = std::ldexp(1.0, c.n) * (3.0 * passes + 2.0) + 64.0 * c.n_gates;
        b->items.push_back(it);
    }
    // work classes by local width (groups of 16, 8, 4, 2, 1 warps), longest first in a class
    auto cls_of = [&](int k) {
        const int nl = std::min(b->items[k].n, kLocal);
        return nl >= 13 ? 0 : nl == 12 ? 1 : nl == 11 ? 2 : nl == 10 ? 3 : 4;
    };
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const int cx = cls_of(x), cy = cls_of(y);
        return cx != cy ? cx < cy : cost[x] > cost[y];
    });
    for (int c = 0; c <= kClasses; c++) b->cls_begin[c] = 0;
    for (int k = 0; k < count; k++) b->cls_begin[cls_of(k) + 1]++;
    for (int c = 0; c < kClasses; c++) b->cls_begin[c + 1] += b->cls_begin[c];
    QS_TRY_CUDA(cudaGetDevice(&b->device));
    int sms = 1;
    QS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, std::min(sms, count));
    b->smem = 2 * sizeof(float2) * kChunk;
    b->ws_stride = b->max_n > kLocal ? (uint64_t(1) << b->max_n) : 1;
    try {
        upload(&b->d_items, b->items);
        upload(&b->d_order, b->order);
        upload(&b->d_passes, b->passes);
        upload(&b->d_stages, b->stages);
        upload(&b->d_gates, b->gates);
        upload(&b->d_terms, b->terms);
        QS_TRY_CUDA(cudaMalloc(&b->d_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMalloc(&b->d_cs, sizeof(float2) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMalloc(&b->d_ws, sizeof(float2) * 2 * b->ws_stride * b->grid));
        QS_TRY_CUDA(cudaMalloc(&b->d_energy, sizeof(double) * count));
        QS_TRY_CUDA(cudaMalloc(&b->d_grad, sizeof(double) * std::max(1, b->total_grads)));
        QS_TRY_CUDA(cudaMalloc(&b->d_counter, sizeof(unsigned int) * kClasses));
        QS_TRY_CUDA(cudaMallocHost(&b->h_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMallocHost(&b->h_energy, sizeof(double) * count));
        QS_TRY_CUDA(cudaMallocHost(&b->h_grad, sizeof(double) * std::max(1, b->total_grads)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem)));
    } catch (...) {
        free_batch(b.get());
        throw;
    }
    *out = b.release();
    BATCH_END
}

qs_status qs_batch_info(const qs_batch* b, int* total_params, int* total_passes, size_t* workspace_bytes) {
    BATCH_BEGIN
    QS_REQUIRE(b != nullptr, "null batch");
    if (total_params) *total_params = b->total_grads;
    if (total_passes) *total_passes = int(b->passes.size());
    // (stages are reported through the pass count only)
    if (workspace_bytes) *workspace_bytes = sizeof(float2) * 2 * b->ws_stride * b->grid;
    BATCH_END
}

qs_status qs_batch_run(qs_batch* b, const double* theta, void* stream, int use_graph, double* energies,
                       double* grads) {
    BATCH_BEGIN
    QS_REQUIRE(b != nullptr && energies != nullptr, "null batch or output");
    QS_REQUIRE(b->total_grads == 0 || grads != nullptr, "null gradient output");
    // angle slots from the caller's concatenated parameters (or the gates' fixed angles)
    for (int s = 0; s < b->total_angles; s++) {
        const int p = b->angle_param[s];
        b->h_theta[s] = p >= 0 ? (theta ? theta[b->param0[b->angle_item[s]] + p] : 0.0) : b->angle_fixed[s];
    }
    QS_REQUIRE(theta != nullptr || b->total_grads == 0, "parametric batch needs theta");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (use_graph) {
        if (!b->exec) {
            QS_TRY_CUDA(cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking));
            QS_TRY_CUDA(cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal));
            try {
                enqueue(b, b->graph_stream);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->graph_stream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            QS_TRY_CUDA(cudaStreamEndCapture(b->graph_stream, &b->graph));
            QS_TRY_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        QS_TRY_CUDA(cudaGraphLaunch(b->exec, st));
    } else {
        enqueue(b, st);
    }
    QS_TRY_CUDA(cudaStreamSynchronize(st));
    std::memcpy(energies, b->h_energy, sizeof(double) * b->count);
    if (b->total_grads) std::memcpy(grads, b->h_grad, sizeof(double) * b->total_grads);
    BATCH_END
}

qs_status qs_batch_destroy(qs_batch* b) {
    BATCH_BEGIN
    if (!b) return QS_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
    BATCH_END
}

}  // extern "C"
