// Batched execution of many small parametric circuits in one persistent kernel launch,
// replayed from a CUDA graph: for every (circuit, observable) pair the energy
// E = <psi|H|psi> and the adjoint gradient dE/dtheta (reverse sweep of Sec. 4.4 parametric
// circuits, rotation convention exp(+i theta P / 2) of the paper's gate table), complex64
// storage; gradient partials are FP32 within a warp (at most 32 x 32 products) and FP64 across
// warps and chunks; the energy is a compensated (double-float) sum.
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
#include <atomic>
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
struct __align__(16) BGate {
    uint8_t kind;
    uint8_t a;      // local bit of the target
    uint8_t b;      // local bit of the second qubit (CZ) or of the control (CNOT)
    uint8_t ja;     // register bit holding the target, or kNoReg when it is not a register bit
    uint8_t jb;     // register bit holding the second qubit / control, or kNoReg
    uint8_t pad[3];
    int32_t grad;   // gradient index (parametric rotations), -1 otherwise
    float c, s;     // cos, sin of theta/2 (rotations; written before every run), else 1, 0
};
constexpr uint8_t kNoReg = 0xff;

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

enum LevelKind : int32_t { LV_FWD = 0, LV_LAMBDA = 1, LV_REV = 2, LV_FINAL = 3 };
struct LevelEntry {
    int32_t item;
    int32_t pass;                 // pass index (forward / reverse levels)
    int32_t unit0;                // first unit of this entry within the level
    int32_t kind;
};
constexpr long long kBarrierSpinLimit = 1ll << 25;  // x 256 ns sleeps: ~10 s
// test hooks of the grid barrier (kernel arguments): polls before a wait gives up, and CTA 0
// holding back its arrival at the first barrier
std::atomic<long long> g_batch_polls{kBarrierSpinLimit};
std::atomic<int> g_batch_hold{0};

struct BatchDev {
    const BItem* items;
    const int32_t* order;         // resident items grouped by class, longest first within a class
    const BPass* passes;
    const BStage* stages;
    const BGate* gates;
    const BTerm* terms;
    float2* ws;                   // psi and lambda of every circuit wider than the window
    const uint64_t* ws_off;       // item -> offset of its psi buffer (lambda follows)
    double* energy;
    double* grad;
    double* part_e;               // per wide item: energy partial per chunk
    const int64_t* part_e_off;
    double* part_g;               // per wide item: gradient partial per (parameter, chunk)
    const int64_t* part_g_off;
    const LevelEntry* lev_entries;
    const int32_t* lev_off;       // nlevels + 1
    const int32_t* lev_units;     // units per level
    int32_t nlevels;
    unsigned int* counters;       // kClasses resident counters, then one per level
    unsigned int* bar_count;
    unsigned int* bar_gen;
    int* err;
    long long barrier_polls;      // polls of a grid-barrier wait before it gives up
    int hold_cta;                 // test hook: CTA 0 does not arrive at the first grid barrier
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

// |0...0> restricted to a chunk: amplitude 1 at local index 0 of the chunk with base 0
__device__ __forceinline__ void sp_init(float2* s, uint32_t l, uint32_t base) {
    s[l ^ ((l >> 4) & 15u) ^ ((l >> 8) & 15u)] = make_float2((base == 0 && l == 0) ? 1.f : 0.f, 0.f);
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

// 2x2 update of the register pairs (r, r | 2^J) by a general complex matrix (H, X, Y)
template <int J>
__device__ __forceinline__ void pairs_1q(float2 (&v)[kRegs], int R, const M2& m) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        const int r1 = r | (1 << J);
        const float2 u = v[r], w = v[r1];
        v[r] = cfma2(m.m01, w, cfma2(m.m00, u, make_float2(0.f, 0.f)));
        v[r1] = cfma2(m.m11, w, cfma2(m.m10, u, make_float2(0.f, 0.f)));
    }
}

// RY = [[c, s], [-s, c]] (real): 8 FMA per pair
template <int J>
__device__ __forceinline__ void pairs_ry(float2 (&v)[kRegs], int R, float c, float sn) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        const int r1 = r | (1 << J);
        const float2 u = v[r], w = v[r1];
        v[r] = make_float2(fmaf(c, u.x, sn * w.x), fmaf(c, u.y, sn * w.y));
        v[r1] = make_float2(fmaf(c, w.x, -sn * u.x), fmaf(c, w.y, -sn * u.y));
    }
}

// RX = [[c, i s], [i s, c]]: 8 FMA per pair
template <int J>
__device__ __forceinline__ void pairs_rx(float2 (&v)[kRegs], int R, float c, float sn) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        const int r1 = r | (1 << J);
        const float2 u = v[r], w = v[r1];
        v[r] = make_float2(fmaf(c, u.x, -sn * w.y), fmaf(c, u.y, sn * w.x));
        v[r1] = make_float2(fmaf(c, w.x, -sn * u.y), fmaf(c, w.y, sn * u.x));
    }
}

template <int J>
__device__ __forceinline__ void pairs_kind(float2 (&v)[kRegs], int R, uint8_t kind, float c, float sn) {
    if (kind == BK_RY) pairs_ry<J>(v, R, c, sn);
    else if (kind == BK_RX) pairs_rx<J>(v, R, c, sn);
    else pairs_1q<J>(v, R, gate_m2(kind, c, sn));
}

// which of the 16 registers have local bit `bit` set: a fixed pattern when the bit is one of the
// register bits (position j), else all or none according to the thread's base
__device__ __forceinline__ uint32_t reg_mask(uint8_t j, uint32_t base, uint8_t bit) {
    const uint32_t pat[kRegBits] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};
    if (j != kNoReg) return pat[j & 3];
    return ((base >> bit) & 1u) ? 0xFFFFu : 0u;
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
__device__ __forceinline__ void pairs_cnot(float2 (&v)[kRegs], uint32_t cmask) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        const int r1 = r | (1 << J);
        if ((cmask >> r) & 1u) {
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
            const uint32_t m = reg_mask(g.ja, li.base, g.a);
#pragma unroll
            for (int r = 0; r < kRegs; r++) v[r] = cmulf(make_float2(c, ((m >> r) & 1u) ? -sn : sn), v[r]);
            break;
        }
        case BK_Z: {
            const uint32_t m = reg_mask(g.ja, li.base, g.a);
#pragma unroll
            for (int r = 0; r < kRegs; r++)
                if ((m >> r) & 1u) v[r] = make_float2(-v[r].x, -v[r].y);
            break;
        }
        case BK_CZ: {
            const uint32_t m = reg_mask(g.ja, li.base, g.a) & reg_mask(g.jb, li.base, g.b);
#pragma unroll
            for (int r = 0; r < kRegs; r++)
                if ((m >> r) & 1u) v[r] = make_float2(-v[r].x, -v[r].y);
            break;
        }
        case BK_CNOT: {
            const uint32_t m = reg_mask(g.jb, li.base, g.b);
            switch (g.ja) {
                case 0: pairs_cnot<0>(v, m); break;
                case 1: pairs_cnot<1>(v, m); break;
                case 2: pairs_cnot<2>(v, m); break;
                default: pairs_cnot<3>(v, m); break;
            }
            break;
        }
        default:
            switch (g.ja) {
                case 0: pairs_kind<0>(v, R, g.kind, c, sn); break;
                case 1: pairs_kind<1>(v, R, g.kind, c, sn); break;
                case 2: pairs_kind<2>(v, R, g.kind, c, sn); break;
                default: pairs_kind<3>(v, R, g.kind, c, sn); break;
            }
            break;
    }
}

// Im sum conj(lam) (P psi) over this thread's registers, P the axis of rotation g. The thread's
// partial (at most 32 products of complex64 data) is an FP32 FMA chain; the sums across threads,
// warps and chunks are FP64.
template <int J>
__device__ __forceinline__ void grad_pairs(const float2 (&p)[kRegs], const float2 (&l)[kRegs], int R, uint8_t kind,
                                           float& im) {
#pragma unroll
    for (int r = 0; r < kRegs; r++) {
        if ((r >> J) & 1) continue;
        const int r1 = r | (1 << J);
        const float2 a = p[r], b = p[r1], la = l[r], lb = l[r1];
        float2 p0, p1;  // X -> (b, a); Y -> (-i b, i a)
        if (kind == BK_RX) { p0 = b; p1 = a; }
        else { p0 = make_float2(b.y, -b.x); p1 = make_float2(-a.y, a.x); }
        im = fmaf(la.x, p0.y, im);
        im = fmaf(-la.y, p0.x, im);
        im = fmaf(lb.x, p1.y, im);
        im = fmaf(-lb.y, p1.x, im);
    }
}

__device__ __forceinline__ float grad_reg(const float2 (&p)[kRegs], const float2 (&l)[kRegs], const LocalMap& li,
                                          int R, const BGate& g) {
    float im = 0.f;
    if (g.kind == BK_RZ) {  // Z: (a, -b) by the target bit
        const uint32_t m = reg_mask(g.ja, li.base, g.a);
#pragma unroll
        for (int r = 0; r < kRegs; r++) {
            const float sg = ((m >> r) & 1u) ? -1.f : 1.f;
            im = fmaf(sg * l[r].x, p[r].y, im);
            im = fmaf(-sg * l[r].y, p[r].x, im);
        }
    } else {
        switch (g.ja) {
            case 0: grad_pairs<0>(p, l, R, g.kind, im); break;
            case 1: grad_pairs<1>(p, l, R, g.kind, im); break;
            case 2: grad_pairs<2>(p, l, R, g.kind, im); break;
            default: grad_pairs<3>(p, l, R, g.kind, im); break;
        }
    }
    return im;
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

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- stage bodies
// forward: registers <- slice, gates, slice <- registers
__device__ __forceinline__ void stage_forward(const BatchDev& B, const BStage& S, int nl, int tg, int T, float2* sp) {
    if (tg >= T) return;
    const LocalMap li = stage_map(S, nl, tg);
    float2 v[kRegs];
#pragma unroll
    for (int r = 0; r < kRegs; r++) v[r] = sp[swz(li.at(r))];
    BGate g = B.gates[S.g0];
    for (int gi = S.g0; gi < S.g1; gi++) {
        const BGate gn = gi + 1 < S.g1 ? B.gates[gi + 1] : g;  // prefetch
        apply_reg(v, li, kRegs, g, make_float2(g.c, g.s), false);
        g = gn;
    }
#pragma unroll
    for (int r = 0; r < kRegs; r++) sp[swz(li.at(r))] = v[r];
}

// reverse: gradient partials of the stage's rotations into red[slot][warp], un-apply from psi
// and lambda. Every lane reaches the warp reductions; lanes beyond T hold no amplitudes.
__device__ __forceinline__ void stage_reverse(const BatchDev& B, const BStage& S, int nl, int tg, int T, float2* sp,
                                              float2* sl, double (*red)[kWarps], int warp, int lane) {
    const bool active = tg < T;
    LocalMap li;
    float2 v[kRegs], u[kRegs];
    if (active) {
        li = stage_map(S, nl, tg);
#pragma unroll
        for (int r = 0; r < kRegs; r++) {
            v[r] = sp[swz(li.at(r))];
            u[r] = sl[swz(li.at(r))];
        }
    }
    int slot = 0;
    BGate g = B.gates[S.g1 - 1];
    for (int gi = S.g1 - 1; gi >= S.g0; gi--) {
        const BGate gn = gi > S.g0 ? B.gates[gi - 1] : g;  // prefetch
        const float2 c2 = make_float2(g.c, g.s);
        if (g.grad >= 0) {
            // lane partials (<= 32 FP32 products) summed in FP32 across the warp, then FP64
            const float gw = warp_sum_f(active ? grad_reg(v, u, li, kRegs, g) : 0.f);
            if (lane == 0) red[slot][warp] = double(gw);
            slot++;
        }
        if (active) {
            apply_reg(v, li, kRegs, g, c2, true);
            apply_reg(u, li, kRegs, g, c2, true);
        }
        g = gn;
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < kRegs; r++) {
            sp[swz(li.at(r))] = v[r];
            sl[swz(li.at(r))] = u[r];
        }
    }
}

// after the stage barrier: thread tg < S.nparam owns the tg-th rotation of the stage (reverse
// order); returns its gradient index and the sum of the warps' partials (fixed order)
__device__ __forceinline__ int stage_param(const BatchDev& B, const BStage& S, int tg, const double (*red)[kWarps],
                                           int w0, int G, double* sum) {
    if (tg >= S.nparam) return -1;
    int slot = 0, gidx = -1;
    for (int gi = S.g1 - 1; gi >= S.g0; gi--) {
        const int gr = B.gates[gi].grad;
        if (gr >= 0) {
            if (slot == tg) { gidx = gr; break; }
            slot++;
        }
    }
    double v = 0.0;
    for (int w = w0; w < w0 + G; w++) v += red[tg][w];
    *sum = v;
    return gidx;
}

// lambda_y = sum_t coef i^{#Y} s(y ^ f) psi_{y ^ f} for y in [y0, y1) (stride nthr), and this
// thread's share of Re <psi|lambda>; src/dst are shared slices (resident) or global buffers
template <bool RES>
__device__ __forceinline__ double lambda_range(const BatchDev& B, const BItem& it, const float2* src, float2* dst,
                                               uint32_t y0, uint32_t y1, int tg, int nthr) {
    DFAcc e;
    df_zero(e);
    const int nt = it.t1 - it.t0;
    for (uint32_t y = y0 + tg; y < y1; y += nthr) {
        float2 s4[4];
#pragma unroll
        for (int t = 0; t < 4; t++)
            if (t < nt) {
                const uint32_t y2 = y ^ B.terms[it.t0 + t].xmask;
                s4[t] = RES ? src[swz(y2)] : src[y2];
            }
        const float2 ps = RES ? src[swz(y)] : src[y];
        float re = 0.f, im = 0.f;  // lambda is stored as complex64
        for (int t = 0; t < nt; t++) {
            const BTerm Tm = B.terms[it.t0 + t];
            const uint32_t y2 = y ^ Tm.xmask;
            float2 v = t < 4 ? s4[min(t, 3)] : (RES ? src[swz(y2)] : src[y2]);
            v = mul_ipow(v, Tm.nY + 2 * (__popc(y2 & Tm.zmask) & 1));
            re = fmaf(float(Tm.coef), v.x, re);
            im = fmaf(float(Tm.coef), v.y, im);
        }
        const float2 lam = make_float2(re, im);
        if (RES) dst[swz(y)] = lam; else dst[y] = lam;
        df_add_prod(e, ps.x, lam.x);
        df_add_prod(e, ps.y, lam.y);
    }
    return df_value(e);
}

// grid-wide barrier with a bounded wait (all CTAs are co-resident: cooperative launch). On
// timeout it sets the error flag and returns false; every caller then leaves the kernel. A CTA
// told to hold back (a test of the timeout) waits without arriving, so that every wait runs out.
__device__ bool grid_barrier(unsigned int* count, unsigned int* gen, int* err, long long polls, bool hold) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = gen;
        const unsigned int g = *vgen;
        __threadfence();
        int ok = 1;
        if (!hold && atomicAdd(count, 1u) == gridDim.x - 1) {
            *count = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g) {
                if (++spins > polls || *(volatile int*)err) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok && !*(volatile int*)err;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kBT, 1) k_batch(const BatchDev B) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* smem_p = reinterpret_cast<float2*>(smem);
    float2* smem_l = smem_p + kChunk;
    __shared__ double red[2][kMaxStageParams][kWarps];  // gradient partials per stage parity
    __shared__ double redE[kWarps];
    __shared__ int s_claim[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int parity = 0;
    bool first_barrier = true;

    // ================= circuits wider than the window: level-synchronous over the grid
    for (int lv = 0; lv < B.nlevels; lv++) {
        const int total = B.lev_units[lv];
        while (true) {
            if (threadIdx.x == 0) s_claim[0] = int(atomicAdd(&B.counters[kClasses + lv], 1u));
            __syncthreads();
            const int u = s_claim[0];
            __syncthreads();
            if (u >= total) break;
            // entry of this unit: last entry with unit0 <= u
            int lo = B.lev_off[lv], hi = B.lev_off[lv + 1] - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (B.lev_entries[mid].unit0 <= u) lo = mid; else hi = mid - 1;
            }
            const LevelEntry E = B.lev_entries[lo];
            const int item = E.item;
            const BItem it = B.items[item];
            const uint32_t c = uint32_t(u - E.unit0);
            const uint32_t nch = 1u << (it.n - kLocal);
            float2* gpsi = B.ws + B.ws_off[item];
            float2* glam = gpsi + (uint64_t(1) << it.n);
            const int tg = threadIdx.x;
            if (E.kind == LV_FWD) {
                const BPass& P = B.passes[E.pass];
                const uint32_t base = chunk_base(P.nonlocal, c);
                if (E.pass == it.p0) {
                    for (uint32_t l = tg; l < kChunk; l += kBT) sp_init(smem_p, l, base);
                } else {
                    chunk_load(P, base, gpsi, smem_p, tg);
                }
                __syncthreads();
                for (int s = P.s0; s < P.s1; s++) {
                    stage_forward(B, B.stages[s], kLocal, tg, kBT, smem_p);
                    __syncthreads();
                }
                chunk_store(P, base, gpsi, smem_p, tg);
                __syncthreads();
            } else if (E.kind == LV_LAMBDA) {
                const uint32_t y0 = c << kLocal;
                const double ew = warp_sum(lambda_range<false>(B, it, gpsi, glam, y0, y0 + kChunk, tg, kBT));
                if (lane == 0) redE[warp] = ew;
                __syncthreads();
                if (tg == 0) {
                    double e = 0.0;
                    for (int w = 0; w < kWarps; w++) e += redE[w];
                    B.part_e[B.part_e_off[item] + c] = e;
                }
                __syncthreads();
            } else if (E.kind == LV_REV) {
                const BPass& P = B.passes[E.pass];
                const uint32_t base = chunk_base(P.nonlocal, c);
                chunk_load(P, base, gpsi, smem_p, tg);
                chunk_load(P, base, glam, smem_l, tg);
                __syncthreads();
                double* pg = B.part_g + B.part_g_off[item];
                for (int s = P.s1 - 1; s >= P.s0; s--) {
                    const BStage S = B.stages[s];
                    stage_reverse(B, S, kLocal, tg, kBT, smem_p, smem_l, red[parity], warp, lane);
                    __syncthreads();
                    double sum;
                    const int gidx = stage_param(B, S, tg, red[parity], 0, kWarps, &sum);
                    if (gidx >= 0) pg[size_t(gidx) * nch + c] -= sum;  // dE/dtheta = -Im <lambda|P|psi>
                    parity ^= 1;
                }
                chunk_store(P, base, gpsi, smem_p, tg);
                chunk_store(P, base, glam, smem_l, tg);
                __syncthreads();
            } else {  // LV_FINAL: energy and gradients of the item, sums in chunk order
                if (tg == 0) {
                    double e = 0.0;
                    for (uint32_t k = 0; k < nch; k++) e += B.part_e[B.part_e_off[item] + k];
                    B.energy[item] = e;
                }
                const double* pg = B.part_g + B.part_g_off[item];
                for (int j = tg; j < it.ngrad; j += kBT) {
                    double gsum = 0.0;
                    for (uint32_t k = 0; k < nch; k++) gsum += pg[size_t(j) * nch + k];
                    B.grad[it.grad0 + j] = gsum;
                }
                __syncthreads();
            }
        }
        if (!grid_barrier(B.bar_count, B.bar_gen, B.err, B.barrier_polls, B.hold_cta && blockIdx.x == 0 && first_barrier))
            return;
        first_barrier = false;
    }

    // ================= circuits within the window: whole circuit per warp group, in shared memory
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
            const int nl = it.n;
            const uint32_t size = 1u << nl;
            const int T = int(size) / kRegs;
            for (int j = tg; j < it.ngrad; j += nthr) B.grad[it.grad0 + j] = 0.0;
            for (uint32_t l = tg; l < size; l += nthr) sp_init(sp, l, 0u);
            gbar(G, w0);
            const BPass& P = B.passes[it.p0];  // one pass holds the whole circuit
            for (int s = P.s0; s < P.s1; s++) {
                stage_forward(B, B.stages[s], nl, tg, T, sp);
                gbar(G, w0);
            }
            {
                const double ew = warp_sum(lambda_range<true>(B, it, sp, sl, 0u, size, tg, nthr));
                if (lane == 0) redE[warp] = ew;
                gbar(G, w0);
                if (tg == 0) {
                    double E = 0.0;
                    for (int w = w0; w < w0 + G; w++) E += redE[w];
                    B.energy[item] = E;
                }
                gbar(G, w0);
            }
            for (int s = P.s1 - 1; s >= P.s0; s--) {
                const BStage S = B.stages[s];
                stage_reverse(B, S, nl, tg, T, sp, sl, red[parity], warp, lane);
                gbar(G, w0);
                double sum;
                const int gidx = stage_param(B, S, tg, red[parity], w0, G, &sum);
                if (gidx >= 0) B.grad[it.grad0 + gidx] -= sum;
                parity ^= 1;
            }
        }
    }
}

// (cos, sin) of theta/2 into every rotation's gate record
__global__ void k_angles(const double* __restrict__ theta, const int32_t* __restrict__ gate_slot,
                         BGate* __restrict__ gates, int ng) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const int sl = gate_slot[i];
        if (sl < 0) continue;
        double s, c;
        sincos(0.5 * theta[sl], &s, &c);
        gates[i].c = float(c);
        gates[i].s = float(s);
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
    std::vector<int32_t> gate_slot;     // emitted gate -> absolute angle slot (or -1)
    std::vector<qs::BTerm> terms;
    std::vector<int32_t> angle_param;   // angle slot -> parameter index of its circuit (or -1)
    std::vector<double> angle_fixed;    // angle slot -> fixed angle (when not parametric)
    std::vector<int32_t> angle_item;    // angle slot -> item
    std::vector<int32_t> param0;        // item -> first parameter in the caller's theta array
    std::vector<int32_t> grad_of_item;  // item -> grad0
    // circuits wider than the window: buffers and levels
    std::vector<uint64_t> ws_off;       // item -> psi offset (amplitudes)
    std::vector<int64_t> part_e_off, part_g_off;
    std::vector<qs::LevelEntry> lev_entries;
    std::vector<int32_t> lev_off, lev_units;
    uint64_t ws_amps = 0;
    int64_t part_e_total = 0, part_g_total = 0;
    // device buffers
    void* d_items = nullptr;
    void* d_order = nullptr;
    void* d_passes = nullptr;
    void* d_stages = nullptr;
    void* d_gates = nullptr;
    void* d_gate_slot = nullptr;
    void* d_terms = nullptr;
    double* d_theta = nullptr;
    float2* d_ws = nullptr;
    void* d_ws_off = nullptr;
    double* d_part_e = nullptr;
    void* d_part_e_off = nullptr;
    double* d_part_g = nullptr;
    void* d_part_g_off = nullptr;
    void* d_lev_entries = nullptr;
    void* d_lev_off = nullptr;
    void* d_lev_units = nullptr;
    unsigned int* d_bar = nullptr;    // count, generation
    int* d_err = nullptr;
    int* h_err = nullptr;             // pinned
    double* d_energy = nullptr;
    double* d_grad = nullptr;
    unsigned int* d_counter = nullptr;
    double* h_theta = nullptr;   // pinned
    double* h_energy = nullptr;  // pinned
    double* h_grad = nullptr;    // pinned
    int cls_begin[qs::kClasses + 1] = {};
    int grid = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    long long graph_polls = 0;   // wait-test settings the graph was captured with
    int graph_hold = 0;
    int device = 0;
};

namespace qs {
namespace {

// split one circuit into passes over windows of <= kLocal qubits
void plan_passes(const qs_circuit& c, const std::vector<BGate>& gl, const std::vector<uint32_t>& gmask,
                 const std::vector<int32_t>& gslot,
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
        std::vector<int32_t> cur_slot;
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
            auto regpos = [&](int bit) {
                const auto f = std::find(act.begin(), act.end(), bit);
                return f == act.end() ? kNoReg : uint8_t(f - act.begin());
            };
            for (size_t q = 0; q < cur.size(); q++) {
                BGate g = cur[q];
                g.ja = regpos(g.a);
                g.jb = (g.kind == BK_CZ || g.kind == BK_CNOT) ? regpos(g.b) : kNoReg;
                b.gates.push_back(g);
                b.gate_slot.push_back(cur_slot[q]);
            }
            st.g1 = int(b.gates.size());
            b.stages.push_back(st);
            cur.clear();
            cur_slot.clear();
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
            cur_slot.push_back(gslot[gi]);
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
    void* dev[] = {b->d_items, b->d_order, b->d_passes, b->d_stages, b->d_gates, b->d_gate_slot, b->d_terms,
                   b->d_theta, b->d_ws, b->d_ws_off, b->d_part_e, b->d_part_e_off, b->d_part_g, b->d_part_g_off,
                   b->d_lev_entries, b->d_lev_off, b->d_lev_units, b->d_bar, b->d_err, b->d_energy, b->d_grad,
                   b->d_counter};
    for (void* p : dev)
        if (p) dev_free(p);
    if (b->h_theta) host_free_pinned(b->h_theta);
    if (b->h_energy) host_free_pinned(b->h_energy);
    if (b->h_grad) host_free_pinned(b->h_grad);
    if (b->h_err) host_free_pinned(b->h_err);
}

template <typename T>
void upload(void** d, const std::vector<T>& h) {
    const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    QS_TRY_CUDA(dev_malloc(d, bytes));
    if (!h.empty()) QS_TRY_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// enqueue one batch evaluation on `st` (used directly and under graph capture)
void enqueue(qs_batch* b, cudaStream_t st) {
    QS_TRY_CUDA(cudaMemcpyAsync(b->d_theta, b->h_theta, sizeof(double) * std::max(1, b->total_angles),
                                cudaMemcpyHostToDevice, st));
    const int ng = int(b->gates.size());
    k_angles<<<std::max(1, std::min(1024, (ng + 255) / 256)), 256, 0, st>>>(
        b->d_theta, static_cast<const int32_t*>(b->d_gate_slot), static_cast<BGate*>(b->d_gates), ng);
    const int nlev = int(b->lev_units.size());
    QS_TRY_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int) * (kClasses + nlev), st));
    QS_TRY_CUDA(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned int) * 2, st));
    QS_TRY_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), st));
    if (b->part_g_total) QS_TRY_CUDA(cudaMemsetAsync(b->d_part_g, 0, sizeof(double) * b->part_g_total, st));
    BatchDev B;
    B.items = static_cast<const BItem*>(b->d_items);
    B.order = static_cast<const int32_t*>(b->d_order);
    B.passes = static_cast<const BPass*>(b->d_passes);
    B.stages = static_cast<const BStage*>(b->d_stages);
    B.gates = static_cast<const BGate*>(b->d_gates);
    B.terms = static_cast<const BTerm*>(b->d_terms);
    B.ws = b->d_ws;
    B.ws_off = static_cast<const uint64_t*>(b->d_ws_off);
    B.energy = b->d_energy;
    B.grad = b->d_grad;
    B.part_e = b->d_part_e;
    B.part_e_off = static_cast<const int64_t*>(b->d_part_e_off);
    B.part_g = b->d_part_g;
    B.part_g_off = static_cast<const int64_t*>(b->d_part_g_off);
    B.lev_entries = static_cast<const LevelEntry*>(b->d_lev_entries);
    B.lev_off = static_cast<const int32_t*>(b->d_lev_off);
    B.lev_units = static_cast<const int32_t*>(b->d_lev_units);
    B.nlevels = nlev;
    B.counters = b->d_counter;
    B.bar_count = b->d_bar;
    B.bar_gen = b->d_bar + 1;
    B.err = b->d_err;
    B.barrier_polls = g_batch_polls.load();
    B.hold_cta = g_batch_hold.load();
    for (int c = 0; c <= kClasses; c++) B.cls_begin[c] = b->cls_begin[c];
    // cooperative launch: every CTA is resident at once, so the grid barrier cannot wait on a
    // CTA that never runs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    QS_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_batch, B));
    QS_TRY_CUDA(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
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
        QS_REQUIRE(c.n >= 4 && c.n <= kMaxBatchQubits, "batched circuits have 4..24 qubits");
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
        std::vector<int32_t> gs;  // absolute angle slot of each gate (-1: none)
        int slots = 0;
        for (int i = 0; i < c.n_gates; i++) {
            const qs_gate& g = c.gates[i];
            check_qubits(c.n, g.targets, g.m, g.controls, g.mc);
            BGate bg;
            std::memset(&bg, 0, sizeof(bg));
            bg.grad = -1;
            bg.c = 1.f;
            bg.s = 0.f;
            int32_t aslot = -1;
            bg.a = uint8_t(g.targets[0]);
            uint32_t m = 1u << g.targets[0];
            QS_REQUIRE(g.kind == QS_GATE_NAMED, "batched circuits take named gates only");
            switch (g.named) {
                case QS_NAMED_RX:
                case QS_NAMED_RY:
                case QS_NAMED_RZ:
                    QS_REQUIRE(g.mc == 0 && g.m == 1, "batched rotations act on one qubit, uncontrolled");
                    bg.kind = g.named == QS_NAMED_RX ? BK_RX : g.named == QS_NAMED_RY ? BK_RY : BK_RZ;
                    aslot = b->total_angles + slots++;
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
            gs.push_back(aslot);
        }
        plan_passes(c, gl, gm, gs, *b, it);
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
    // circuits within the window: work classes by width (groups of 16, 8, 4, 2, 1 warps),
    // longest first in a class; wider circuits (class kClasses) go through the levels instead
    auto cls_of = [&](int k) {
        const int n = b->items[k].n;
        if (n > kLocal) return kClasses;
        return n == 13 ? 0 : n == 12 ? 1 : n == 11 ? 2 : n == 10 ? 3 : 4;
    };
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const int cx = cls_of(x), cy = cls_of(y);
        return cx != cy ? cx < cy : cost[x] > cost[y];
    });
    for (int c = 0; c <= kClasses; c++) b->cls_begin[c] = 0;
    for (int k = 0; k < count; k++)
        if (cls_of(k) < kClasses) b->cls_begin[cls_of(k) + 1]++;
    for (int c = 0; c < kClasses; c++) b->cls_begin[c + 1] += b->cls_begin[c];
    QS_TRY_CUDA(cudaGetDevice(&b->device));
    int sms = 1;
    QS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->smem = 2 * sizeof(float2) * kChunk;
    QS_TRY_CUDA(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem)));
    int per_sm = 0;
    QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kBT, b->smem));
    if (per_sm < 1) throw Error{QS_ERR_UNSUPPORTED, "batch kernel does not fit on an SM"};
    b->grid = sms * per_sm;  // all co-resident (cooperative launch)
    // circuits wider than the window get their own psi / lambda buffers and partial-sum slots,
    // and their passes become levels shared by the whole grid
    b->ws_off.assign(count, 0);
    b->part_e_off.assign(count, 0);
    b->part_g_off.assign(count, 0);
    int maxp = 0;
    std::vector<int> wide;
    for (int k = 0; k < count; k++) {
        const BItem& it = b->items[k];
        if (it.n <= kLocal) continue;
        wide.push_back(k);
        const int64_t nch = int64_t(1) << (it.n - kLocal);
        b->ws_off[k] = b->ws_amps;
        b->ws_amps += 2 * (uint64_t(1) << it.n);
        b->part_e_off[k] = b->part_e_total;
        b->part_e_total += nch;
        b->part_g_off[k] = b->part_g_total;
        b->part_g_total += nch * it.ngrad;
        maxp = std::max(maxp, it.p1 - it.p0);
    }
    // longest circuits first inside every level
    std::stable_sort(wide.begin(), wide.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    auto add_level = [&](int kind, int r) {
        int units = 0;
        b->lev_off.push_back(int(b->lev_entries.size()));
        for (int k : wide) {
            const BItem& it = b->items[k];
            const int np_ = it.p1 - it.p0;
            const int nch = 1 << (it.n - kLocal);
            LevelEntry e;
            e.item = k;
            e.kind = kind;
            e.unit0 = units;
            if (kind == LV_FWD) {
                if (r >= np_) continue;
                e.pass = it.p0 + r;
                units += nch;
            } else if (kind == LV_REV) {
                if (r >= np_) continue;
                e.pass = it.p1 - 1 - r;
                units += nch;
            } else if (kind == LV_LAMBDA) {
                e.pass = -1;
                units += nch;
            } else {
                e.pass = -1;
                units += 1;
            }
            b->lev_entries.push_back(e);
        }
        b->lev_units.push_back(units);
    };
    if (!wide.empty()) {
        for (int r = 0; r < maxp; r++) add_level(LV_FWD, r);
        add_level(LV_LAMBDA, 0);
        for (int r = 0; r < maxp; r++) add_level(LV_REV, r);
        add_level(LV_FINAL, 0);
        b->lev_off.push_back(int(b->lev_entries.size()));
    } else {
        b->lev_off.push_back(0);
    }
    try {
        upload(&b->d_items, b->items);
        upload(&b->d_order, b->order);
        upload(&b->d_passes, b->passes);
        upload(&b->d_stages, b->stages);
        upload(&b->d_gates, b->gates);
        upload(&b->d_gate_slot, b->gate_slot);
        upload(&b->d_terms, b->terms);
        QS_TRY_CUDA(dev_malloc(&b->d_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(dev_malloc(&b->d_ws, sizeof(float2) * std::max<uint64_t>(1, b->ws_amps)));
        upload(&b->d_ws_off, b->ws_off);
        upload(&b->d_part_e_off, b->part_e_off);
        upload(&b->d_part_g_off, b->part_g_off);
        QS_TRY_CUDA(dev_malloc(&b->d_part_e, sizeof(double) * std::max<int64_t>(1, b->part_e_total)));
        QS_TRY_CUDA(dev_malloc(&b->d_part_g, sizeof(double) * std::max<int64_t>(1, b->part_g_total)));
        upload(&b->d_lev_entries, b->lev_entries);
        upload(&b->d_lev_off, b->lev_off);
        upload(&b->d_lev_units, b->lev_units);
        QS_TRY_CUDA(dev_malloc(&b->d_bar, sizeof(unsigned int) * 2));
        QS_TRY_CUDA(dev_malloc(&b->d_err, sizeof(int)));
        QS_TRY_CUDA(host_malloc_pinned(&b->h_err, sizeof(int)));
        QS_TRY_CUDA(dev_malloc(&b->d_energy, sizeof(double) * count));
        QS_TRY_CUDA(dev_malloc(&b->d_grad, sizeof(double) * std::max(1, b->total_grads)));
        QS_TRY_CUDA(dev_malloc(&b->d_counter, sizeof(unsigned int) * (kClasses + b->lev_units.size())));
        QS_TRY_CUDA(host_malloc_pinned(&b->h_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(host_malloc_pinned(&b->h_energy, sizeof(double) * count));
        QS_TRY_CUDA(host_malloc_pinned(&b->h_grad, sizeof(double) * std::max(1, b->total_grads)));
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
    if (workspace_bytes)
        *workspace_bytes = sizeof(float2) * b->ws_amps + sizeof(double) * size_t(b->part_e_total + b->part_g_total);
    BATCH_END
}

qs_status qs_batch_traffic(const qs_batch* b, double* bytes) {
    BATCH_BEGIN
    QS_REQUIRE(b != nullptr && bytes != nullptr, "null batch or output");
    // circuits wider than the window: the first forward pass writes psi (it starts from |0..0> in
    // shared memory), every later one reads and writes it; lambda = H psi reads psi and writes
    // lambda; every reverse pass reads and writes both. Narrower circuits stay in shared memory.
    double total = 0.0;
    for (const BItem& it : b->items) {
        if (it.n <= kLocal) continue;
        const double amp = 8.0 * std::ldexp(1.0, it.n);  // complex64
        const int np_ = it.p1 - it.p0;
        if (np_ > 0) total += amp + 2.0 * amp * (np_ - 1);
        total += 2.0 * amp + 4.0 * amp * np_;
    }
    *bytes = total;
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
        if (b->exec && (b->graph_polls != g_batch_polls.load() || b->graph_hold != g_batch_hold.load())) {
            // the wait-test settings are kernel arguments: a graph captured under others is redone
            QS_TRY_CUDA(cudaStreamSynchronize(b->graph_stream));
            cudaGraphExecDestroy(b->exec);
            cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = nullptr;
        }
        if (!b->exec) {
            b->graph_polls = g_batch_polls.load();
            b->graph_hold = g_batch_hold.load();
            if (!b->graph_stream) QS_TRY_CUDA(cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking));
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
    if (*b->h_err) throw Error{QS_ERR_TIMEOUT, "batch kernel: a grid barrier wait ran out (work abandoned)"};
    std::memcpy(energies, b->h_energy, sizeof(double) * b->count);
    if (b->total_grads) std::memcpy(grads, b->h_grad, sizeof(double) * b->total_grads);
    BATCH_END
}

}  // extern "C"

namespace qs {
void batch_set_wait_polls(long long polls) { g_batch_polls.store(polls < 0 ? kBarrierSpinLimit : polls); }
void batch_set_hold_cta(bool on) { g_batch_hold.store(on ? 1 : 0); }
}  // namespace qs

extern "C" {

qs_status qs_batch_destroy(qs_batch* b) {
    BATCH_BEGIN
    if (!b) return QS_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
    BATCH_END
}

}  // extern "C"
