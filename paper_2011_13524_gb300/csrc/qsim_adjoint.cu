// Fused reverse step of the adjoint gradient for a single-qubit rotation
// R_P(theta) = exp(+i theta P / 2), P in {X, Y, Z} (the paper's gate table sign).
//
// At gate j of the reverse sweep psi holds psi_j (the state after the gate) and lambda holds
// lambda_j = U_{j+1}^+ ... U_G^+ H psi_G. Then dE/dtheta_j = -Im <lambda_j|P|psi_j>; afterwards
// both buffers are multiplied by R_P(theta)^+. One pass over the qubit's amplitude pairs does
// both: each pair contributes conj(lambda) * (P psi) to the block's partial sum, then the 2x2
// adjoint is applied to the pair in psi and in lambda. Per-block partials land in their own
// slots (deterministic); one final kernel reduces every gate's slots.
#include <algorithm>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kAdjThreads = 256;

// accumulators of conj(l) * p for each arithmetic policy, FP64-class in all three
template <typename P>
struct GradAcc;

template <>
struct GradAcc<NativeArith<double>> {
    double re = 0.0, im = 0.0;
    __device__ void add(double2 l, double2 p) {
        re = fma(l.x, p.x, re);
        re = fma(l.y, p.y, re);
        im = fma(l.x, p.y, im);
        im = fma(-l.y, p.x, im);
    }
    __device__ double imag() const { return im; }
};

template <>
struct GradAcc<NativeArith<float>> {
    DFAcc im;
    __device__ GradAcc() { df_zero(im); }
    __device__ void add(float2 l, float2 p) {
        df_add_prod(im, l.x, p.y);
        df_add_prod(im, -l.y, p.x);
    }
    __device__ double imag() const { return df_value(im); }
};

template <>
struct GradAcc<DFArith> {
    float s = 0.f, c = 0.f;  // imaginary part only: lx py - ly px
    __device__ void add(float4 l, float4 p) {
        DFArith::dprod(s, c, l.x, l.y, p.z, p.w);
        DFArith::dprod(s, c, -l.z, -l.w, p.x, p.y);
    }
    __device__ double imag() const { return double(s) + double(c); }
};

// the imaginary part of an FP32-pair gradient accumulator as its unevaluated pair (s, c)
__device__ __forceinline__ void acc_pair(const GradAcc<DFArith>& g, float& s, float& c) {
    s = g.s;
    c = g.c;
}
__device__ __forceinline__ void acc_pair(const GradAcc<NativeArith<float>>& g, float& s, float& c) {
    s = g.im.hi;
    c = g.im.lo;
}

// Block sums of NR gradient partials, to part[r * gridDim.x + blockIdx.x]. FP32-pair
// accumulators are summed as FP32 pairs (TwoSum) across each warp and then across the eight warp
// sums, and converted to FP64 once per block: on GB300 FP64 warp stages (or a conversion in every
// lane) cost microseconds per launch. FP64 accumulators keep FP64 sums. One barrier for all NR
// sums; the order is fixed, so results are reproducible.
__device__ __forceinline__ void pair_sum_down(float& s, float& c, int o) {
    const float os = __shfl_down_sync(0xffffffffu, s, o), oc = __shfl_down_sync(0xffffffffu, c, o);
    float h, e;
    DFArith::two_sum(s, os, h, e);
    s = h;
    c = __fadd_rn(c, __fadd_rn(oc, e));
}
template <typename P, int NR>
__device__ __forceinline__ void grad_block_sums(const GradAcc<P> (&g)[NR], double* part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int W = kAdjThreads / 32;
    if constexpr (std::is_same<P, NativeArith<double>>::value) {
        __shared__ double sh[NR][W];
#pragma unroll
        for (int r = 0; r < NR; r++) {
            double v = g[r].imag();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[r][wid] = v;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int r = 0; r < NR; r++) {
                double v = lane < W ? sh[r][lane] : 0.0;
#pragma unroll
                for (int o = W / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) part[size_t(r) * gridDim.x + blockIdx.x] = v;
            }
        }
    } else {
        __shared__ float2 sh[NR][W];
#pragma unroll
        for (int r = 0; r < NR; r++) {
            float s, c;
            acc_pair(g[r], s, c);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pair_sum_down(s, c, o);
            if (lane == 0) sh[r][wid] = make_float2(s, c);
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const float2 v = lane < W ? sh[r][lane] : make_float2(0.f, 0.f);
                float s = v.x, c = v.y;
#pragma unroll
                for (int o = W / 2; o > 0; o >>= 1) pair_sum_down(s, c, o);
                if (lane == 0) part[size_t(r) * gridDim.x + blockIdx.x] = double(s) + double(c);
            }
        }
    }
}

template <typename P>
struct AdjRotParams {
    IndexPlan ip;            // pivot bit = the rotation's qubit
    uint64_t bit;            // 1 << qubit
    typename P::K U[4];      // R^+ as a 2x2 matrix, row-major
    int32_t axis;            // 1 = X, 2 = Y, 3 = Z
};

template <typename P>
__global__ void __launch_bounds__(kAdjThreads) k_adj_rot(typename P::C* __restrict__ psi, typename P::C* __restrict__ lam,
                                                          const __grid_constant__ AdjRotParams<P> A, double* part) {
    using C = typename P::C;
    GradAcc<P> g;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < A.ip.n_iter; i += stride) {
        const uint64_t i0 = expand(i, A.ip), i1 = i0 | A.bit;
        const C a = psi[i0], b = psi[i1], la = lam[i0], lb = lam[i1];
        // (P psi) on the pair: X -> (b, a); Y -> (-i b, i a); Z -> (a, -b)
        if (A.axis == 1) {
            g.add(la, b);
            g.add(lb, a);
        } else if (A.axis == 2) {
            g.add(la, P::ipow(b, 3));
            g.add(lb, P::ipow(a, 1));
        } else {
            g.add(la, a);
            g.add(lb, P::ipow(b, 2));
        }
        typename P::Acc r0 = P::zero(), r1 = P::zero(), s0 = P::zero(), s1 = P::zero();
        P::mac(r0, A.U[0], a); P::mac(r0, A.U[1], b);
        P::mac(r1, A.U[2], a); P::mac(r1, A.U[3], b);
        P::mac(s0, A.U[0], la); P::mac(s0, A.U[1], lb);
        P::mac(s1, A.U[2], la); P::mac(s1, A.U[3], lb);
        psi[i0] = P::out(r0);
        psi[i1] = P::out(r1);
        lam[i0] = P::out(s0);
        lam[i1] = P::out(s1);
    }
    const GradAcc<P> ga[1] = {g};
    grad_block_sums<P, 1>(ga, part);
}

// NR consecutive reverse steps (2 to 4) for rotations on distinct qubits q_0 (the latest in the
// circuit), q_1, ...: each group of 2^NR amplitudes (bits q_0..q_{NR-1}) gets, rotation by
// rotation in that order, the gradient partial of rotation r and the un-apply of R_r, all in
// registers. (The rotations commute, so each gradient is the same whichever others are already
// un-applied.) Partials of rotation r go to part[r grid .. (r + 1) grid).
template <typename P, int NR>
struct AdjRotNParams {
    IndexPlan ip;            // the NR bits inserted
    uint64_t bit[NR];        // 1 << q_r
    typename P::K U[NR][4];  // R_r^+
    int32_t axis[NR];
};

template <typename P>
__device__ __forceinline__ void rot_step(typename P::C& a, typename P::C& b, typename P::C& la, typename P::C& lb,
                                         int axis, const typename P::K* U, GradAcc<P>& g) {
    if (axis == 1) {
        g.add(la, b);
        g.add(lb, a);
    } else if (axis == 2) {
        g.add(la, P::ipow(b, 3));
        g.add(lb, P::ipow(a, 1));
    } else {
        g.add(la, a);
        g.add(lb, P::ipow(b, 2));
    }
    typename P::Acc r0 = P::first(U[0], a), r1 = P::first(U[2], a), s0 = P::first(U[0], la), s1 = P::first(U[2], la);
    P::mac(r0, U[1], b);
    P::mac(r1, U[3], b);
    P::mac(s0, U[1], lb);
    P::mac(s1, U[3], lb);
    a = P::out(r0);
    b = P::out(r1);
    la = P::out(s0);
    lb = P::out(s1);
}

// The double-float update of a pair by R^+ for X or Y axes, whose entries are real multiples of
// 1 and i (X: [[c, -i s], [-i s, c]]; Y: [[c, -s], [s, c]]): every output component is a sum of
// two real products, formed as one double-float dot product (the general 2 x 2 complex form
// costs twice the products, half of them by zero). Z axes keep the general form.
__device__ __forceinline__ void df_dot_re(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                          float dl, float& h, float& l) {
    float s, c;
    DFArith::dprod0(s, c, ah, al, bh, bl);
    DFArith::dprod(s, c, ch, cl, dh, dl);
    DFArith::two_sum(s, c, h, l);
}
__device__ __forceinline__ void df_rot_pair(float4& a, float4& b, int axis, float ch, float cl, float sh, float sl) {
    float4 ra, rb;
    if (axis == 1) {  // a' = c a - i s b, b' = -i s a + c b
        df_dot_re(ch, cl, a.x, a.y, sh, sl, b.z, b.w, ra.x, ra.y);
        df_dot_re(ch, cl, a.z, a.w, -sh, -sl, b.x, b.y, ra.z, ra.w);
        df_dot_re(sh, sl, a.z, a.w, ch, cl, b.x, b.y, rb.x, rb.y);
        df_dot_re(-sh, -sl, a.x, a.y, ch, cl, b.z, b.w, rb.z, rb.w);
    } else {  // a' = c a - s b, b' = s a + c b
        df_dot_re(ch, cl, a.x, a.y, -sh, -sl, b.x, b.y, ra.x, ra.y);
        df_dot_re(ch, cl, a.z, a.w, -sh, -sl, b.z, b.w, ra.z, ra.w);
        df_dot_re(sh, sl, a.x, a.y, ch, cl, b.x, b.y, rb.x, rb.y);
        df_dot_re(sh, sl, a.z, a.w, ch, cl, b.z, b.w, rb.z, rb.w);
    }
    a = ra;
    b = rb;
}
template <>
__device__ __forceinline__ void rot_step<DFArith>(float4& a, float4& b, float4& la, float4& lb, int axis,
                                                  const float4* U, GradAcc<DFArith>& g) {
    if (axis == 3) {  // general form
        g.add(la, a);
        g.add(lb, DFArith::ipow(b, 2));
        DFArith::Acc r0 = DFArith::first(U[0], a), r1 = DFArith::first(U[2], a), s0 = DFArith::first(U[0], la),
                     s1 = DFArith::first(U[2], la);
        DFArith::mac(r0, U[1], b);
        DFArith::mac(r1, U[3], b);
        DFArith::mac(s0, U[1], lb);
        DFArith::mac(s1, U[3], lb);
        a = DFArith::out(r0);
        b = DFArith::out(r1);
        la = DFArith::out(s0);
        lb = DFArith::out(s1);
        return;
    }
    if (axis == 1) {
        g.add(la, b);
        g.add(lb, a);
    } else {
        g.add(la, DFArith::ipow(b, 3));
        g.add(lb, DFArith::ipow(a, 1));
    }
    // c = Re U[0]; s = -Im U[1] (X) or -Re U[1] (Y)
    const float ch = U[0].x, cl = U[0].y;
    const float sh = axis == 1 ? -U[1].z : -U[1].x, sl = axis == 1 ? -U[1].w : -U[1].y;
    df_rot_pair(a, b, axis, ch, cl, sh, sl);
    df_rot_pair(la, lb, axis, ch, cl, sh, sl);
}

// Four CTAs per SM (64 registers; a few bytes spill): 8.37 -> 8.05 ms for the n = 20 HEA gradient.
template <typename P, int NR>
__global__ void __launch_bounds__(kAdjThreads, 4) k_adj_rotn(typename P::C* __restrict__ psi, typename P::C* __restrict__ lam,
                                                           const __grid_constant__ AdjRotNParams<P, NR> A, double* part) {
    using C = typename P::C;
    constexpr int E = 1 << NR;
    GradAcc<P> g[NR];
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < A.ip.n_iter; i += stride) {
        const uint64_t i0 = expand(i, A.ip);
        uint64_t ix[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            uint64_t x = i0;
#pragma unroll
            for (int r = 0; r < NR; r++)
                if ((e >> r) & 1) x |= A.bit[r];
            ix[e] = x;
        }
        C v[E], l[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            v[e] = psi[ix[e]];
            l[e] = lam[ix[e]];
        }
#pragma unroll
        for (int r = 0; r < NR; r++)
#pragma unroll
            for (int e = 0; e < E; e++)
                if (!((e >> r) & 1)) rot_step<P>(v[e], v[e | (1 << r)], l[e], l[e | (1 << r)], A.axis[r], A.U[r], g[r]);
#pragma unroll
        for (int e = 0; e < E; e++) {
            psi[ix[e]] = v[e];
            lam[ix[e]] = l[e];
        }
    }
    grad_block_sums<P, NR>(g, part);
}

// out[s] = sum of part[s * nb .. s * nb + nb) in a fixed order, one block per slot
__global__ void __launch_bounds__(kAdjThreads) k_slot_sums(const double* __restrict__ part, int nb, double* out) {
    __shared__ double sh[kAdjThreads / 32];
    double v = 0.0;
    for (int j = threadIdx.x; j < nb; j += kAdjThreads) v += part[size_t(blockIdx.x) * nb + j];
    const double r = block_sum<kAdjThreads>(v, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = r;
}

// ---- reverse step for a run of diagonal gates
// Diagonal gates commute with each other and with every diagonal Pauli string P (a Z string),
// so for a parametric gate exp(i theta P / 2) inside a run of diagonal gates,
// <lambda_j|P|psi_j> = <lambda|P|psi> with psi, lambda taken after the whole run: one pass
// computes every such gradient of the run and then multiplies both buffers by the run's inverse
// (the product of the conjugated diagonals). Each factor of that product is either a table over
// up to 6 qubits (applied where a condition on other bits holds) or a sign (-1)^popc(x & zmask).
// FP64-class running sums: double for the FP64 policy, an FP32 (sum, compensation) pair
// (Knuth TwoSum) for the FP32 and double-float policies
template <typename P>
struct RedSum {
    float s = 0.f, c = 0.f;
    __device__ void add(float ws, float wc, bool neg) {
        if (neg) { ws = -ws; wc = -wc; }
        float h, e;
        DFArith::two_sum(s, ws, h, e);
        s = h;
        c = __fadd_rn(c, __fadd_rn(e, wc));
    }
    __device__ void add(const RedSum& o, bool neg) { add(o.s, o.c, neg); }
    __device__ double value() const { return double(s) + double(c); }
};
template <>
struct RedSum<NativeArith<double>> {
    double v = 0.0;
    __device__ void add(const RedSum& o, bool neg) { v += neg ? -o.v : o.v; }
    __device__ double value() const { return v; }
};
// Im(conj(l) p) of one amplitude as a RedSum
__device__ __forceinline__ RedSum<DFArith> im_conj_prod(float4 l, float4 p, RedSum<DFArith>) {
    RedSum<DFArith> w;
    DFArith::dprod0(w.s, w.c, l.x, l.y, p.z, p.w);
    DFArith::dprod(w.s, w.c, -l.z, -l.w, p.x, p.y);
    return w;
}
__device__ __forceinline__ RedSum<NativeArith<float>> im_conj_prod(float2 l, float2 p, RedSum<NativeArith<float>>) {
    RedSum<NativeArith<float>> w;
    DFArith::dprod0(w.s, w.c, l.x, 0.f, p.y, 0.f);
    DFArith::dprod(w.s, w.c, -l.y, 0.f, p.x, 0.f);
    return w;
}
__device__ __forceinline__ RedSum<NativeArith<double>> im_conj_prod(double2 l, double2 p, RedSum<NativeArith<double>>) {
    RedSum<NativeArith<double>> w;
    w.v = fma(l.x, p.y, -l.y * p.x);
    return w;
}

// The Walsh-Hadamard transform of one value per lane: lane l ends with the sum over lanes s of
// (-1)^{popc(s & l)} v_s (five butterfly stages across the warp, (a + b, a - b) per lane pair).
template <typename P>
__device__ __forceinline__ RedSum<P> lane_wht(RedSum<P> v, int lane) {
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        RedSum<P> o;
        o.s = __shfl_xor_sync(0xffffffffu, v.s, m);
        o.c = __shfl_xor_sync(0xffffffffu, v.c, m);
        const bool hi = (lane & m) != 0;  // this lane takes o - v, its partner v + o
        RedSum<P> r = hi ? o : v;
        r.add(hi ? v : o, hi);
        v = r;
    }
    return v;
}
template <>
__device__ __forceinline__ RedSum<NativeArith<double>> lane_wht(RedSum<NativeArith<double>> v, int lane) {
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const double o = __shfl_xor_sync(0xffffffffu, v.v, m);
        v.v = (lane & m) ? o - v.v : v.v + o;
    }
    return v;
}
template <typename P>
__device__ __forceinline__ RedSum<P> lane_fetch(const RedSum<P>& v, int src) {
    RedSum<P> o;
    o.s = __shfl_sync(0xffffffffu, v.s, src);
    o.c = __shfl_sync(0xffffffffu, v.c, src);
    return o;
}
template <>
__device__ __forceinline__ RedSum<NativeArith<double>> lane_fetch(const RedSum<NativeArith<double>>& v, int src) {
    RedSum<NativeArith<double>> o;
    o.v = __shfl_sync(0xffffffffu, v.v, src);
    return o;
}

__device__ __forceinline__ float4 kmul(float4 a, float4 b) { return DFArith::out(DFArith::first(a, b)); }
__device__ __forceinline__ float2 kmul(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 kmul(double2 a, double2 b) { return cmul(a, b); }
template <typename K>
__device__ __forceinline__ K kone();
template <>
__device__ __forceinline__ float4 kone<float4>() { return make_float4(1.f, 0.f, 0.f, 0.f); }
template <>
__device__ __forceinline__ float2 kone<float2>() { return make_float2(1.f, 0.f); }
template <>
__device__ __forceinline__ double2 kone<double2>() { return make_double2(1.0, 0.0); }

constexpr int kDiagKA = 4;  // amplitudes per thread between two gradient flushes

// Thread t of T = grid x 256 threads takes the amplitudes x = j T + t, kDiagKA values of j at a
// time, each giving w_x = Im(conj(lam_x) psi_x). Per j the warp transforms its 32 values
// (Walsh-Hadamard across the lanes), and lane g takes the coefficient at its gradient term's Z
// bits among the lane bits, with the sign of the rest of the term's Z bits: every term of the
// run from one transform, so the per-amplitude cost does not grow with the number of gradients.
template <typename P>
__global__ void __launch_bounds__(kAdjThreads) k_adj_diag(typename P::C* __restrict__ psi, typename P::C* __restrict__ lam,
                                                           const typename P::K* __restrict__ tab,
                                                           const __grid_constant__ AdjDiagParams A, double* part) {
    using C = typename P::C;
    using K = typename P::K;
    using R = RedSum<P>;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    K* stab = reinterpret_cast<K*>(adj_smem);
    R* wred = reinterpret_cast<R*>(adj_smem + ((size_t(A.ntab) * sizeof(K) + 15) & ~size_t(15)));  // [warp][g]
    for (int i = threadIdx.x; i < A.ntab; i += kAdjThreads) stab[i] = tab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t T = uint64_t(gridDim.x) * kAdjThreads;
    const uint64_t t = uint64_t(blockIdx.x) * kAdjThreads + threadIdx.x;
    const uint64_t J = (A.n_amp + T - 1) / T;
    const uint64_t gz = lane < A.ng ? A.gz[lane] : 0;
    R gsum;  // lane g: this warp's sum for gradient term g
    const uint64_t t0 = t - uint64_t(lane);  // the warp's first thread
    for (uint64_t j0 = 0; j0 < J; j0 += kDiagKA) {
        R acc[kDiagKA];
#pragma unroll
        for (int j = 0; j < kDiagKA; j++) {
            const uint64_t x = (j0 + j) * T + t;
            if (j0 + j >= J || x >= A.n_amp) continue;
            C p = psi[x], l = lam[x];
            if (A.ng) acc[j] = im_conj_prod(l, p, R());
            K f = kone<K>();
            int sign = 0;
#pragma unroll 1
            for (int k = 0; k < A.nf; k++) {
                const AdjDiagFactor& F = A.f[k];
                if ((x & F.cond_mask) != F.cond_val) continue;
                sign ^= parity64(x & F.zmask);
                if (F.pair_shift) sign ^= parity64(x & (x >> F.pair_shift) & F.pair_mask);
                if (F.sign_only) {
                    sign ^= 1;
                } else if (F.tab_off >= 0) {
                    uint32_t li = 0;
                    for (int b = 0; b < F.nrun; b++) {
                        const uint32_t c = F.run[b];
                        li |= (uint32_t(x >> (c & 0xFFu)) & ((1u << ((c >> 8) & 0xFFu)) - 1u)) << (c >> 16);
                    }
                    f = kmul(f, stab[F.tab_off + int(li)]);
                }
            }
            p = P::out(P::first(f, p));
            l = P::out(P::first(f, l));
            if (sign) {
                p = P::ipow(p, 2);
                l = P::ipow(l, 2);
            }
            psi[x] = p;
            lam[x] = l;
        }
        if (A.ng) {
            // gradient term g over the warp's 32 amplitudes of item j, x = (j0 + j) T + t0 + s:
            // the lane bits s, the warp's bits of t0 and the item's bits of (j0 + j) T are
            // disjoint (T is a power of two), so the sign (-1)^{popc(x & z_g)} factors into
            // (-1)^{popc(s & z_g)}, whose sum over s is the warp's Walsh-Hadamard coefficient at
            // z_g mod 32, times the sign of the rest
#pragma unroll
            for (int j = 0; j < kDiagKA; j++) {
                const R w = lane_fetch(lane_wht(acc[j], lane), int(gz & 31u));
                if (lane < A.ng && j0 + j < J) gsum.add(w, parity64(((j0 + j) * T + t0) & gz) != 0);
            }
        }
    }
    if (A.ng) {
        if (lane < A.ng) wred[warp * 32 + lane] = gsum;
        __syncthreads();
        if (threadIdx.x < A.ng) {
            R total;
            for (int w = 0; w < kAdjThreads / 32; w++) total.add(wred[w * 32 + threadIdx.x], false);
            part[size_t(threadIdx.x) * gridDim.x + blockIdx.x] = total.value();
        }
    }
}

size_t adj_diag_smem(int ntab, Arith ar) {
    const size_t rs = ar == Arith::F64 ? sizeof(double) : 2 * sizeof(float);
    return ((size_t(ntab) * kernel_entry_bytes(ar) + 15) & ~size_t(15)) + rs * (kAdjThreads / 32) * 32;
}

// R_P(theta)^+ = cos(theta/2) I - i sin(theta/2) P as a row-major 2x2 matrix
void rot_dagger(int axis, double theta, cplx (&U)[4]) {
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    if (axis == 1) { U[0] = c; U[1] = cplx(0, -s); U[2] = cplx(0, -s); U[3] = c; }
    else if (axis == 2) { U[0] = c; U[1] = -s; U[2] = s; U[3] = c; }
    else { U[0] = cplx(c, -s); U[1] = 0.0; U[2] = 0.0; U[3] = cplx(c, s); }
}

template <typename P, int NR>
void launch_rotn(void* psi, void* lam, int n, const int* qubit, const int* axis, const double* theta, double* part,
                 unsigned grid, cudaStream_t st) {
    AdjRotNParams<P, NR> A;
    A.ip = make_index_plan(n, std::vector<int>(qubit, qubit + NR), 0);
    for (int r = 0; r < NR; r++) {
        A.bit[r] = 1ull << qubit[r];
        A.axis[r] = axis[r];
        cplx U[4];
        rot_dagger(axis[r], theta[r], U);
        for (int e = 0; e < 4; e++) A.U[r][e] = P::host_k(U[e].real(), U[e].imag());
    }
    k_adj_rotn<P, NR><<<grid, kAdjThreads, 0, st>>>(reinterpret_cast<typename P::C*>(psi),
                                                    reinterpret_cast<typename P::C*>(lam), A, part);
}

// Two rotations per pass: three or four (8 or 16 amplitudes of psi and lambda per thread) were
// measured slower in every arithmetic at n = 20 (the registers cut the resident warps), so only
// NR = 2 is instantiated.
template <typename P>
void launch_rotn_any(int nr, void* psi, void* lam, int n, const int* qubit, const int* axis, const double* theta,
                     double* part, unsigned grid, cudaStream_t st) {
    QS_REQUIRE(nr == 2, "two rotations per pass");
    launch_rotn<P, 2>(psi, lam, n, qubit, axis, theta, part, grid, st);
}

template <typename P>
void launch_rot(void* psi, void* lam, int n, int qubit, int axis, double theta, double* part, unsigned grid,
                cudaStream_t st) {
    AdjRotParams<P> A;
    A.ip = make_index_plan(n, {qubit}, 0);
    A.bit = 1ull << qubit;
    A.axis = axis;
    // R^+ = cos(theta/2) I - i sin(theta/2) P
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    cplx U[4];
    if (axis == 1) { U[0] = c; U[1] = cplx(0, -s); U[2] = cplx(0, -s); U[3] = c; }
    else if (axis == 2) { U[0] = c; U[1] = -s; U[2] = s; U[3] = c; }
    else { U[0] = cplx(c, -s); U[1] = 0.0; U[2] = 0.0; U[3] = cplx(c, s); }
    for (int e = 0; e < 4; e++) A.U[e] = P::host_k(U[e].real(), U[e].imag());
    k_adj_rot<P><<<grid, kAdjThreads, 0, st>>>(reinterpret_cast<typename P::C*>(psi),
                                               reinterpret_cast<typename P::C*>(lam), A, part);
}

}  // namespace

unsigned adj_grid(int n) {
    const uint64_t pairs = 1ull << (n - 1);
    // a power of two (the diagonal-run kernel's amplitude partition relies on it)
    uint64_t want = 1;
    while (want * 2 * kAdjThreads <= pairs && want < 1024) want *= 2;
    return unsigned(want);
}

void launch_adjoint_rotation(void* psi, void* lam, int n, Arith ar, int qubit, int axis, double theta, double* part,
                             unsigned grid, cudaStream_t st) {
    switch (ar) {
        case Arith::F32: launch_rot<NativeArith<float>>(psi, lam, n, qubit, axis, theta, part, grid, st); break;
        case Arith::F64: launch_rot<NativeArith<double>>(psi, lam, n, qubit, axis, theta, part, grid, st); break;
        case Arith::DF: launch_rot<DFArith>(psi, lam, n, qubit, axis, theta, part, grid, st); break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

int adjoint_max_rotations(Arith) { return 2; }

void launch_adjoint_rotations(void* psi, void* lam, int n, Arith ar, int nr, const int* qubit, const int* axis,
                              const double* theta, double* part, unsigned grid, cudaStream_t st) {
    QS_REQUIRE(nr >= 2 && nr <= adjoint_max_rotations(ar), "rotations per pass out of range");
    QS_REQUIRE(n >= nr, "fewer qubits than rotations");
    switch (ar) {
        case Arith::F32: launch_rotn_any<NativeArith<float>>(nr, psi, lam, n, qubit, axis, theta, part, grid, st); break;
        case Arith::F64: launch_rotn_any<NativeArith<double>>(nr, psi, lam, n, qubit, axis, theta, part, grid, st); break;
        case Arith::DF: launch_rotn_any<DFArith>(nr, psi, lam, n, qubit, axis, theta, part, grid, st); break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_adjoint_diag(void* psi, void* lam, int n, Arith ar, const void* tab, const AdjDiagParams& A, double* part,
                         unsigned grid, cudaStream_t st) {
    const size_t smem = adj_diag_smem(A.ntab, ar);
    switch (ar) {
        case Arith::F32:
            k_adj_diag<NativeArith<float>><<<grid, kAdjThreads, smem, st>>>(
                static_cast<float2*>(psi), static_cast<float2*>(lam), static_cast<const float2*>(tab), A, part);
            break;
        case Arith::F64:
            k_adj_diag<NativeArith<double>><<<grid, kAdjThreads, smem, st>>>(
                static_cast<double2*>(psi), static_cast<double2*>(lam), static_cast<const double2*>(tab), A, part);
            break;
        case Arith::DF:
            k_adj_diag<DFArith><<<grid, kAdjThreads, smem, st>>>(
                static_cast<float4*>(psi), static_cast<float4*>(lam), static_cast<const float4*>(tab), A, part);
            break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_slot_sums(const double* part, int nslots, unsigned nb, double* out, cudaStream_t st) {
    if (nslots <= 0) return;
    k_slot_sums<<<nslots, kAdjThreads, 0, st>>>(part, int(nb), out);
    QS_TRY_CUDA(cudaGetLastError());
}

}  // namespace qs
