// Device helpers shared by the kernels of libqsim_gb300.so: complex arithmetic on
// interleaved (re, im) pairs, the B(0) enumeration of Eq. (update_mat), and exact
// float products / double-float accumulation used for FP64-class sums of FP32 data.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsim_internal.h"

namespace qs {

template <typename R>
struct CT;
template <>
struct CT<float> {
    using type = float2;
};
template <>
struct CT<double> {
    using type = double2;
};

template <typename C>
__device__ __forceinline__ C cmake(double re, double im);
template <>
__device__ __forceinline__ float2 cmake<float2>(double re, double im) {
    return make_float2(float(re), float(im));
}
template <>
__device__ __forceinline__ double2 cmake<double2>(double re, double im) {
    return make_double2(re, im);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

// Multiply by one of {1, i, -1, -i} (k mod 4): a permutation with sign changes only.
template <typename C>
__device__ __forceinline__ C mul_ipow(C a, int k) {
    switch (k & 3) {
        case 0: return a;
        case 1: { C r; r.x = -a.y; r.y = a.x; return r; }
        case 2: { C r; r.x = -a.x; r.y = -a.y; return r; }
        default: { C r; r.x = a.y; r.y = -a.x; return r; }
    }
}

// i -> the i-th element of B(0) with the fixed bits inserted as zeros (ascending
// positions), then the bits that must be one or'ed in.
__device__ __forceinline__ uint64_t expand(uint64_t i, const IndexPlan& p) {
#pragma unroll 1
    for (int j = 0; j < p.nfix; j++) {
        const uint64_t lo = i & ((1ull << p.fixpos[j]) - 1ull);
        i = ((i ^ lo) << 1) | lo;
    }
    return i | p.setmask;
}

__device__ __forceinline__ int parity64(uint64_t v) { return __popcll(v) & 1; }

// ---- double-float accumulation of exact FP32 products (Knuth TwoSum, FMA TwoProd)
struct DFAcc {
    float hi, lo;
};
__device__ __forceinline__ void df_zero(DFAcc& a) { a.hi = 0.f; a.lo = 0.f; }
// acc += a * b without rounding the product; the sum error goes to acc.lo
__device__ __forceinline__ void df_add_prod(DFAcc& acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ double df_value(const DFAcc& a) { return double(a.hi) + double(a.lo); }

// ---- block reductions (deterministic order)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

}  // namespace qs
