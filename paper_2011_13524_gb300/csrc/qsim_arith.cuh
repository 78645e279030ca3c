// Arithmetic policies of the gate kernels.
//
//   NativeArith<float>  complex64 storage, FP32 multiply-adds.
//   NativeArith<double> complex128 storage, FP64 multiply-adds.
//   DFArith             complex128 values held as double-float pairs: each real number is
//                       hi + lo with two FP32 words (float4 {re_hi, re_lo, im_hi, im_lo}, the
//                       same 16 bytes as an IEEE complex128 amplitude), updated on the FP32
//                       pipes. GB300 executes FP64 at 1/64 of the FP32 rate, so the IEEE-double
//                       update of a dense gate is arithmetic-bound far below HBM speed; the
//                       double-float form keeps ~2^-46 relative accuracy per update.
//
// Double-float products use the FMA error-free transformation (the exact error of p = a*b is
// fma(a, b, -p)) and Knuth's TwoSum for additions, accumulated as in the compensated dot
// product of Ogita, Rump & Oishi (SIAM J. Sci. Comput. 26, 2005): the rounded partial sum in
// s, every rounding error and cross term in c, and one TwoSum at the end. Intrinsics with an
// explicit rounding mode keep the compiler from contracting these steps into FMAs.
#pragma once

#include "qsim_kernels.cuh"

namespace qs {

template <typename R>
struct NativeArith {
    using C = typename CT<R>::type;
    using K = C;
    using Acc = C;
    __device__ __forceinline__ static Acc zero() { return cmake<C>(0.0, 0.0); }
    __device__ __forceinline__ static void mac(Acc& a, const K& k, const C& v) { a = cfma(k, v, a); }
    // accumulator holding k * v (the first term of a sum)
    __device__ __forceinline__ static Acc first(const K& k, const C& v) { return cmul(k, v); }
    __device__ __forceinline__ static C out(const Acc& a) { return a; }
    __device__ __forceinline__ static C ipow(const C& v, int k) { return mul_ipow(v, k); }
    __device__ __forceinline__ static C basis(bool one) { return cmake<C>(one ? 1.0 : 0.0, 0.0); }
    __host__ static K host_k(double re, double im) {
        K k;
        k.x = R(re);
        k.y = R(im);
        return k;
    }
};

// a = hi + lo with |lo| <= ulp(hi)/2 (round to nearest)
__host__ __device__ inline void split_double(double x, float& hi, float& lo) {
    hi = float(x);
    lo = float(x - double(hi));
}

struct DFArith {
    using C = float4;  // {re_hi, re_lo, im_hi, im_lo}
    using K = float4;
    struct Acc {
        float rs, rc, is, ic;  // real: partial sum, compensation; imaginary likewise
    };
    __device__ __forceinline__ static Acc zero() { return Acc{0.f, 0.f, 0.f, 0.f}; }
    // (s, c) += (ah + al) * (bh + bl), dropping al * bl
    __device__ __forceinline__ static void dprod(float& s, float& c, float ah, float al, float bh, float bl) {
        const float p = __fmul_rn(ah, bh);
        float e = __fmaf_rn(ah, bh, -p);
        e = __fmaf_rn(ah, bl, e);
        e = __fmaf_rn(al, bh, e);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(d, e));
    }
    __device__ __forceinline__ static void mac(Acc& a, const K& k, const C& v) {
        dprod(a.rs, a.rc, k.x, k.y, v.x, v.y);      // + kr vr
        dprod(a.rs, a.rc, -k.z, -k.w, v.z, v.w);    // - ki vi
        dprod(a.is, a.ic, k.x, k.y, v.z, v.w);      // + kr vi
        dprod(a.is, a.ic, k.z, k.w, v.x, v.y);      // + ki vr
    }
    // (s, c) = (ah + al) * (bh + bl) without the TwoSum of dprod (the sum starts here)
    __device__ __forceinline__ static void dprod0(float& s, float& c, float ah, float al, float bh, float bl) {
        s = __fmul_rn(ah, bh);
        float e = __fmaf_rn(ah, bh, -s);
        e = __fmaf_rn(ah, bl, e);
        c = __fmaf_rn(al, bh, e);
    }
    __device__ __forceinline__ static Acc first(const K& k, const C& v) {
        Acc a;
        dprod0(a.rs, a.rc, k.x, k.y, v.x, v.y);
        dprod(a.rs, a.rc, -k.z, -k.w, v.z, v.w);
        dprod0(a.is, a.ic, k.x, k.y, v.z, v.w);
        dprod(a.is, a.ic, k.z, k.w, v.x, v.y);
        return a;
    }
    __device__ __forceinline__ static void two_sum(float a, float b, float& h, float& l) {
        h = __fadd_rn(a, b);
        const float bp = __fsub_rn(h, a);
        l = __fadd_rn(__fsub_rn(a, __fsub_rn(h, bp)), __fsub_rn(b, bp));
    }
    __device__ __forceinline__ static C out(const Acc& a) {
        C r;
        two_sum(a.rs, a.rc, r.x, r.y);
        two_sum(a.is, a.ic, r.z, r.w);
        return r;
    }
    __device__ __forceinline__ static C ipow(const C& v, int k) {
        switch (k & 3) {
            case 0: return v;
            case 1: return make_float4(-v.z, -v.w, v.x, v.y);
            case 2: return make_float4(-v.x, -v.y, -v.z, -v.w);
            default: return make_float4(v.z, v.w, -v.x, -v.y);
        }
    }
    __device__ __forceinline__ static C basis(bool one) { return make_float4(one ? 1.f : 0.f, 0.f, 0.f, 0.f); }
    __host__ static K host_k(double re, double im) {
        K k;
        split_double(re, k.x, k.y);
        split_double(im, k.z, k.w);
        return k;
    }
};

// value of a stored element widened to FP64 (re, im)
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double2 widen(float4 v) {
    return make_double2(double(v.x) + double(v.y), double(v.z) + double(v.w));
}
// FP64 (re, im) -> stored element
template <typename C>
__device__ __forceinline__ C narrow(double re, double im);
template <>
__device__ __forceinline__ float2 narrow<float2>(double re, double im) {
    return make_float2(float(re), float(im));
}
template <>
__device__ __forceinline__ double2 narrow<double2>(double re, double im) {
    return make_double2(re, im);
}
template <>
__device__ __forceinline__ float4 narrow<float4>(double re, double im) {
    float4 r;
    split_double(re, r.x, r.y);
    split_double(im, r.z, r.w);
    return r;
}

// double -> (hi, lo) floats with hi = RN(x) and lo = RN(x - hi), as split_double, but on the
// integer pipes (GB300 runs FP64 and its conversions at 1/64 of the FP32 rate): hi takes the top
// 24 significant bits rounded to nearest-even, lo the remainder, an integer number of the
// double's last places below 2^29, converted to float with rounding to nearest and scaled by
// powers of two (exact, as lo is then a normal float): lo = RN(x - hi). Below 2^-74 (a double
// exponent field under 949) a nonzero remainder can be subnormal in FP32, where a second
// rounding could creep in; those magnitudes take the FP64 split. Zero is split directly.
// Magnitudes below 2^-126 (under FP32's normal range) become a signed zero: the absolute change
// is below 1.2e-38. At or above 2^125 (huge, non-finite) it falls back to the FP64 instructions.
__device__ __forceinline__ void split_double_int(double x, float& hi, float& lo) {
    const uint64_t b = uint64_t(__double_as_longlong(x));
    const uint32_t e = uint32_t(b >> 52) & 0x7FFu;
    const uint32_t sign = uint32_t(b >> 63) << 31;
    if (e < 897u) {  // +-0 and |x| < 2^-126
        hi = __uint_as_float(sign);
        lo = 0.f;
        return;
    }
    if (e > 1148u || e < 949u) {
        split_double(x, hi, lo);
        return;
    }
    const uint64_t m = b & ((1ull << 52) - 1);
    const uint32_t hm = uint32_t(m >> 29);
    const uint32_t rem = uint32_t(m & ((1ull << 29) - 1));
    const uint32_t up = (rem > (1u << 28) || (rem == (1u << 28) && (hm & 1u))) ? 1u : 0u;
    hi = __uint_as_float(sign | (((e - 1023u + 127u) << 23) + hm + up));
    const int32_t li = int32_t(rem) - int32_t(up << 29);
    const float scale = __uint_as_float((e - 1075u + 127u) << 23);  // 2^(e - 1075), normal for e >= 949
    const float l = __fmul_rn(__int2float_rn(li), scale);
    lo = sign ? -l : l;
}
// float -> double exactly, on the integer pipes for zero and normal floats
__device__ __forceinline__ double widen_float_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if ((u << 1) == 0u) return __longlong_as_double(static_cast<long long>(uint64_t(u >> 31) << 63));
    if (e == 0u || e == 255u) return double(f);
    const uint64_t b = (uint64_t(u >> 31) << 63) | (uint64_t(e - 127u + 1023u) << 52) | (uint64_t(u & 0x7FFFFFu) << 29);
    return __longlong_as_double(static_cast<long long>(b));
}

// RN(hi + lo) as a double for a double-float pair, on the integer pipes when both are normal and
// lo's exponent is 24..55 below hi's (every pair with |lo| <= ulp(hi)/2 has it at least 24
// below). In units of the last place of a double with hi's exponent, |lo| = L + F / 2^s: for a
// gap d <= 29 an integer (F = 0), for d = 29 + s a 32-bit integer part and an s-bit fraction.
// Rounded to nearest-even from F, the change of hi's significand is + L (+1) for equal signs and
// - (L + [F != 0]) (+1) for opposite ones; it never leaves hi's binade except below a power of
// two, so it is added to the bit pattern of hi as a double (a carry into the exponent is the
// exact power of two). Selects, not branches, on the gap and the signs. Otherwise (zero hi,
// subnormal, non-finite, lo far smaller, a power-of-two hi with lo of the other sign) the FP64
// add.
__device__ __forceinline__ double join_df_general(float hi, float lo) {
    const uint32_t uh = __float_as_uint(hi), ul = __float_as_uint(lo);
    if ((ul << 1) == 0u) return widen_float_int(hi);
    const uint32_t eh = (uh >> 23) & 0xFFu, el = (ul >> 23) & 0xFFu;
    const uint32_t d = eh - el;
    const bool sub = ((uh ^ ul) >> 31) != 0u;
    if (eh == 0u || eh == 255u || el == 0u || d - 24u > 31u || (sub && (uh & 0x7FFFFFu) == 0u))
        return widen_float_int(hi) + widen_float_int(lo);
    const uint32_t ml = (ul & 0x7FFFFFu) | 0x800000u;
    const uint32_t sl = d < 29u ? 29u - d : 0u;  // d <= 29: lo's bits all land on the significand
    const uint32_t sr = d > 29u ? d - 29u : 0u;  // d > 29: sr bits of lo below it
    const uint32_t L = (ml << sl) >> sr;
    const uint32_t F = ml & ((1u << sr) - 1u);
    const uint32_t half = (1u << sr) >> 1;
    const uint32_t frac = F != 0u ? 1u : 0u;
    const uint32_t t = sub ? L + frac : L;  // the parity of the significand after the change
    const uint32_t odd = t & 1u;
    const uint32_t up = sub ? (frac && (F < half || (F == half && odd))) : (F > half || (frac && F == half && odd));
    const long long dm = sub ? (long long)up - (long long)t : (long long)t + (long long)up;
    const uint32_t w_hi = (uh & 0x80000000u) | ((eh + 896u) << 20) | ((uh & 0x7FFFFFu) >> 3);
    const uint32_t w_lo = uh << 29;
    return __longlong_as_double(__double_as_longlong(__hiloint2double(int(w_hi), int(w_lo))) + dm);
}

// The same value with fewer instructions for the common case. With u the last place of a double
// in hi's binade (2^(E - 52), E hi's exponent), y = lo / u with hi's sign taken out is exact in
// FP32 (a power-of-two scaling; |y| <= 2^28 for |lo| <= ulp(hi)/2), the exact sum is
// hi + y u = (S + y) u with S hi's significand shifted to 53 bits, an even integer, and its
// rounding to the double grid of hi's binade is S + RN_int(y) (ties to even on the integer:
// S is even). The sum stays in hi's binade (|y| <= 2^28 cannot reach the next power of two up),
// except below a power-of-two hi with y < 0, where the grid below is finer: that case, and zero,
// subnormal, non-finite or tiny (|hi| < 2^-74, where 2^(52 - E) leaves FP32's range) hi, take the
// general join above.
__device__ __forceinline__ double join_df_int(float hi, float lo) {
    const uint32_t uh = __float_as_uint(hi);
    const uint32_t eb = (uh >> 23) & 0xFFu, mant = uh & 0x7FFFFFu, sign = uh & 0x80000000u;
    const float y = __fmul_rn(__uint_as_float(__float_as_uint(lo) ^ sign), __uint_as_float((306u - eb) << 23));
    if (eb < 53u || eb == 255u || (mant == 0u && y < 0.f)) return join_df_general(hi, lo);
    const uint32_t w_hi = sign | ((eb + 896u) << 20) | (mant >> 3);
    const long long w = (static_cast<long long>(w_hi) << 32) | static_cast<long long>(mant << 29);
    return __longlong_as_double(w + static_cast<long long>(__float2int_rn(y)));
}

}  // namespace qs
