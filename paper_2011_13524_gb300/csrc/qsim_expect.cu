// Pauli-observable expectation E = sum_P alpha_P <psi|P|psi> (Sec. 4.5) over tiles of the state,
// several flip-mask groups per pass, in double-float arithmetic on the FP32 pipes.
//
// Terms are grouped by their flip mask f (the X-or-Y positions). For a pair representative y
// (pivot bit of f clear) and A = conj(psi_{y^f}) psi_y, the pair (y, y^f) contributes
//   i^{nY} (-1)^{popc(y & z)} (A + (-1)^{nY} conj(A))
//     = 2 (-1)^{nY/2} (-1)^{popc(y & z)} Re A            (nY even)
//     = 2 (-1)^{(nY+1)/2} (-1)^{popc(y & z)} Im A        (nY odd),
// and the diagonal group f = 0 contributes (-1)^{popc(y & z)} |psi_y|^2 per amplitude.
//
// A tile is the 2^b amplitudes whose bits outside a set T of b <= 12 qubits (always holding
// qubits 0..2, so that a tile is read in runs of 8 contiguous amplitudes) equal a fixed rest
// index r; it occupies 2^12 slots in shared memory, the slots of a smaller state's missing
// (virtual) tile bits holding zeros. Every group with f inside T is evaluated from the tile, so
// one read of the state serves all of them: a transverse-field Ising chain of 30 qubits (31
// groups) takes 3 reads. Within a group each of the 256 threads owns 16 amplitudes (diagonal
// group) or 8 pair representatives that differ in the group's item bits; the signs that vary
// over the items are handled by a Walsh-Hadamard transform of the thread's item values, the signs
// over the thread's own bits and over the rest index by per-term factors. Terms that share
// (component, item mask, thread mask) share one slot, whose coefficient sum over the rest-index
// signs is formed once per tile. The transition amplitude (second half of this file) uses the
// same packing on tiles of 2^11 slots of two states.
//
// Item values and their transforms are exact sums on a power-of-two grid: each value
// h + l (double-float) is split into H = RN(h + c) - c with c = 1.5 * 2^e above the thread's
// |sum|, whose sums and differences are exact in FP32, and the remainder (h - H) + l, which is
// small. Per-thread sums are double-float and go to an FP64 accumulator once per tile, so the
// result has the accuracy of an FP64 sum (about 2^-44 relative per tile).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "qsim_arith.cuh"

namespace qs {

namespace {

int sm_count() { return device_sms(); }

// smem element of a tile: complex64 stays float2, complex128 becomes double-float float4
template <typename C>
struct TileElem;
template <>
struct TileElem<float2> {
    using T = float2;
    static constexpr bool kLo = false;
};
template <>
struct TileElem<double2> {
    using T = float4;
    static constexpr bool kLo = true;
};
template <>
struct TileElem<float4> {
    using T = float4;
    static constexpr bool kLo = true;
};

// double -> hi + lo for tile values, on the integer pipes: hi = x truncated to 24 significant
// bits, built by moving the exponent and mantissa fields (for 2^-126 <= |x| < 2^127 the float
// exponent is the low 8 bits of the double exponent with bit 7 flipped); lo = the next 23
// remainder bits, as (F - base) * 2^-23 where F has hi's sign and exponent and those bits as
// mantissa and base = hi's power of two (both operations exact). |x - hi - lo| < 2^-46 |x|.
// Magnitudes below 2^-126 become a signed zero; 2^127 and above use the FP64 split.
__device__ __forceinline__ void split_tile(double x, float& hi, float& lo) {
    const uint32_t bh = uint32_t(__double2hiint(x)), bl = uint32_t(__double2loint(x));
    const uint32_t e = (bh >> 20) & 0x7FFu;
    if (e - 897u > 253u) {
        if (e < 897u) {
            hi = __uint_as_float(bh & 0x80000000u);
            lo = 0.f;
        } else {
            split_double(x, hi, lo);
        }
        return;
    }
    const uint32_t fb = __funnelshift_l(bl, bh, 3);  // double exponent bits 7..0 at 30..23, 23 mantissa bits
    const uint32_t hb = (bh & 0x80000000u) | ((fb & 0x7FFFFFFFu) ^ 0x40000000u);
    const uint32_t se = hb & 0xFF800000u;
    hi = __uint_as_float(hb);
    lo = __fmul_rn(__fsub_rn(__uint_as_float(se | ((bl >> 6) & 0x7FFFFFu)), __uint_as_float(se)), 1.1920928955078125e-07f);
}

// A complex128 tile element is held as {re_hi, im_hi, re_lo, im_lo}: the high words of the real
// and imaginary parts side by side, and the low words, so that both parts are processed as
// packed FP32 pairs.
__device__ __forceinline__ float2 to_tile(float2 v) { return v; }
__device__ __forceinline__ float4 to_tile(float4 v) { return make_float4(v.x, v.z, v.y, v.w); }
__device__ __forceinline__ float4 to_tile(double2 v) {
    float4 r;
    split_tile(v.x, r.x, r.z);
    split_tile(v.y, r.y, r.w);
    return r;
}

struct DFc {
    float rh, rl, ih, il;
};
__device__ __forceinline__ DFc dfc(float2 e) { return DFc{e.x, 0.f, e.y, 0.f}; }
__device__ __forceinline__ DFc dfc(float4 e) { return DFc{e.x, e.z, e.y, e.w}; }

__device__ __forceinline__ void two_sum_f(float a, float b, float& h, float& l) {
    h = __fadd_rn(a, b);
    const float bp = __fsub_rn(h, a);
    l = __fadd_rn(__fsub_rn(a, __fsub_rn(h, bp)), __fsub_rn(b, bp));
}

// h + l ~ x1 y1 + x2 y2 for double-float operands (the lo x lo products dropped)
template <bool kLo>
__device__ __forceinline__ void df_dot2(float x1h, float x1l, float y1h, float y1l, float x2h, float x2l, float y2h,
                                        float y2l, float& h, float& l) {
    const float p1 = __fmul_rn(x1h, y1h), p2 = __fmul_rn(x2h, y2h);
    const float e1 = __fmaf_rn(x1h, y1h, -p1), e2 = __fmaf_rn(x2h, y2h, -p2);
    float e3;
    two_sum_f(p1, p2, h, e3);
    l = __fadd_rn(__fadd_rn(e1, e2), e3);
    if (kLo) {
        l = __fmaf_rn(x1h, y1l, l);
        l = __fmaf_rn(x1l, y1h, l);
        l = __fmaf_rn(x2h, y2l, l);
        l = __fmaf_rn(x2l, y2h, l);
    }
}

// Sums over K items on the grid described above. full: the Walsh-Hadamard transform
// Q[m] = sum_k (-1)^{popc(k & m)} x_k for every m; otherwise only Q[0]. Result (h[m], l[m]).
template <int K>
__device__ __forceinline__ void grid_transform(float* h, float* l, bool full) {
    float t[K];
#pragma unroll
    for (int k = 0; k < K; k++) t[k] = fabsf(h[k]);
#pragma unroll
    for (int s = 1; s < K; s <<= 1)
#pragma unroll
        for (int k = 0; k < K; k += 2 * s) t[k] = __fadd_rn(t[k], t[k + s]);
    const float S = t[0];
    uint32_t e = (__float_as_uint(S) >> 23) & 0xFFu;
    e = e > 250u ? 250u : e;
    const float c = __uint_as_float(((e + 2u) << 23) | 0x400000u);  // 1.5 * 2^(e - 125) > 3 S
#pragma unroll
    for (int k = 0; k < K; k++) {
        const float H = __fsub_rn(__fadd_rn(h[k], c), c);
        l[k] = __fadd_rn(__fsub_rn(h[k], H), l[k]);
        h[k] = H;
    }
    if (full) {
#pragma unroll
        for (int s = 1; s < K; s <<= 1) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (k & s) continue;
                const float a = h[k], b = h[k | s], u = l[k], v = l[k | s];
                h[k] = __fadd_rn(a, b);
                h[k | s] = __fsub_rn(a, b);
                l[k] = __fadd_rn(u, v);
                l[k | s] = __fsub_rn(u, v);
            }
        }
    } else {
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k < K; k += 2 * s) {
                h[k] = __fadd_rn(h[k], h[k + s]);
                l[k] = __fadd_rn(l[k], l[k + s]);
            }
    }
}

// (ah, al) += (gh + gl) * (qh + ql)
__device__ __forceinline__ void acc_prod(float& ah, float& al, float gh, float gl, float qh, float ql) {
    const float p = __fmul_rn(gh, qh);
    float e = __fmaf_rn(gh, qh, -p);
    e = __fmaf_rn(gh, ql, e);
    e = __fmaf_rn(gl, qh, e);
    float s, t;
    two_sum_f(ah, p, s, t);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, e));
}

__device__ __forceinline__ float flip_sign(float x, uint32_t flip) { return __uint_as_float(__float_as_uint(x) ^ flip); }

constexpr int top_bit(int k) { return k >= 8 ? 3 : k >= 4 ? 2 : k >= 2 ? 1 : 0; }

// Item values of one group for the thread whose item 0 (pivot and item bits clear) is tile slot
// tb: kind kTileDiag -> |psi|^2 of 16 amplitudes in (qh, ql)[0..15]; flip kinds -> Re A of the 8
// pair representatives in [0..7] and / or Im A in [8..15], A = conj(psi_{y^f}) psi_y.
template <typename E, bool kLo, int kKind>
__device__ __forceinline__ void group_values(const E* tile, uint32_t tb, uint32_t f, const uint32_t* im, float* qh,
                                             float* ql) {
    constexpr int K = kKind == kTileDiag ? 16 : 8;
    uint32_t o[K];
    o[0] = tb;
#pragma unroll
    for (int k = 1; k < K; k++) o[k] = o[k ^ (1 << top_bit(k))] | im[top_bit(k)];
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (kKind == kTileDiag) {
            const DFc v = dfc(tile[o[k]]);
            df_dot2<kLo>(v.rh, v.rl, v.rh, v.rl, v.ih, v.il, v.ih, v.il, qh[k], ql[k]);
        } else {
            const DFc a = dfc(tile[o[k]]), b = dfc(tile[o[k] ^ f]);
            if (kKind & kTileRe)  // Re conj(b) a = a.re b.re + a.im b.im
                df_dot2<kLo>(a.rh, a.rl, b.rh, b.rl, a.ih, a.il, b.ih, b.il, qh[k], ql[k]);
            if (kKind & kTileIm)  // Im conj(b) a = a.im b.re - a.re b.im
                df_dot2<kLo>(a.ih, a.il, b.rh, b.rl, -a.rh, -a.rl, b.ih, b.il, qh[8 + k], ql[8 + k]);
        }
    }
}

// slots of buckets [B0, B1): (ah, al) += sign(thread bits) * gamma_s * Q[bucket]
template <int B0, int B1>
__device__ __forceinline__ void slot_sums(const TileGroup& G, const TileSlot* S, const float2* gam, uint32_t tid,
                                          const float* qh, const float* ql, float& ah, float& al) {
#pragma unroll
    for (int bk = B0; bk < B1; bk++) {
        const int s1 = G.slot0 + G.bstart[bk + 1];
        for (int s = G.slot0 + G.bstart[bk]; s < s1; s++) {
            const float2 g = gam[s];
            const uint32_t flip = uint32_t(__popc(tid & S[s].zthr) & 1) << 31;
            acc_prod(ah, al, flip_sign(g.x, flip), flip_sign(g.y, flip), qh[bk], ql[bk]);
        }
    }
}

// The plain sum over the thread's 8 items of b.re c.re + b.im c.im (kIm false) or
// b.re c.im - b.im c.re (kIm true), b = tb_[o[k]] and c = tc_[o[k] ^ f], as (h, l), with the two
// products of each item as a packed pair. A grid above three times the thread's sum of |hi x hi|
// products is chosen first (as grid_transform does); each hi product P is then cut into
// H = RN(P + c) - c, exact on the grid, whose sum is exact, and the rest b c - H, formed by one FMA
// with -H (exactly -H as c - RN(P + c)) plus the hi x lo cross products, summed in FP32 (it is
// below the grid's unit). The expectation's pair sums Re A (A = conj(psi_{y^f}) psi_y) and the
// transition amplitude's Re and Im of conj(bra_y) ket_{y^f} are such sums.
template <typename E, bool kLo, bool kIm>
__device__ __forceinline__ void cross_sum_packed(const E* tb_, const E* tc_, const uint32_t (&o)[8], uint32_t f,
                                                 float& h, float& l) {
    // operand pairs: (b.re, b.im) times (c.re, c.im), or (c.im, c.re) for the imaginary part
    auto cs = [](const E& c) { return kIm ? make_float2(c.y, c.x) : make_float2(c.x, c.y); };
    // hi x hi products (kept for the cut below) and the sum of their magnitudes as a tree: the
    // eight items are independent until the sums, which take three levels instead of a chain
    float2 P[8];
    float t[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const E b = tb_[o[k]], c = tc_[o[k] ^ f];
        P[k] = __fmul2_rn(make_float2(b.x, b.y), cs(c));
        t[k] = __fadd_rn(fabsf(P[k].x), fabsf(P[k].y));
    }
#pragma unroll
    for (int s = 1; s < 8; s <<= 1)
#pragma unroll
        for (int k = 0; k < 8; k += 2 * s) t[k] = __fadd_rn(t[k], t[k + s]);
    uint32_t e = (__float_as_uint(t[0]) >> 23) & 0xFFu;
    e = e > 250u ? 250u : e;
    const float c = __uint_as_float(((e + 2u) << 23) | 0x400000u);  // 1.5 * 2^(e - 125) > 3 S
    const float2 C2 = make_float2(c, c), NC2 = make_float2(-c, -c), M1 = make_float2(-1.f, -1.f);
    float2 H[8], L[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const E b = tb_[o[k]], cc = tc_[o[k] ^ f];
        const float2 bh = make_float2(b.x, b.y), ch = cs(cc);
        const float2 T = __fadd2_rn(P[k], C2);
        H[k] = __fadd2_rn(T, NC2);
        const float2 NH = __ffma2_rn(T, M1, C2);  // c - T = -H exactly
        L[k] = __ffma2_rn(bh, ch, NH);            // b c - H (one rounding, far below the grid's unit)
        if constexpr (kLo) {
            const float4& b4 = reinterpret_cast<const float4&>(b);
            const float4& c4 = reinterpret_cast<const float4&>(cc);
            L[k] = __ffma2_rn(bh, kIm ? make_float2(c4.w, c4.z) : make_float2(c4.z, c4.w), L[k]);
            L[k] = __ffma2_rn(make_float2(b4.z, b4.w), ch, L[k]);
        }
    }
    // the H sum is exact in any order (multiples of the grid's unit, far below 2^24 of it)
#pragma unroll
    for (int s = 1; s < 8; s <<= 1)
#pragma unroll
        for (int k = 0; k < 8; k += 2 * s) {
            H[k] = __fadd2_rn(H[k], H[k + s]);
            L[k] = __fadd2_rn(L[k], L[k + s]);
        }
    h = kIm ? __fsub_rn(H[0].x, H[0].y) : __fadd_rn(H[0].x, H[0].y);  // both on the grid: exact
    l = kIm ? __fsub_rn(L[0].x, L[0].y) : __fadd_rn(L[0].x, L[0].y);
}

template <typename E, bool kLo>
__device__ __forceinline__ void re_sum_packed(const E* tile, uint32_t tb, uint32_t f, const uint32_t* im, float& h,
                                              float& l) {
    uint32_t o[8];
    o[0] = tb;
#pragma unroll
    for (int k = 1; k < 8; k++) o[k] = o[k ^ (1 << top_bit(k))] | im[top_bit(k)];
    cross_sum_packed<E, kLo, false>(tile, tile, o, f, h, l);
}

template <typename E, bool kLo, int kKind>
__device__ __forceinline__ void group_kind(const TileGroup& G, const TileSlot* S, const E* tile, const float2* gam,
                                           uint32_t tid, uint32_t tb, float& ah, float& al) {
    uint32_t im[4];
#pragma unroll
    for (int i = 0; i < 4; i++) im[i] = G.imask[i];
    const bool full = G.wht != 0;
    if constexpr (kKind == kTileRe) {
        if (!full) {  // only the plain sum of Re A: packed pairs
            float qh[1], ql[1];
            re_sum_packed<E, kLo>(tile, tb, G.f, im, qh[0], ql[0]);
            slot_sums<0, 1>(G, S, gam, tid, qh, ql, ah, al);
            return;
        }
    }
    float qh[16], ql[16];
    group_values<E, kLo, kKind>(tile, tb, G.f, im, qh, ql);
    if (kKind == kTileDiag) {
        grid_transform<16>(qh, ql, full);
    } else {
        if (kKind & kTileRe) grid_transform<8>(qh, ql, full);
        if (kKind & kTileIm) grid_transform<8>(qh + 8, ql + 8, full);
    }
    constexpr int B0 = kKind == kTileIm ? 8 : 0;
    constexpr int B1 = kKind == kTileRe ? 8 : 16;
    if (full) {
        slot_sums<B0, B1>(G, S, gam, tid, qh, ql, ah, al);
    } else {  // every slot of the group uses the plain sum, Q[0] or Q[8]
        if (kKind != kTileIm) slot_sums<0, 1>(G, S, gam, tid, qh, ql, ah, al);
        if (kKind & kTileIm) slot_sums<8, 9>(G, S, gam, tid, qh, ql, ah, al);
    }
}

__device__ __forceinline__ uint32_t thread_slot(uint32_t tid, uint32_t ex) {
    // thread index -> tile slot of its item 0: zero bits inserted at the 4 excluded positions
    uint32_t tb = tid;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const uint32_t p = (ex >> (8 * e)) & 0xFFu;
        const uint32_t lo = tb & ((1u << p) - 1u);
        tb = ((tb ^ lo) << 1) | lo;
    }
    return tb;
}

// two flip groups that use only Re A and its plain sum, evaluated together so that their
// independent arithmetic interleaves
template <typename E, bool kLo>
__device__ __forceinline__ void tile_group_pair_re(const TileGroup& G1, const TileGroup& G2, const TileSlot* S,
                                                   const E* tile, const float2* gam, uint32_t tid, uint32_t tb1,
                                                   uint32_t tb2, float& ah, float& al) {
    uint32_t im1[4], im2[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        im1[i] = G1.imask[i];
        im2[i] = G2.imask[i];
    }
    float qh1[1], ql1[1], qh2[1], ql2[1];
    re_sum_packed<E, kLo>(tile, tb1, G1.f, im1, qh1[0], ql1[0]);
    re_sum_packed<E, kLo>(tile, tb2, G2.f, im2, qh2[0], ql2[0]);
    slot_sums<0, 1>(G1, S, gam, tid, qh1, ql1, ah, al);
    slot_sums<0, 1>(G2, S, gam, tid, qh2, ql2, ah, al);
}

// one group's contribution from the tile in shared memory
template <typename E, bool kLo>
__device__ __forceinline__ void tile_group(const TileGroup& G, const TileSlot* __restrict__ S, const E* tile,
                                           const float2* gam, uint32_t tid, uint32_t tb, float& ah, float& al) {
    switch (G.kind) {
        case kTileDiag: group_kind<E, kLo, kTileDiag>(G, S, tile, gam, tid, tb, ah, al); break;
        case kTileRe: group_kind<E, kLo, kTileRe>(G, S, tile, gam, tid, tb, ah, al); break;
        case kTileIm: group_kind<E, kLo, kTileIm>(G, S, tile, gam, tid, tb, ah, al); break;
        default: group_kind<E, kLo, kTileReIm>(G, S, tile, gam, tid, tb, ah, al); break;
    }
}

__device__ __forceinline__ uint64_t deposit64(uint64_t x, uint64_t mask) {
    uint64_t r = 0;
    for (uint64_t m = mask; m && x; m &= m - 1, x >>= 1)
        if (x & 1) r |= m & (~m + 1);
    return r;
}

constexpr size_t tile_smem_bytes(size_t elem) {
    return elem * kTileAmps + sizeof(float2) * kTileMaxSlots + sizeof(TileSlot) * kTileMaxSlots +
           sizeof(TileTerm) * kTileMaxTerms + sizeof(uint16_t) * kTileMaxGroups * kTileThreads;
}

template <typename C>
__global__ void __launch_bounds__(kTileThreads, 2) k_expect_tiled(const C* __restrict__ psi,
                                                                   const __grid_constant__ TileParams P,
                                                                   double* __restrict__ part) {
    using E = typename TileElem<C>::T;
    extern __shared__ __align__(16) unsigned char tsm[];
    E* tile = reinterpret_cast<E*>(tsm);
    float2* gam = reinterpret_cast<float2*>(tsm + sizeof(E) * kTileAmps);
    TileSlot* slots = reinterpret_cast<TileSlot*>(gam + kTileMaxSlots);
    TileTerm* terms = reinterpret_cast<TileTerm*>(slots + kTileMaxSlots);
    // tile slot of each group's item 0 for each thread, formed once (the same for every tile)
    uint16_t* tbt = reinterpret_cast<uint16_t*>(terms + kTileMaxTerms);
    const uint32_t tid = threadIdx.x;
    for (int i = tid; i < P.nslots; i += kTileThreads) slots[i] = P.s[i];
    for (int i = tid; i < P.nterms; i += kTileThreads) terms[i] = P.t[i];
    for (int g = 0; g < P.ngroups; g++) tbt[g * kTileThreads + tid] = uint16_t(thread_slot(tid, P.g[g].excl));
    const int namps = 1 << P.b;
    uint64_t dthr = 0;
    for (int i = 0; i < 8 && i < P.b; i++)
        if ((tid >> i) & 1) dthr |= 1ull << P.tpos[i];
    // tile slots above 2^b (virtual tile bits of a small state) hold zero amplitudes
    for (int j = namps + int(tid); j < kTileAmps; j += kTileThreads) tile[j] = E{};
    uint64_t rbase = deposit64(blockIdx.x, P.rest_mask);
    const uint64_t step = deposit64(gridDim.x, P.rest_mask);
    double acc = 0.0;
    __syncthreads();
    for (uint64_t r = blockIdx.x; r < P.n_tiles; r += gridDim.x) {
        __syncthreads();  // the previous tile's readers are done
        // two halves of 8 amplitudes per thread: 8 loads in flight, then their stores
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {
            constexpr int kH = kTileAmps / kTileThreads / 2;
            C v[kH];
#pragma unroll
            for (int k = 0; k < kH; k++)
                if (int(tid) + kTileThreads * (hf * kH + k) < namps) v[k] = psi[rbase | dthr | P.dep_hi[hf * kH + k]];
#pragma unroll
            for (int k = 0; k < kH; k++)
                if (int(tid) + kTileThreads * (hf * kH + k) < namps)
                    tile[tid + kTileThreads * (hf * kH + k)] = to_tile(v[k]);
        }
        // complex64: the lines of this CTA's next tile into L2 while this one is evaluated
        // (measured at n = 30 on the Ising chain's three reads: 25.7 -> 24.3 ms; for complex128
        // it measured slower, 32.4 -> 33.1 ms, and is not issued)
        if (sizeof(C) == sizeof(float2) && r + gridDim.x < P.n_tiles) {
            const uint64_t rn = ((rbase | ~P.rest_mask) + step) & P.rest_mask;
#pragma unroll
            for (int k = 0; k < kTileAmps / kTileThreads; k++)
                if (int(tid) + kTileThreads * k < namps)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + (rn | dthr | P.dep_hi[k])));
        }
        // slot coefficients for this tile: sum of alpha (-1)^{popc(r & zR)}
        if (int(tid) < P.nslots) {
            const TileSlot sl = slots[tid];
            double gsum = 0.0;
            for (int t = sl.term0; t < sl.term0 + sl.nterm; t++) {
                const TileTerm T = terms[t];
                gsum += (__popcll(rbase & T.zR) & 1) ? -T.alpha : T.alpha;
            }
            float h, l;
            split_double_int(gsum, h, l);
            gam[tid] = make_float2(h, l);
        }
        __syncthreads();
        float ah = 0.f, al = 0.f;
        for (int g = 0; g < P.ngroups;) {
            const TileGroup& G = P.g[g];
            if (g + 1 < P.ngroups && G.kind == kTileRe && !G.wht && P.g[g + 1].kind == kTileRe && !P.g[g + 1].wht) {
                tile_group_pair_re<E, TileElem<C>::kLo>(G, P.g[g + 1], slots, tile, gam, tid, tbt[g * kTileThreads + tid],
                                                        tbt[(g + 1) * kTileThreads + tid], ah, al);
                g += 2;
            } else {
                tile_group<E, TileElem<C>::kLo>(G, slots, tile, gam, tid, tbt[g * kTileThreads + tid], ah, al);
                g += 1;
            }
        }
        acc += widen_float_int(ah) + widen_float_int(al);
        rbase = ((rbase | ~P.rest_mask) + step) & P.rest_mask;
    }
    __shared__ double sh[kTileThreads / 32];
    const double tot = block_sum<kTileThreads>(acc, sh);
    if (tid == 0) {
        part[2 * blockIdx.x] = tot;
        part[2 * blockIdx.x + 1] = 0.0;
    }
}

// ---------------------------------------------------------------- diagonal observables
// E = sum_x c(r(x)) |psi_x|^2 in one streaming read. Each CTA forms the table c(r) for every
// index r of the union of the Z qubits in FP64 (the sum over terms of alpha_t with the sign of
// r's bits at term t's qubits) and keeps it as double-float in shared memory. Chunks of 2^11
// amplitudes, four per thread: r(x) = r(chunk base) | r(x mod 2^11) (a gather is an OR over
// disjoint bits), the low part fixed per thread. |psi_x|^2 is formed as a double-float (exact
// hi x hi products), multiplied by the entry and added to a double-float accumulator per thread;
// per-block FP64 sums.
constexpr int kDiagObsThreads = 512;
constexpr int kDiagObsPer = 4;
constexpr int kDiagObsChunkBits = 11;
static_assert(kDiagObsThreads * kDiagObsPer == 1 << kDiagObsChunkBits, "chunk size");

__device__ __forceinline__ uint32_t gather_obs(uint64_t x, const uint32_t* run, int nrun) {
    uint32_t r = 0;
    for (int k = 0; k < nrun; k++) {
        const uint32_t c = run[k];
        r |= (uint32_t(x >> (c & 0xFFu)) & ((1u << ((c >> 8) & 0xFFu)) - 1u)) << (c >> 16);
    }
    return r;
}

// |v|^2 as a double-float (h, l) for each storage type
__device__ __forceinline__ void norm2_df(double2 v, float& h, float& l) {
    float rh, rl, ih, il;
    split_tile(v.x, rh, rl);
    split_tile(v.y, ih, il);
    df_dot2<true>(rh, rl, rh, rl, ih, il, ih, il, h, l);
}
__device__ __forceinline__ void norm2_df(float4 v, float& h, float& l) {
    df_dot2<true>(v.x, v.y, v.x, v.y, v.z, v.w, v.z, v.w, h, l);
}
__device__ __forceinline__ void norm2_df(float2 v, float& h, float& l) {
    df_dot2<false>(v.x, 0.f, v.x, 0.f, v.y, 0.f, v.y, 0.f, h, l);
}

template <typename C>
__global__ void __launch_bounds__(kDiagObsThreads, 2) k_expect_diag(const C* __restrict__ psi,
                                                                    const __grid_constant__ DiagObsParams P,
                                                                    double* __restrict__ part) {
    __shared__ float2 ctab[1 << kDiagObsBits];
    __shared__ double sh[kDiagObsThreads / 32];
    for (int r = threadIdx.x; r < (1 << P.m); r += kDiagObsThreads) {
        double c = 0.0;
        for (int t = 0; t < P.nterms; t++) c += (__popc(uint32_t(r) & P.z[t]) & 1) ? -P.alpha[t] : P.alpha[t];
        float h, l;
        split_double_int(c, h, l);
        ctab[r] = make_float2(h, l);
    }
    __syncthreads();
    uint32_t rl[kDiagObsPer];
#pragma unroll
    for (int u = 0; u < kDiagObsPer; u++) rl[u] = gather_obs(threadIdx.x + uint64_t(u) * kDiagObsThreads, P.run, P.nrun);
    float ah = 0.f, al = 0.f;
    const uint64_t n_chunks = (P.N + (1ull << kDiagObsChunkBits) - 1) >> kDiagObsChunkBits;
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint64_t base = ch << kDiagObsChunkBits;
        const uint32_t rh = gather_obs(base, P.run, P.nrun);
        C v[kDiagObsPer];
#pragma unroll
        for (int u = 0; u < kDiagObsPer; u++) {
            const uint64_t x = base + threadIdx.x + uint64_t(u) * kDiagObsThreads;
            if (x < P.N) v[u] = __ldcs(psi + x);
        }
#pragma unroll
        for (int u = 0; u < kDiagObsPer; u++) {
            const uint64_t x = base + threadIdx.x + uint64_t(u) * kDiagObsThreads;
            if (x >= P.N) continue;
            float h, l;
            norm2_df(v[u], h, l);
            const float2 c = ctab[rh | rl[u]];
            acc_prod(ah, al, c.x, c.y, h, l);
        }
    }
    const double tot = block_sum<kDiagObsThreads>(widen_float_int(ah) + widen_float_int(al), sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = tot;
        part[2 * blockIdx.x + 1] = 0.0;
    }
}

// ---------------------------------------------------------------- transition amplitude
// <bra| sum_t alpha_t P_t |ket> with P_t |x> = i^{nY} (-1)^{popc(x & z)} |x ^ f>: per flip group,
// sum_y conj(bra_y) ket_{y^f} alpha (-i)^{nY} (-1)^{popc(y & z)} over every y (no pairing), on
// tiles of 2^11 slots of both states. Each thread takes 8 items of a group (3 item bits); the
// slot's rotation (-i)^{nY} picks the component and sign of Q = Q_re + i Q_im for each output.
__device__ __forceinline__ uint32_t thread_slot3(uint32_t tid, uint32_t ex) {
    uint32_t tb = tid;
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const uint32_t p = (ex >> (8 * e)) & 0xFFu;
        const uint32_t lo = tb & ((1u << p) - 1u);
        tb = ((tb ^ lo) << 1) | lo;
    }
    return tb;
}

template <int B0, int B1>
__device__ __forceinline__ void trans_slot_sums(const TileGroup& G, const TileSlot* S, const float2* gam, uint32_t tid,
                                                const float* qr, const float* qrl, const float* qi,
                                                const float* qil, float& rh, float& rl, float& ih, float& il) {
#pragma unroll
    for (int bk = B0; bk < B1; bk++) {
        const int s1 = G.slot0 + G.bstart[bk + 1];
        for (int s = G.slot0 + G.bstart[bk]; s < s1; s++) {
            const float2 g = gam[s];
            const TileSlot sl = S[s];
            const uint32_t flip = uint32_t(__popc(tid & sl.zthr) & 1) << 31;
            const uint32_t rot = sl.pad;
            const bool odd = rot & 1u;
            const uint32_t fr = flip ^ (uint32_t(rot >= 2u) << 31);
            const uint32_t fi = flip ^ (uint32_t(rot == 1u || rot == 2u) << 31);
            acc_prod(rh, rl, flip_sign(g.x, fr), flip_sign(g.y, fr), odd ? qi[bk] : qr[bk], odd ? qil[bk] : qrl[bk]);
            acc_prod(ih, il, flip_sign(g.x, fi), flip_sign(g.y, fi), odd ? qr[bk] : qi[bk], odd ? qrl[bk] : qil[bk]);
        }
    }
}

template <typename E, bool kLo>
__device__ __forceinline__ void trans_group(const TileGroup& G, const TileSlot* S, const E* tbra, const E* tket,
                                            const float2* gam, uint32_t tid, uint32_t tb, float& rh, float& rl,
                                            float& ih, float& il) {
    const uint32_t f = G.f;
    uint32_t o[8];
    o[0] = tb;
#pragma unroll
    for (int k = 1; k < 8; k++) o[k] = o[k ^ (1 << top_bit(k))] | G.imask[top_bit(k)];
    if (!G.wht) {  // every slot uses the plain sums: packed pairs
        float qr[1], qrl[1], qi[1], qil[1];
        cross_sum_packed<E, kLo, false>(tbra, tket, o, f, qr[0], qrl[0]);
        cross_sum_packed<E, kLo, true>(tbra, tket, o, f, qi[0], qil[0]);
        trans_slot_sums<0, 1>(G, S, gam, tid, qr, qrl, qi, qil, rh, rl, ih, il);
        return;
    }
    float qr[8], qrl[8], qi[8], qil[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const DFc b = dfc(tbra[o[k]]), c = dfc(tket[o[k] ^ f]);
        // conj(b) c = (b.re c.re + b.im c.im) + i (b.re c.im - b.im c.re)
        df_dot2<kLo>(b.rh, b.rl, c.rh, c.rl, b.ih, b.il, c.ih, c.il, qr[k], qrl[k]);
        df_dot2<kLo>(b.rh, b.rl, c.ih, c.il, -b.ih, -b.il, c.rh, c.rl, qi[k], qil[k]);
    }
    grid_transform<8>(qr, qrl, true);
    grid_transform<8>(qi, qil, true);
    trans_slot_sums<0, 8>(G, S, gam, tid, qr, qrl, qi, qil, rh, rl, ih, il);
}

constexpr size_t trans_smem_bytes(size_t elem) {
    return 2 * elem * (size_t(1) << kTransBits) + sizeof(float2) * kTileMaxSlots + sizeof(TileSlot) * kTileMaxSlots +
           sizeof(TileTerm) * kTileMaxTerms + sizeof(uint16_t) * kTileMaxGroups * kTileThreads;
}

template <typename C>
__global__ void __launch_bounds__(kTileThreads, 2) k_transition_tiled(const C* __restrict__ bra,
                                                                       const C* __restrict__ ket,
                                                                       const __grid_constant__ TileParams P,
                                                                       double* __restrict__ part) {
    using E = typename TileElem<C>::T;
    constexpr int kA = 1 << kTransBits;
    extern __shared__ __align__(16) unsigned char tsm[];
    E* tbra = reinterpret_cast<E*>(tsm);
    E* tket = tbra + kA;
    float2* gam = reinterpret_cast<float2*>(tket + kA);
    TileSlot* slots = reinterpret_cast<TileSlot*>(gam + kTileMaxSlots);
    TileTerm* terms = reinterpret_cast<TileTerm*>(slots + kTileMaxSlots);
    // tile slot of each group's item 0 for each thread, formed once (the same for every tile)
    uint16_t* tbt = reinterpret_cast<uint16_t*>(terms + kTileMaxTerms);
    const uint32_t tid = threadIdx.x;
    for (int i = tid; i < P.nslots; i += kTileThreads) slots[i] = P.s[i];
    for (int i = tid; i < P.nterms; i += kTileThreads) terms[i] = P.t[i];
    for (int g = 0; g < P.ngroups; g++) tbt[g * kTileThreads + tid] = uint16_t(thread_slot3(tid, P.g[g].excl));
    const int namps = 1 << P.b;
    for (int j = namps + int(tid); j < kA; j += kTileThreads) {
        tbra[j] = E{};
        tket[j] = E{};
    }
    uint64_t dthr = 0;
    for (int i = 0; i < 8 && i < P.b; i++)
        if ((tid >> i) & 1) dthr |= 1ull << P.tpos[i];
    uint64_t rbase = deposit64(blockIdx.x, P.rest_mask);
    const uint64_t step = deposit64(gridDim.x, P.rest_mask);
    double accr = 0.0, acci = 0.0;
    __syncthreads();
    for (uint64_t r = blockIdx.x; r < P.n_tiles; r += gridDim.x) {
        __syncthreads();  // the previous tile's readers are done
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {
            constexpr int kH = kA / kTileThreads / 2;
            C v[kH], w[kH];
#pragma unroll
            for (int k = 0; k < kH; k++) {
                const int j = int(tid) + kTileThreads * (hf * kH + k);
                if (j < namps) {
                    const uint64_t a = rbase | dthr | P.dep_hi[hf * kH + k];
                    v[k] = bra[a];
                    w[k] = ket[a];
                }
            }
#pragma unroll
            for (int k = 0; k < kH; k++) {
                const int j = int(tid) + kTileThreads * (hf * kH + k);
                if (j < namps) {
                    tbra[j] = to_tile(v[k]);
                    tket[j] = to_tile(w[k]);
                }
            }
        }
        if (int(tid) < P.nslots) {
            const TileSlot sl = slots[tid];
            double gsum = 0.0;
            for (int t = sl.term0; t < sl.term0 + sl.nterm; t++) {
                const TileTerm T = terms[t];
                gsum += (__popcll(rbase & T.zR) & 1) ? -T.alpha : T.alpha;
            }
            float h, l;
            split_double_int(gsum, h, l);
            gam[tid] = make_float2(h, l);
        }
        __syncthreads();
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int g = 0; g < P.ngroups; g++)
            trans_group<E, TileElem<C>::kLo>(P.g[g], slots, tbra, tket, gam, tid, tbt[g * kTileThreads + tid], rh, rl,
                                             ih, il);
        accr += widen_float_int(rh) + widen_float_int(rl);
        acci += widen_float_int(ih) + widen_float_int(il);
        rbase = ((rbase | ~P.rest_mask) + step) & P.rest_mask;
    }
    __shared__ double sh[kTileThreads / 32];
    const double tr = block_sum<kTileThreads>(accr, sh);
    const double ti = block_sum<kTileThreads>(acci, sh);
    if (tid == 0) {
        part[2 * blockIdx.x] = tr;
        part[2 * blockIdx.x + 1] = ti;
    }
}

// CTAs per SM of the tiled kernels at their shared-memory size (attribute raised once per device)
template <typename C>
int trans_blocks_per_sm() {
    static PerDevice setup;
    static int b[kMaxDevices];
    setup.once([](int dev) {
        const size_t bytes = trans_smem_bytes(sizeof(typename TileElem<C>::T));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_transition_tiled<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
        int nb = 0;
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_transition_tiled<C>, kTileThreads, bytes));
        b[dev] = nb > 0 ? nb : 1;
    });
    return b[current_device()];
}

template <typename C>
int tile_blocks_per_sm() {
    static PerDevice setup;
    static int b[kMaxDevices];
    setup.once([](int dev) {
        const size_t bytes = tile_smem_bytes(sizeof(typename TileElem<C>::T));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_expect_tiled<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
        int nb = 0;
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_expect_tiled<C>, kTileThreads, bytes));
        b[dev] = nb > 0 ? nb : 1;
    });
    return b[current_device()];
}

template <typename C>
unsigned pass_grid_t(const TileParams& P) {
    const uint64_t want = uint64_t(tile_blocks_per_sm<C>()) * uint64_t(sm_count());
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(P.n_tiles, want)));
}

// ---------------------------------------------------------------- host planner
uint32_t compress_bits(uint64_t x, const int* pos, int npos) {
    uint32_t r = 0;
    for (int i = 0; i < npos; i++)
        if ((x >> pos[i]) & 1) r |= 1u << i;
    return r;
}

struct Chunk {
    const PauliGroup* g;
    size_t t0, t1;
};

void build_group(const Chunk& ch, const int* tpos, int b, uint64_t T, TileParams& P) {
    QS_REQUIRE(P.ngroups < kTileMaxGroups, "tile pass group overflow");
    TileGroup& G = P.g[P.ngroups++];
    G = TileGroup();
    const uint64_t f = ch.g->xmask;
    G.f = compress_bits(f, tpos, b);
    const int pivot = f ? 31 - __builtin_clz(G.f) : -1;
    const int nitem = f ? 3 : 4;
    // item bits: the tile-local bits (virtual ones included) where the fewest terms have Z
    // (ideally none: then no transform is needed), the highest first so that the low bits
    // index consecutive threads
    std::vector<std::pair<int, int>> cand;  // (score, -bit)
    for (int q = 0; q < kTileBits; q++) {
        if (q == pivot) continue;
        int score = 0;
        if (q < b)
            for (size_t t = ch.t0; t < ch.t1; t++) score += int((ch.g->zmask[t] >> tpos[q]) & 1);
        cand.push_back({score, -q});
    }
    std::sort(cand.begin(), cand.end());
    int items[4] = {0, 0, 0, 0};
    for (int i = 0; i < nitem; i++) items[i] = -cand[size_t(i)].second;
    std::sort(items, items + nitem);
    std::vector<int> excl(items, items + nitem);
    if (pivot >= 0) excl.push_back(pivot);
    std::sort(excl.begin(), excl.end());
    int thr[kTileBits];
    int nthr = 0;
    for (int q = 0; q < kTileBits; q++)
        if (std::find(excl.begin(), excl.end(), q) == excl.end()) thr[nthr++] = q;
    QS_REQUIRE(excl.size() == 4 && nthr == 8, "tile bit split");
    for (int e = 0; e < 4; e++) G.excl |= uint32_t(excl[size_t(e)]) << (8 * e);
    for (int i = 0; i < nitem; i++) G.imask[i] = 1u << items[i];
    // terms -> slots keyed by (bucket, thread mask), in key order
    std::map<std::pair<int, uint32_t>, std::vector<TileTerm>> keyed;
    int comps = 0;
    for (size_t t = ch.t0; t < ch.t1; t++) {
        const uint64_t z = ch.g->zmask[t];
        const uint32_t zl = compress_bits(z & T, tpos, b);
        const int m = int(compress_bits(zl, items, nitem));
        const uint32_t zthr = compress_bits(zl, thr, nthr);
        const int nY = __builtin_popcountll(f & z);
        int comp = 0;
        double a = ch.g->coef[t];
        if (f) {
            comp = nY & 1;
            const int e = comp ? (nY + 1) / 2 : nY / 2;
            a *= (e & 1) ? -2.0 : 2.0;
        }
        comps |= 1 << comp;
        if (m) G.wht = 1;
        keyed[{comp * 8 + m, zthr}].push_back(TileTerm{z & ~T, a});
    }
    G.kind = uint8_t(f ? comps : int(kTileDiag));
    G.slot0 = uint16_t(P.nslots);
    int cnt[16] = {};
    for (const auto& kv : keyed) {
        QS_REQUIRE(P.nslots < kTileMaxSlots, "tile pass slot overflow");
        TileSlot& S = P.s[P.nslots++];
        S.term0 = uint16_t(P.nterms);
        S.nterm = uint16_t(kv.second.size());
        S.zthr = uint16_t(kv.first.second);
        S.bucket = uint8_t(kv.first.first);
        for (const TileTerm& tt : kv.second) {
            QS_REQUIRE(P.nterms < kTileMaxTerms, "tile pass term overflow");
            P.t[P.nterms++] = tt;
        }
        cnt[kv.first.first]++;
    }
    G.bstart[0] = 0;
    for (int k = 0; k < 16; k++) G.bstart[k + 1] = uint8_t(G.bstart[k] + cnt[k]);
}

}  // namespace

namespace {

// Packs the flip-mask groups into tiles of tbits qubits (qubits 0..2 plus tbits - 3 others, or
// the whole state) with the fewest new tile qubits per group; a group whose flip mask has more
// than tbits - 3 bits above qubit 2 goes to plan.heavy. build(chunk, tpos, b, T, P) adds a group.
template <class Build>
void pack_tiles(const std::vector<PauliGroup>& groups, int n, int tbits, ExpectPlan& plan, Build build) {
    const int b = std::min(n, tbits);
    const uint64_t full = n >= 64 ? ~0ull : ((1ull << n) - 1);
    const uint64_t low = n <= tbits ? full : ((1ull << kTileLowBits) - 1);
    const int hbudget = b - __builtin_popcountll(low);
    std::vector<const PauliGroup*> order;
    for (const auto& g : groups) order.push_back(&g);
    std::stable_sort(order.begin(), order.end(),
                     [](const PauliGroup* a, const PauliGroup* c) { return a->xmask < c->xmask; });
    struct Pass {
        uint64_t T;
        std::vector<Chunk> ch;
        int terms;
    };
    std::vector<Pass> passes;
    for (const PauliGroup* g : order) {
        const uint64_t h = g->xmask & ~low;
        if (__builtin_popcountll(h) > hbudget) {
            for (size_t t0 = 0; t0 < g->coef.size(); t0 += kHeavyChunkTerms)
                plan.heavy.push_back(HeavyChunk{g, t0, std::min(g->coef.size(), t0 + kHeavyChunkTerms)});
            continue;
        }
        for (size_t t0 = 0; t0 < g->coef.size(); t0 += kTileGroupTerms) {
            const size_t t1 = std::min(g->coef.size(), t0 + kTileGroupTerms);
            const int nt = int(t1 - t0);
            int best = -1, best_growth = 1 << 30;
            for (size_t p = 0; p < passes.size(); p++) {
                const Pass& B = passes[p];
                if (B.ch.size() >= size_t(kTileMaxGroups) || B.terms + nt > kTileMaxTerms) continue;
                const uint64_t U = B.T | h;
                if (__builtin_popcountll(U & ~low) > hbudget) continue;
                const int growth = __builtin_popcountll(U) - __builtin_popcountll(B.T);
                if (growth < best_growth) {
                    best_growth = growth;
                    best = int(p);
                }
            }
            if (best < 0) {
                passes.push_back(Pass{low | h, {}, 0});
                best = int(passes.size()) - 1;
            }
            passes[size_t(best)].T |= h;
            passes[size_t(best)].ch.push_back(Chunk{g, t0, t1});
            passes[size_t(best)].terms += nt;
        }
    }
    for (Pass& B : passes) {
        // pad T with the lowest unused qubits up to b bits
        for (int q = 0; q < n && __builtin_popcountll(B.T) < b; q++) B.T |= 1ull << q;
        TileParams P{};
        P.b = b;
        int tpos[kTileBits];
        int nt = 0;
        for (int q = 0; q < n; q++)
            if ((B.T >> q) & 1) tpos[nt++] = q;
        for (int i = 0; i < b; i++) P.tpos[i] = uint8_t(tpos[i]);
        P.rest_mask = full & ~B.T;
        P.n_tiles = 1ull << (n - b);
        for (int k = 0; k < (1 << (tbits - 8)); k++) {
            uint64_t o = 0;
            for (int i = 8; i < b; i++)
                if (((k << 8) >> i) & 1) o |= 1ull << tpos[i];
            P.dep_hi[k] = o;
        }
        for (const Chunk& c : B.ch) build(c, tpos, b, B.T, P);
        plan.passes.push_back(P);
        plan.tmask.push_back(B.T);
    }
}

// transition group: 3 item bits (no pivot: every tile slot y is a term), slots keyed by
// (item mask, thread mask, nY mod 4)
void build_trans_group(const Chunk& ch, const int* tpos, int b, uint64_t T, TileParams& P) {
    QS_REQUIRE(P.ngroups < kTileMaxGroups, "tile pass group overflow");
    TileGroup& G = P.g[P.ngroups++];
    G = TileGroup();
    const uint64_t f = ch.g->xmask;
    G.f = compress_bits(f, tpos, b);
    std::vector<std::pair<int, int>> cand;  // (score, -bit)
    for (int q = 0; q < kTransBits; q++) {
        int score = 0;
        if (q < b)
            for (size_t t = ch.t0; t < ch.t1; t++) score += int((ch.g->zmask[t] >> tpos[q]) & 1);
        cand.push_back({score, -q});
    }
    std::sort(cand.begin(), cand.end());
    int items[3];
    for (int i = 0; i < 3; i++) items[i] = -cand[size_t(i)].second;
    std::sort(items, items + 3);
    int thr[kTransBits];
    int nthr = 0;
    for (int q = 0; q < kTransBits; q++)
        if (q != items[0] && q != items[1] && q != items[2]) thr[nthr++] = q;
    QS_REQUIRE(nthr == 8, "tile bit split");
    for (int e = 0; e < 3; e++) G.excl |= uint32_t(items[e]) << (8 * e);
    for (int i = 0; i < 3; i++) G.imask[i] = 1u << items[i];
    std::map<std::tuple<int, uint32_t, int>, std::vector<TileTerm>> keyed;
    for (size_t t = ch.t0; t < ch.t1; t++) {
        const uint64_t z = ch.g->zmask[t];
        const uint32_t zl = compress_bits(z & T, tpos, b);
        const int m = int(compress_bits(zl, items, 3));
        const uint32_t zthr = compress_bits(zl, thr, nthr);
        if (m) G.wht = 1;
        keyed[std::make_tuple(m, zthr, __builtin_popcountll(f & z) & 3)].push_back(TileTerm{z & ~T, ch.g->coef[t]});
    }
    G.kind = kTileReIm;
    G.slot0 = uint16_t(P.nslots);
    int cnt[16] = {};
    for (const auto& kv : keyed) {
        QS_REQUIRE(P.nslots < kTileMaxSlots, "tile pass slot overflow");
        TileSlot& S = P.s[P.nslots++];
        S.term0 = uint16_t(P.nterms);
        S.nterm = uint16_t(kv.second.size());
        S.zthr = uint16_t(std::get<1>(kv.first));
        S.bucket = uint8_t(std::get<0>(kv.first));
        S.pad = uint8_t(std::get<2>(kv.first));  // (-i)^{nY} rotation
        for (const TileTerm& tt : kv.second) {
            QS_REQUIRE(P.nterms < kTileMaxTerms, "tile pass term overflow");
            P.t[P.nterms++] = tt;
        }
        cnt[std::get<0>(kv.first)]++;
    }
    G.bstart[0] = 0;
    for (int k = 0; k < 16; k++) G.bstart[k + 1] = uint8_t(G.bstart[k] + cnt[k]);
}

}  // namespace

// a diagonal observable whose Z qubits number at most kDiagObsBits (and whose table costs at
// most 2^17 term evaluations per CTA): the streaming pass's parameters, else false
bool plan_diag_obs(const std::vector<PauliGroup>& groups, int n, DiagObsParams& P) {
    if (groups.size() != 1 || groups[0].xmask != 0) return false;
    const PauliGroup& G = groups[0];
    uint64_t u = 0;
    for (uint64_t z : G.zmask) u |= z;
    const int m = __builtin_popcountll(u);
    const int nt = int(G.coef.size());
    if (m > kDiagObsBits || nt > kDiagObsMaxTerms || (uint64_t(nt) << m) > (1ull << 17)) return false;
    int pos[64], np_ = 0;
    for (int q = 0; q < n; q++)
        if ((u >> q) & 1) pos[np_++] = q;
    P.N = 1ull << n;
    P.m = m;
    P.nterms = nt;
    P.nrun = 0;
    for (int j = 0; j < np_;) {  // runs of consecutive qubits
        int k = j + 1;
        while (k < np_ && pos[k] == pos[k - 1] + 1) k++;
        P.run[P.nrun++] = uint32_t(pos[j]) | (uint32_t(k - j) << 8) | (uint32_t(j) << 16);
        j = k;
    }
    for (int t = 0; t < nt; t++) {
        P.z[t] = compress_bits(G.zmask[t], pos, np_);
        P.alpha[t] = G.coef[t];
    }
    return true;
}

ExpectPlan plan_expectation(const std::vector<PauliGroup>& groups, int n) {
    ExpectPlan plan;
    if (plan_diag_obs(groups, n, plan.dp)) {
        plan.diag = true;
        uint64_t u = 0;
        for (uint64_t z : groups[0].zmask) u |= z;
        plan.tmask.push_back(u);
        return plan;
    }
    pack_tiles(groups, n, kTileBits, plan, build_group);
    // groups that use only the plain sum of Re A first, so that the kernel takes them in pairs
    for (TileParams& P : plan.passes)
        std::stable_partition(P.g, P.g + P.ngroups, [](const TileGroup& G) { return G.kind == kTileRe && !G.wht; });
    return plan;
}

ExpectPlan plan_transition(const std::vector<PauliGroup>& groups, int n) {
    ExpectPlan plan;
    pack_tiles(groups, n, kTransBits, plan, build_trans_group);
    return plan;
}

unsigned expect_diag_grid(int n, Arith ar) {
    static PerDevice setup;
    static int resident_of[kMaxDevices][3];
    setup.once([](int dev) {
        int* r = resident_of[dev];
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[0], k_expect_diag<float2>, kDiagObsThreads, 0));
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[1], k_expect_diag<double2>, kDiagObsThreads, 0));
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[2], k_expect_diag<float4>, kDiagObsThreads, 0));
    });
    const int res = std::max(1, resident_of[current_device()][ar == Arith::F32 ? 0 : ar == Arith::F64 ? 1 : 2]);
    const uint64_t chunks = ((1ull << n) + (1ull << kDiagObsChunkBits) - 1) >> kDiagObsChunkBits;
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(chunks, uint64_t(res) * uint64_t(sm_count()))));
}

void launch_expect_diag(const DiagObsParams& P, const void* psi, Arith ar, double* part, unsigned grid,
                        cudaStream_t st) {
    switch (ar) {
        case Arith::F32:
            k_expect_diag<float2><<<grid, kDiagObsThreads, 0, st>>>(static_cast<const float2*>(psi), P, part);
            break;
        case Arith::F64:
            k_expect_diag<double2><<<grid, kDiagObsThreads, 0, st>>>(static_cast<const double2*>(psi), P, part);
            break;
        default:
            k_expect_diag<float4><<<grid, kDiagObsThreads, 0, st>>>(static_cast<const float4*>(psi), P, part);
            break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

unsigned expect_pass_grid(const TileParams& P, Arith ar) {
    switch (ar) {
        case Arith::F32: return pass_grid_t<float2>(P);
        case Arith::F64: return pass_grid_t<double2>(P);
        default: return pass_grid_t<float4>(P);
    }
}

void launch_expect_pass(const TileParams& P, const void* psi, Arith ar, double* part, unsigned grid,
                        cudaStream_t st) {
    switch (ar) {
        case Arith::F32:
            tile_blocks_per_sm<float2>();
            k_expect_tiled<float2><<<grid, kTileThreads, tile_smem_bytes(sizeof(float2)), st>>>(
                static_cast<const float2*>(psi), P, part);
            break;
        case Arith::F64:
            tile_blocks_per_sm<double2>();
            k_expect_tiled<double2><<<grid, kTileThreads, tile_smem_bytes(sizeof(float4)), st>>>(
                static_cast<const double2*>(psi), P, part);
            break;
        default:
            tile_blocks_per_sm<float4>();
            k_expect_tiled<float4><<<grid, kTileThreads, tile_smem_bytes(sizeof(float4)), st>>>(
                static_cast<const float4*>(psi), P, part);
            break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

unsigned trans_pass_grid(const TileParams& P, Arith ar) {
    int bps = 1;
    switch (ar) {
        case Arith::F32: bps = trans_blocks_per_sm<float2>(); break;
        case Arith::F64: bps = trans_blocks_per_sm<double2>(); break;
        default: bps = trans_blocks_per_sm<float4>(); break;
    }
    const uint64_t want = uint64_t(bps) * uint64_t(sm_count());
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(P.n_tiles, want)));
}

void launch_transition_pass(const TileParams& P, const void* bra, const void* ket, Arith ar, double* part,
                            unsigned grid, cudaStream_t st) {
    switch (ar) {
        case Arith::F32:
            trans_blocks_per_sm<float2>();
            k_transition_tiled<float2><<<grid, kTileThreads, trans_smem_bytes(sizeof(float2)), st>>>(
                static_cast<const float2*>(bra), static_cast<const float2*>(ket), P, part);
            break;
        case Arith::F64:
            trans_blocks_per_sm<double2>();
            k_transition_tiled<double2><<<grid, kTileThreads, trans_smem_bytes(sizeof(float4)), st>>>(
                static_cast<const double2*>(bra), static_cast<const double2*>(ket), P, part);
            break;
        default:
            trans_blocks_per_sm<float4>();
            k_transition_tiled<float4><<<grid, kTileThreads, trans_smem_bytes(sizeof(float4)), st>>>(
                static_cast<const float4*>(bra), static_cast<const float4*>(ket), P, part);
            break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

}  // namespace qs
