// Fused 4-qubit dense blocks on a double-float complex128 state with the tensor cores
// (tcgen05.mma kind::f16, bf16 operands, FP32 accumulation in TMEM), exact-product splitting.
//
// A fused block applies a 16 x 16 complex matrix K~ to 2^(n-4) vectors of 16 amplitudes
// (Eq. update_mat with m = 4), a dense (16 x 16) . (16 x 2^(n-4)) contraction. As real
// arithmetic with interleaved (re, im) indices, y = A v with A the 32 x 32 real form of K~.
//
// Precision (the splitting method of Ozaki, Ogita, Oishi and Rump): every row n of A is scaled
// by a power of two mu_n >= max |A_n.|, every group vector v by a power of two nu >= max |v|,
// and both are cut into six slices of 8 significant bits on fixed grids, slice s a multiple of
// 2^-8(s+1). A product of a state slice s and a matrix slice t is then an exact multiple of
// 2^-8(s+t+2), every sum of the products with the same s + t = d is an integer number of those
// units below 2^24, and the tensor cores add them without rounding (checked on the hardware
// for sums up to 2^23.3 units). The 26 products with s + t <= 6 go to seven FP32 accumulators
// D_0..D_6, one per d; D_6 + D_5 + D_4 is summed in FP32 (its rounding lies below 2^-50 of the
// output scale), then D_3..D_0 are added exactly (each D_d is a multiple of the unit in the
// last place of the partial sum below it, so Fast2Sum is error-free) into a double-float value,
// scaled back by mu_n nu. What is dropped (slice remainders below
// 2^-48 and the products with s + t >= 7) bounds the error at about 2^-45 of max|v| max|K~|
// per output, the accuracy of the double-float CUDA-core kernels.
//
// Tile: 128 groups (the MMA's M = 128, TMEM lane = group), K = 32 real inputs. The stacked
// matrix slices [B_0; ...; B_5] (192 x 32) let one MMA per state slice s and K-step cover all
// its products: columns (s + t) * 32 of the accumulator block receive A_s B_t, so a single
// MMA with N = 32 * min(6, 7 - s) feeds diagonals s..min(s + 5, 6).
//
// Pipeline: two CTAs per SM (256 threads, ~110 KB of shared memory and 256 TMEM columns each).
// A thread owns half of one group (8 amplitudes): it loads them straight into registers,
// slices them, and later writes that half's outputs straight back, so no staging copies are
// needed (for low targets the loads and stores are strided; the rest of each 32-byte sector is
// touched by the same thread and served by L2). Per tile j: the loads of tile j + 1 are issued,
// tile j is sliced into the second slice buffer while the MMAs of tile j - 1 run, tile j - 1's
// accumulators are folded and stored, and the MMAs of tile j start. One thread issues the MMAs
// and commits them to an mbarrier; every thread waits on that mbarrier itself before it reads
// the accumulators (no block barrier after the wait). Every wait is bounded; on expiry the warp
// (by a vote) and then the block stop folding and issuing, the kernel records an error, waits
// (bounded) for its MMAs and frees TMEM.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kOzQ = 4;                 // targets
constexpr int kOzD = 1 << kOzQ;         // amplitudes per group
constexpr int kOzR = 2 * kOzD;          // reals per group (K and N of one product)
constexpr int kOzTG = 128;              // groups per tile (M)
constexpr int kOzNS = 6;                // slices per operand
constexpr int kOzND = 7;                // accumulated diagonals d = s + t <= 6
constexpr int kOzThreads = 256;                                // two CTAs per SM
constexpr int kOzAmpsPerThread = kOzD / (kOzThreads / kOzTG);  // 8
constexpr uint32_t kOzSbo = (kOzR / 8) * 128;                  // 8-row group stride (K-major)
constexpr uint32_t kOzLbo = 128;
constexpr size_t kOzSlice = size_t(kOzTG) * kOzR * 2;          // one state slice, bf16
constexpr size_t kOzABuf = kOzNS * kOzSlice;                   // 48 KB
constexpr size_t kOzMat = size_t(kOzNS) * kOzR * kOzR * 2;     // 12 KB
constexpr int kOzAccCols = kOzND * kOzR;                       // 224 columns per accumulator set
constexpr int kOzTmemCols = 256;                               // one set, rounded to a power of 2
constexpr long long kOzSpinLimit = 1ll << 22;

static_assert(kOzAccCols <= kOzTmemCols, "accumulators fit the TMEM allocation");
static_assert(kOzND == 7, "the epilogue folds seven diagonals");

// shared-memory plan (bytes), ~110 KB: two CTAs per SM
constexpr size_t kOffA = 0;                             // 2 x 48 KB state slices
constexpr size_t kOffMat = kOffA + 2 * kOzABuf;         // 12 KB
constexpr size_t kOffMu = kOffMat + kOzMat;             // 32 floats
constexpr size_t kOffNuPart = kOffMu + kOzR * 4;        // 2 x 128 floats
constexpr size_t kOzSmem = kOffNuPart + 2 * kOzTG * 4;

struct OzParams {
    IndexPlan ip;            // 4 targets (and controls) inserted
    uint64_t offs[kOzD];     // s(w), targets ascending
    uint64_t n_groups;
    long long wait_spins;    // try_wait attempts of each accumulator wait before it gives up
    int force_late;          // test hook: the first accumulator wait reports a timeout at once
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major core-matrix offset of bf16 element (row r, column k), K = 32
__device__ __forceinline__ uint32_t kmaj(uint32_t r, uint32_t k) {
    return (r >> 3) * kOzSbo + (k >> 3) * kOzLbo + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((kOzLbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((kOzSbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;  // tcgen05 descriptor version; no swizzle, base offset 0
    return d;
}
// D F32, A and B BF16, both K-major, M = 128, N given
__device__ __forceinline__ uint32_t idesc(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | (uint32_t(kOzTG >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

// The threads that hold groups 32 s .. 32 s + 31 of a tile (group = tid mod 128, so the warps
// with warp mod 4 = s: a quarter of the block) meet at named barrier 1 + s; shared-memory writes
// before it are visible to those threads after it.
// (Constant barrier ids, so that the kernel reserves five hardware barriers, not all sixteen.)
template <int kBlockThreads>
__device__ __forceinline__ void group_set_sync(int warp) {
    constexpr int n = kBlockThreads / 4;
    switch (warp & 3) {  // warp-uniform
        case 0: asm volatile("bar.sync 1, %0;" ::"n"(n) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"n"(n) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"n"(n) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"n"(n) : "memory"); break;
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kOzSpinLimit) {
    for (long long spins = 0; spins <= limit; spins++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// value rounded to a multiple of 2^-8(s+1) (|x| <= 2^(14-8s)); the magic constant is
// 1.5 * 2^(23 - 8(s+1)), the sum lands in its binade and the low bits are rounded off
template <int S>
__device__ __forceinline__ float grid_round(float x) {
    constexpr float c = 1.5f * float(1 << 15) / float(1ull << (8 * S));
    return __fsub_rn(__fadd_rn(x, c), c);
}

// the six slices of x = (h + l) * inv_nu, each exact in bf16 (see the header comment). inv_nu is
// a power of two and |x| <= 1, so h * inv_nu and l * inv_nu are exact: the scaling rides in the
// FMAs that round to the first grid, form the first remainder and add the low word.
__device__ __forceinline__ void slice6(float h, float l, float inv_nu, float (&a)[kOzNS]) {
    constexpr float c0 = 1.5f * float(1 << 15);
    a[0] = __fsub_rn(__fmaf_rn(h, inv_nu, c0), c0);
    float r = __fmaf_rn(h, inv_nu, -a[0]);  // exact
    a[1] = grid_round<1>(r);
    r = __fsub_rn(r, a[1]);
    a[2] = grid_round<2>(r);
    r = __fmaf_rn(l, inv_nu, __fsub_rn(r, a[2]));  // rounding error below 2^-49
    a[3] = grid_round<3>(r);
    r = __fsub_rn(r, a[3]);
    a[4] = grid_round<4>(r);
    a[5] = grid_round<5>(__fsub_rn(r, a[4]));
}

// two values with at most 8 significant bits (exact in bf16) packed as bf16x2, lo in the low
// half: the upper 16 bits of each FP32 pattern (the lower 16 are zero)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}


// Packed pairs: sm_100 and later execute two FP32 operations per instruction (FADD2, FMUL2,
// FFMA2), each lane rounding exactly as the scalar instruction does, so a pair computation gives
// the same bits as two scalar ones. Written out where the two operands already sit side by side
// (a complex64 amplitude; the real and imaginary columns of an accumulator), they measured
// faster (the 5-target fold: 3.5 % less time per block); the double-float slicing, whose pairs
// would first have to be gathered from {re_hi, re_lo, im_hi, im_lo}, measured 2 % slower packed
// and stays scalar.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
// c - a with one rounding, as fma(a, -1, c)
__device__ __forceinline__ float2 rsub2(float2 c, float2 a) { return __ffma2_rn(a, make_float2(-1.f, -1.f), c); }
template <int S>
__device__ __forceinline__ float2 grid_round2(float2 x) {
    constexpr float c = 1.5f * float(1 << 15) / float(1ull << (8 * S));
    return __fadd2_rn(__fadd2_rn(x, dup2(c)), dup2(-c));
}
// (a + b) exactly as (s, t) when a is a multiple of ulp(b) or |a| >= |b|, both lanes
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& t) {
    s = __fadd2_rn(a, b);
    t = rsub2(b, rsub2(s, a));
}

__device__ __forceinline__ float pow2_ceil(float m) {
    // smallest power of two >= m for m > 0 (1 for m == 0), exponent kept in range
    if (!(m > 0.f)) return 1.f;
    uint32_t e = ((__float_as_uint(m) + 0x007FFFFFu) >> 23) & 0xFFu;
    e = e < 1u ? 1u : (e > 253u ? 253u : e);
    return __uint_as_float(e << 23);
}

// two adjacent amplitudes (32 bytes, 32-byte aligned) in one 256-bit access: used when the
// block's lowest target is qubit 0, where each thread's amplitudes come in such pairs. Loads of
// the state bypass L1 (.cg): every amplitude is read once, and for low targets a warp's access
// spans 32 lines whose other sectors other warps read later, which in L1 only evicts lines early.
__device__ __forceinline__ void ld_pair(const float4* p, float4& a, float4& b) {
    asm("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
__device__ __forceinline__ void st_pair(float4* p, const float4& a, const float4& b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w),
                 "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// L2 prefetch of one line (no register is written; the later load finds the line in L2)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// the 16 bytes of an IEEE complex128 amplitude, loaded as four floats, in the double-float layout
// {re_hi, re_lo, im_hi, im_lo} (the split of the layout-change pass)
__device__ __forceinline__ float4 df_of_ieee(const float4& w) {
    float4 r;
    split_double_int(__hiloint2double(__float_as_int(w.y), __float_as_int(w.x)), r.x, r.y);
    split_double_int(__hiloint2double(__float_as_int(w.w), __float_as_int(w.z)), r.z, r.w);
    return r;
}

template <bool kPairs, bool kIeeeIn>
__global__ void __launch_bounds__(kOzThreads, 2) k_dense_oz4(float4* __restrict__ psi, const unsigned char* __restrict__ dmat,
                                                             const __grid_constant__ OzParams P, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar, drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    // thread (g, h): group g of the tile (= TMEM lane), amplitudes 8h .. 8h + 7
    const int g = tid & (kOzTG - 1), h = tid >> 7;
    const float* mu = reinterpret_cast<const float*>(smem + kOffMu);
    float* nu_part = reinterpret_cast<float*>(smem + kOffNuPart);
    auto abuf = [&](uint64_t j) { return smem + kOffA + (j & 1) * kOzABuf; };

    // matrix slices (stacked, already in the K-major layout) and row scales, once per CTA
    for (int i = tid; i < int((kOzMat + kOzR * 4) / 16); i += kOzThreads)
        reinterpret_cast<uint4*>(smem + kOffMat)[i] = reinterpret_cast<const uint4*>(dmat)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)));
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kOzTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    uint64_t off[kOzAmpsPerThread];  // s(w) of this thread's amplitudes
#pragma unroll
    for (int i = 0; i < kOzAmpsPerThread; i++) off[i] = P.offs[h * kOzAmpsPerThread + i];

    auto group_x0 = [&](uint64_t j) {  // this thread's group in tile j (~0 past the end)
        const uint64_t gi = (blockIdx.x + j * gridDim.x) * kOzTG + uint64_t(g);
        return gi < P.n_groups ? expand(gi, P.ip) : ~0ull;
    };
    auto load = [&](uint64_t x0, float4 (&v)[kOzAmpsPerThread]) {
        if (kPairs) {
#pragma unroll
            for (int i = 0; i < kOzAmpsPerThread; i += 2) {
                if (x0 != ~0ull) {
                    ld_pair(psi + x0 + off[i], v[i], v[i + 1]);
                } else {
                    v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    v[i + 1] = v[i];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < kOzAmpsPerThread; i++)
                v[i] = x0 != ~0ull ? __ldcg(psi + x0 + off[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (kIeeeIn) {
#pragma unroll
            for (int i = 0; i < kOzAmpsPerThread; i++) v[i] = df_of_ieee(v[i]);
        }
    };
    // slices of this thread's amplitudes into abuf(j); returns the group scale nu
    auto slice = [&](uint64_t j, const float4 (&v)[kOzAmpsPerThread]) {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < kOzAmpsPerThread; i++) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].z)));
        nu_part[h * kOzTG + g] = m;
        group_set_sync<kOzThreads>(warp);  // the other thread of each group is in warp +- 4
        m = fmaxf(nu_part[g], nu_part[kOzTG + g]);
        const float nv = pow2_ceil(m);
        const float inv = __uint_as_float((254u - (__float_as_uint(nv) >> 23)) << 23);
        unsigned char* ab = abuf(j);
#pragma unroll
        for (int c = 0; c < 2; c++) {  // 4 amplitudes = K columns 16h + 8c .. +7: one 16-byte chunk per slice
            uint32_t pk[kOzNS][4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                float ar[kOzNS], ai[kOzNS];
                slice6(v[4 * c + i].x, v[4 * c + i].y, inv, ar);
                slice6(v[4 * c + i].z, v[4 * c + i].w, inv, ai);
#pragma unroll
                for (int s2 = 0; s2 < kOzNS; s2++) pk[s2][i] = pack_bf16(ar[s2], ai[s2]);
            }
            const uint32_t o = kmaj(uint32_t(g), uint32_t(16 * h + 8 * c));
#pragma unroll
            for (int s2 = 0; s2 < kOzNS; s2++)
                *reinterpret_cast<uint4*>(ab + s2 * kOzSlice + o) = make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        return nv;
    };
    auto issue = [&](uint64_t j) {  // MMAs of tile j into the accumulator set
        if (tid != 0) return;
        const uint32_t a0 = smem_u32(abuf(j)), m0 = smem_u32(smem + kOffMat);
        // state slice s times matrix slices t0 .. t0 + nt - 1 into diagonals s + t
        auto prod = [&](int s2, int t0, int nt, int ks, uint32_t acc) {
            mma_bf16(tmem + uint32_t((s2 + t0) * kOzR), sdesc(a0 + uint32_t(s2 * kOzSlice) + uint32_t(ks * 256)),
                     sdesc(m0 + uint32_t(t0 * kOzR / 8) * kOzSbo + uint32_t(ks * 256)), idesc(uint32_t(nt * kOzR)), acc);
        };
#pragma unroll
        for (int ks = 0; ks < kOzR / 16; ks++) {
            if (ks == 0) {
                // first writes: slice 1 starts diagonals 1..6, slice 0 starts diagonal 0
                prod(1, 0, kOzNS, 0, 0u);
                prod(0, 0, 1, 0, 0u);
                prod(0, 1, kOzNS - 1, 0, 1u);
            } else {
                prod(0, 0, kOzNS, ks, 1u);
                prod(1, 0, kOzNS, ks, 1u);
            }
#pragma unroll
            for (int s2 = 2; s2 < kOzNS; s2++) prod(s2, 0, kOzND - s2 < kOzNS ? kOzND - s2 : kOzNS, ks, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    };
    // accumulators -> double-float outputs, stored straight to the state
    auto epilogue = [&](uint64_t x0, float nv) {
        const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(16 * h);
#pragma unroll
        for (int c = 0; c < 4; c++) {  // 4 output reals = 2 amplitudes per step
            uint32_t r[kOzND][4];
#pragma unroll
            for (int d = 0; d < kOzND; d++)
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3])
                             : "r"(lane_base + uint32_t(d * kOzR + 4 * c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float2 hi[2], lo[2];  // per amplitude i: (real, imaginary) high and low words
#pragma unroll
            for (int i = 0; i < 2; i++) {
                // columns 2i, 2i + 1 (real and imaginary part of one amplitude) as packed pairs:
                // D_6 + D_5 + D_4 in FP32 (rounding far below 2^-48 of the output), then D_3..D_0
                // added exactly with Fast2Sum, the errors collected in l
                float2 D[kOzND];
#pragma unroll
                for (int d = 0; d < kOzND; d++)
                    D[d] = make_float2(__uint_as_float(r[d][2 * i]), __uint_as_float(r[d][2 * i + 1]));
                float2 sm = __fadd2_rn(__fadd2_rn(D[6], D[5]), D[4]);
                float2 l = make_float2(0.f, 0.f), t;
#pragma unroll
                for (int d = 3; d >= 0; d--) {
                    fast_two_sum2(D[d], sm, sm, t);
                    l = __fadd2_rn(l, t);
                }
                const float2 sc = __fmul2_rn(*reinterpret_cast<const float2*>(mu + 16 * h + 4 * c + 2 * i), dup2(nv));
                fast_two_sum2(__fmul2_rn(sm, sc), __fmul2_rn(l, sc), hi[i], lo[i]);
            }
            if (x0 != ~0ull) {
                const float4 a = make_float4(hi[0].x, lo[0].x, hi[0].y, lo[0].y);
                const float4 b = make_float4(hi[1].x, lo[1].x, hi[1].y, lo[1].y);
                if (kPairs) {
                    st_pair(psi + x0 + off[2 * c], a, b);
                } else {
                    psi[x0 + off[2 * c]] = a;
                    psi[x0 + off[2 * c + 1]] = b;
                }
            }
        }
    };

    // software pipeline: loads of tile j + 1 and the slices of tile j overlap the MMAs of tile
    // j - 1; then tile j - 1 is finished and the MMAs of tile j start
    float4 vcur[kOzAmpsPerThread], vnext[kOzAmpsPerThread];
    uint64_t x0_cur = 0, x0_prev = 0;
    float nv_prev = 1.f;
    bool failed = false;  // a commit wait ran out in this warp, or s_fail was seen (warp-uniform)
    if (my_tiles > 0) {
        x0_cur = group_x0(0);
        load(x0_cur, vcur);
    }
    for (uint64_t j = 0; j <= my_tiles && my_tiles > 0; j++) {
        uint64_t x0_next = 0;
        if (j + 1 < my_tiles) {
            x0_next = group_x0(j + 1);
            load(x0_next, vnext);
        }
        if (j + 2 < my_tiles) {  // tile j + 2 into L2, so that next tile's loads find it there
            const uint64_t xp = group_x0(j + 2);
            if (xp != ~0ull) {
#pragma unroll
                for (int i = 0; i < kOzAmpsPerThread; i += (kPairs ? 2 : 1)) prefetch_l2(psi + xp + off[i]);
            }
        }
        float nv_cur = 1.f;
        if (j < my_tiles) nv_cur = slice(j, vcur);  // abuf(j) was read by the MMAs of tile j - 2
        if (j >= 1) {
            if (!failed) {  // every thread waits itself; the vote reconverges the warp for tcgen05.ld
                const bool late = (P.force_late && j == 1) || !mbar_wait(smem_u32(&mbar), uint32_t((j - 1) & 1), P.wait_spins);
                if (__any_sync(0xffffffffu, late)) {
                    failed = true;
                    s_fail = 1;
                }
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!failed) epilogue(x0_prev, nv_prev);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // slices of tile j written; accumulators of tile j - 1 read
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (s_fail) failed = true;  // read by a converged warp: stays warp-uniform
        if (j < my_tiles && !failed) issue(j);
        x0_prev = x0_cur;
        nv_prev = nv_cur;
        x0_cur = x0_next;
#pragma unroll
        for (int i = 0; i < kOzAmpsPerThread; i++) vcur[i] = vnext[i];
    }
    __syncthreads();  // every thread's s_fail store is visible
    if (s_fail && tid == 0) {
        atomicExch(err, 1);
        // bounded: the MMAs this thread issued finish before TMEM is freed (a commit to a barrier
        // of its own tracks every one of them)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&drain_bar)));
        mbar_wait(smem_u32(&drain_bar), 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
}

// ---------------------------------------------------------------- 5-target blocks
// The same method for 32 x 32 complex blocks: A is the 64 x 64 real form, K = 64 (four K-steps),
// 128 groups of 32 amplitudes per tile. The outputs are split into two halves of 32 reals
// (amplitudes 0..15 and 16..31), each with its own stacked matrix slices (192 x 64), seven
// diagonals of 32 columns (TMEM columns 0..223 and 256..479) and its own commit barrier.
//
// Warp roles: sixteen worker warps (four threads per group, each owning four amplitudes of either
// half) load, slice and fold; one more warp issues the MMAs. The state slices are double-buffered
// so that a tile's MMAs run while the workers slice the next tile: slices 0..4 of a buffer sit in
// shared memory (80 KB each, 2 x 80 + 48 KB of matrix slices = 210 KB) and slice 5 is the MMA's A
// operand straight from TMEM (32 columns per buffer, in the two 32-column gaps after each half's
// accumulators: all 512 columns). Hand-offs are mbarriers, no block barrier inside the loop:
//   full[b]     the 16 worker warps have written the slices of the tile in buffer b
//   accfree[h]  the 16 worker warps have read half h's accumulators (fold done)
//   done[h]     commit of half h's MMAs (the tensor cores finished them)
// Per tile j a worker slices tile j into buffer j & 1 (free: the MMAs of tile j - 2 finished
// before its fold), issues the loads of tile j + 1, then waits for and folds half 0 and half 1 of
// tile j - 1. The issuer waits for full[j & 1], then for each half for accfree of tile j - 1 and issues
// that half's 28 MMAs: half 0 of tile j runs while the workers fold half 1 of tile j - 1 and slice
// tile j + 1. Every wait is bounded; a wait that runs out sets a shared flag that makes every other
// wait give up at once, the kernel records an error, and the issuer waits (bounded, with the full
// limit) for the MMAs it issued before TMEM is freed.
constexpr int kOz5Q = 5;
constexpr int kOz5D = 1 << kOz5Q;                               // 32 amplitudes per group
constexpr int kOz5R = 2 * kOz5D;                                // 64 reals per group
constexpr int kOz5Workers = 512;                                // 16 worker warps
constexpr int kOz5WorkerWarps = kOz5Workers / 32;
constexpr int kOz5Threads = kOz5Workers + 32;                   // + the MMA-issuing warp
// 17 warps: the sub-partition that holds five of them limits every thread to 96 registers
// (16384 / (5 x 32), in steps of 8); the workers issue the next tile's loads after slicing,
// so that at most one tile of amplitudes is live in registers and nothing spills.
constexpr int kOz5TPG = kOz5Workers / kOzTG;                    // 4 threads per group
constexpr int kOz5Amps = kOz5D / kOz5TPG;                       // 8 amplitudes per thread
constexpr uint32_t kOz5Sbo = (kOz5R / 8) * 128;                 // 1024
constexpr size_t kOz5Slice = size_t(kOzTG) * kOz5R * 2;         // 16 KB
constexpr int kOz5SmemSlices = kOzNS - 1;                       // slices 0..4 in shared memory
constexpr size_t kOz5ABuf = kOz5SmemSlices * kOz5Slice;         // 80 KB per buffer
constexpr int kOz5HalfRows = kOzNS * kOz5D;                     // 192 rows per half stack
constexpr size_t kOz5Half = size_t(kOz5HalfRows) * kOz5R * 2;   // 24 KB
constexpr size_t kOz5Mat = 2 * kOz5Half;                        // 48 KB
constexpr int kOz5TmemCols = 512;
constexpr uint32_t kOz5HalfCol = 256;
constexpr uint32_t kOz5A5Col = kOzND * kOz5D;                   // slice 5 of buffer b at b * 256 + 224
constexpr size_t kOff5A = 0;                                    // 2 buffers
constexpr size_t kOff5Mat = kOff5A + 2 * kOz5ABuf;
constexpr size_t kOff5Mu = kOff5Mat + kOz5Mat;
constexpr size_t kOff5NuPart = kOff5Mu + kOz5R * 4;
constexpr size_t kOz5Smem = kOff5NuPart + size_t(kOz5TPG) * kOzTG * 4;
static_assert(kOzND * kOz5D <= int(kOz5A5Col) && kOz5A5Col + kOz5R / 2 <= kOz5HalfCol,
              "a half's accumulators and one slice-5 buffer fit its 256 TMEM columns");
static_assert(kOz5Smem <= 227 * 1024, "shared memory of one CTA");

struct Oz5Params {
    IndexPlan ip;            // 5 targets (and controls) inserted
    uint64_t offs[kOz5D];    // s(w), targets ascending
    uint64_t n_groups;
    long long wait_spins;    // try_wait attempts of each pipeline wait before it gives up
    int force_late;          // test hook: a worker's first accumulator wait reports a timeout at once
};

__device__ __forceinline__ uint32_t kmaj5(uint32_t r, uint32_t k) {
    return (r >> 3) * kOz5Sbo + (k >> 3) * kOzLbo + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t sdesc5(uint32_t saddr) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((kOzLbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((kOz5Sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// A operand from TMEM (lane m = row m of the tile, column c = K elements 2c (low) and 2c + 1)
__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t tmem, uint32_t a_tmem, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
        "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

// bounded wait for the phase of the given parity; gives up at once when *abort is set
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, long long spins,
                                                   const volatile int* abort) {
    for (long long i = 0; i <= spins; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    return false;
}

template <bool kPairs, bool kIeeeIn>
__global__ void __launch_bounds__(kOz5Threads, 1) k_dense_oz5(float4* __restrict__ psi,
                                                               const unsigned char* __restrict__ dmat,
                                                               const __grid_constant__ Oz5Params P, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // full[0..1], accfree[0..1], done[0..1], drain
    __shared__ __align__(8) uint64_t bars[7];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* mu = reinterpret_cast<const float*>(smem + kOff5Mu);
    float* nu_part = reinterpret_cast<float*>(smem + kOff5NuPart);
    const uint32_t full0 = smem_u32(&bars[0]), accfree0 = smem_u32(&bars[2]), done0 = smem_u32(&bars[4]);
    const uint32_t drain = smem_u32(&bars[6]);
    volatile int* fail = &s_fail;

    for (int i = tid; i < int((kOz5Mat + kOz5R * 4) / 16); i += kOz5Threads)
        reinterpret_cast<uint4*>(smem + kOff5Mat)[i] = reinterpret_cast<const uint4*>(dmat)[i];
    if (tid == 0) {
        for (int i = 0; i < 4; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8u * i), "r"(kOz5WorkerWarps));
        for (int i = 4; i < 7; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * i));
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kOz5TmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long spins = P.wait_spins;

    if (warp >= kOz5WorkerWarps) {
        // ---------------------------------------------------------- MMA issuer (one thread)
        if (warp == kOz5WorkerWarps && lane == 0) {
            // descriptors of the slice buffers and of half 0's matrix stack; each MMA adds a
            // constant to them (the 14-bit address field, in 16-byte units, never carries: the
            // shared memory used is below 256 KB)
            const uint64_t abase0 = sdesc5(smem_u32(smem + kOff5A)), abase1 = sdesc5(smem_u32(smem + kOff5A + kOz5ABuf));
            const uint64_t mbase = sdesc5(smem_u32(smem + kOff5Mat));
            for (uint64_t j = 0; j < my_tiles; j++) {
                const uint32_t b = uint32_t(j & 1);
                if (!mbar_wait_or_abort(full0 + 8u * b, uint32_t((j >> 1) & 1), spins, fail)) {
                    *fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t ad = b ? abase1 : abase0;
                const uint32_t a5 = tmem + kOz5HalfCol * b + kOz5A5Col;
                bool stop = false;
#pragma unroll 1
                for (int hv = 0; hv < 2; hv++) {
                    if (j >= 1 && !mbar_wait_or_abort(accfree0 + 8u * hv, uint32_t((j - 1) & 1), spins, fail)) {
                        *fail = 1;
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dh = tmem + kOz5HalfCol * uint32_t(hv);
                    const uint64_t bdh = mbase + uint64_t(hv * (kOz5Half >> 4));
                    // state slice s times matrix slices t0 .. t0 + nt - 1 into diagonals s + t
                    auto prod = [&](int s2, int t0, int nt, int ks, uint32_t acc) {
                        const uint32_t d = dh + uint32_t((s2 + t0) * kOz5D);
                        const uint64_t bd = bdh + uint64_t(((t0 * kOz5D / 8) * kOz5Sbo + ks * 256) >> 4);
                        const uint32_t id = idesc(uint32_t(nt * kOz5D));
                        if (s2 < kOz5SmemSlices)
                            mma_bf16(d, ad + uint64_t((s2 * kOz5Slice + ks * 256) >> 4), bd, id, acc);
                        else
                            mma_bf16_tmem_a(d, a5 + uint32_t(ks * 8), bd, id, acc);
                    };
#pragma unroll
                    for (int ks = 0; ks < kOz5R / 16; ks++) {
                        if (ks == 0) {  // first writes: slice 1 starts diagonals 1..6, slice 0 diagonal 0
                            prod(1, 0, kOzNS, 0, 0u);
                            prod(0, 0, 1, 0, 0u);
                            prod(0, 1, kOzNS - 1, 0, 1u);
                        } else {
                            prod(0, 0, kOzNS, ks, 1u);
                            prod(1, 0, kOzNS, ks, 1u);
                        }
#pragma unroll
                        for (int s2 = 2; s2 < kOzNS; s2++) prod(s2, 0, kOzND - s2 < kOzNS ? kOzND - s2 : kOzNS, ks, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        done0 + 8u * uint32_t(hv)));
                }
                if (stop) break;
            }
            // every MMA issued above has finished before TMEM is freed (bounded, full limit)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain));
            if (!mbar_wait(drain, 0)) *fail = 1;
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- workers
        // thread (g, q): group g of the tile (= TMEM lane); amplitudes 4q..4q+3 (half 0) and
        // 16+4q..16+4q+3 (half 1), held as v[0..3] and v[4..7]
        const int g = tid & (kOzTG - 1), q = tid >> 7;
        // s(w) of this thread's amplitude i, w = (i / 4) * 16 + 4 q + i % 4: s is additive over
        // the disjoint bits of w, so s(w) = s(4q) (once per thread) + s((i / 4) * 16 + i % 4), a
        // parameter at a compile-time index (an operand of the add, no indexed constant load)
        const uint64_t qoff = P.offs[4 * q];
        auto off = [&](int i) { return qoff + P.offs[(i >> 2) * (kOz5D / 2) + (i & 3)]; };
        const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;

        // This thread's group in tile j: group index t 128 + g, whose bit string with the fixed
        // bits inserted is the OR of the insertions of t 128 (the same for the whole CTA) and of g
        // (per thread, once), as the two have disjoint bits. A tail (only when there are fewer
        // than 128 groups, all in one tile) reads the last group instead: valid memory, its
        // outputs are never stored.
        const uint64_t gx = expand(uint64_t(g) < P.n_groups ? uint64_t(g) : P.n_groups - 1, P.ip);
        auto group_x0 = [&](uint64_t j, bool& valid) {
            const uint64_t t = blockIdx.x + j * gridDim.x;
            valid = t * kOzTG + uint64_t(g) < P.n_groups;
            return expand(t * kOzTG, P.ip) | gx;
        };
        auto load = [&](uint64_t x0, float4 (&v)[kOz5Amps]) {
            if (kPairs) {
#pragma unroll
                for (int i = 0; i < kOz5Amps; i += 2) ld_pair(psi + x0 + off(i), v[i], v[i + 1]);
            } else {
#pragma unroll
                for (int i = 0; i < kOz5Amps; i++) v[i] = __ldcg(psi + x0 + off(i));
            }
            if (kIeeeIn) {
#pragma unroll
                for (int i = 0; i < kOz5Amps; i++) v[i] = df_of_ieee(v[i]);
            }
        };
        // slices 0..4 of this thread's amplitudes into shared-memory buffer b, slice 5 into TMEM
        // (this warp's 32 lanes, columns 4q.. and 16 + 4q.. of buffer b's slice-5 block). Every
        // worker takes part in the group-scale barrier; a warp that has given up (`store` false,
        // warp-uniform) writes nothing, so no buffer that an unfinished MMA may read is touched.
        auto slice = [&](uint32_t b, const float4 (&v)[kOz5Amps], bool store) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < kOz5Amps; i++) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].z)));
            nu_part[q * kOzTG + g] = m;
            group_set_sync<kOz5Workers>(warp);  // a group's four threads are in warps w, w + 4, w + 8, w + 12
            m = nu_part[g];
#pragma unroll
            for (int t = 1; t < kOz5TPG; t++) m = fmaxf(m, nu_part[t * kOzTG + g]);
            const float nv = pow2_ceil(m);
            if (!store) return nv;
            const float inv = __uint_as_float((254u - (__float_as_uint(nv) >> 23)) << 23);
            unsigned char* ab = smem + kOff5A + b * kOz5ABuf;
            const uint32_t ta = tmem + lane_off + kOz5HalfCol * b + kOz5A5Col + uint32_t(4 * q);
#pragma unroll
            for (int c = 0; c < 2; c++) {  // 4 amplitudes = K columns 32c + 8q .. +7: one 16-byte chunk per slice
                uint32_t pk[kOzNS][4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    float ar[kOzNS], ai[kOzNS];
                    slice6(v[4 * c + i].x, v[4 * c + i].y, inv, ar);
                    slice6(v[4 * c + i].z, v[4 * c + i].w, inv, ai);
#pragma unroll
                    for (int s2 = 0; s2 < kOzNS; s2++) pk[s2][i] = pack_bf16(ar[s2], ai[s2]);
                }
                const uint32_t o = kmaj5(uint32_t(g), uint32_t(32 * c + 8 * q));
#pragma unroll
                for (int s2 = 0; s2 < kOz5SmemSlices; s2++)
                    *reinterpret_cast<uint4*>(ab + s2 * kOz5Slice + o) = make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
                asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(ta + 16u * c),
                             "r"(pk[kOzNS - 1][0]), "r"(pk[kOzNS - 1][1]), "r"(pk[kOzNS - 1][2]), "r"(pk[kOzNS - 1][3]));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            return nv;
        };
        // half hv's accumulators -> double-float outputs of this thread's 4 amplitudes of that half
        auto epilogue = [&](int hv, uint64_t x0, bool valid, float nv) {
            const uint32_t lane_base = tmem + lane_off + kOz5HalfCol * uint32_t(hv) + uint32_t(8 * q);
#pragma unroll
            for (int c = 0; c < 2; c++) {  // 4 output reals = 2 amplitudes per step
                uint32_t r[kOzND][4];
#pragma unroll
                for (int d = 0; d < kOzND; d++)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3])
                                 : "r"(lane_base + uint32_t(d * kOz5D + 4 * c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float2 hi[2], lo[2];  // per amplitude i: (real, imaginary) high and low words
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    // columns 2i, 2i + 1 (real and imaginary part of one amplitude) as pairs.
                    // D_0 + D_1 + D_2 + D_3 from the largest: each partial sum is a multiple of
                    // the unit of the next diagonal (2^-8(d+2)), which is at least the ulp of
                    // that diagonal's value, so every Fast2Sum is exact; when a partial sum
                    // cancels to below its next diagonal's range it is exact and its error
                    // term is zero. The error terms and D_4 + D_5 + D_6 (FP32, rounding far below
                    // 2^-48 of the output) make up lo.
                    float2 D[kOzND];
#pragma unroll
                    for (int d = 0; d < kOzND; d++)
                        D[d] = make_float2(__uint_as_float(r[d][2 * i]), __uint_as_float(r[d][2 * i + 1]));
                    float2 sm, t1, t2, t3;
                    fast_two_sum2(D[0], D[1], sm, t1);
                    fast_two_sum2(sm, D[2], sm, t2);
                    fast_two_sum2(sm, D[3], sm, t3);
                    const float2 low = __fadd2_rn(__fadd2_rn(D[6], D[5]), D[4]);
                    const float2 l = __fadd2_rn(__fadd2_rn(__fadd2_rn(t3, t2), t1), low);
                    const float2 sc = __fmul2_rn(*reinterpret_cast<const float2*>(mu + kOz5D * hv + 8 * q + 4 * c + 2 * i), dup2(nv));
                    fast_two_sum2(__fmul2_rn(sm, sc), __fmul2_rn(l, sc), hi[i], lo[i]);
                }
                if (valid) {
                    const float4 a = make_float4(hi[0].x, lo[0].x, hi[0].y, lo[0].y);
                    const float4 bb = make_float4(hi[1].x, lo[1].x, hi[1].y, lo[1].y);
                    if (kPairs) {
                        st_pair(psi + x0 + off(4 * hv + 2 * c), a, bb);
                    } else {
                        psi[x0 + off(4 * hv + 2 * c)] = a;
                        psi[x0 + off(4 * hv + 2 * c + 1)] = bb;
                    }
                }
            }
        };

        // Per tile j: slice tile j, then load tile j + 1 into the same registers (their latency is
        // covered by the folds), fold both halves of tile j - 1.
        float4 v[kOz5Amps];
        uint64_t x0_cur = 0, x0_prev = 0;
        bool ok_cur = false, ok_prev = false;
        float nv_prev = 1.f;
        bool failed = false;  // warp-uniform: a wait ran out in this warp, or the shared flag was seen
        if (my_tiles > 0) {
            x0_cur = group_x0(0, ok_cur);
            load(x0_cur, v);
        }
        for (uint64_t j = 0; j <= my_tiles && my_tiles > 0; j++) {
            // tile j + 2 into L2 now, so that the loads of tile j + 1 (issued after this slice) and
            // of tile j + 2 (one tile later) find their lines there: the register loads alone have
            // less than a tile of latency to hide, and the DRAM queue under a full state pass is
            // longer than that (measured: 3.6 % less time per block at n = 30)
            if (j + 2 < my_tiles) {
                bool ok_pf;
                const uint64_t xp = group_x0(j + 2, ok_pf);
#pragma unroll
                for (int i = 0; i < kOz5Amps; i += (kPairs ? 2 : 1)) prefetch_l2(psi + xp + off(i));
            }
            float nv_cur = 1.f;
            if (j < my_tiles) {
                // buffer j & 1 was last read by the MMAs of tile j - 2, which finished before
                // this warp folded half 1 of that tile (the commit tracks every earlier MMA)
                if (__any_sync(0xffffffffu, *fail != 0)) failed = true;
                nv_cur = slice(uint32_t(j & 1), v, !failed);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0 && !failed) mbar_arrive(full0 + 8u * uint32_t(j & 1));
            }
            uint64_t x0_next = 0;
            bool ok_next = false;
            if (j + 1 < my_tiles) {
                x0_next = group_x0(j + 1, ok_next);
                load(x0_next, v);
            }
            if (j >= 1) {
#pragma unroll
                for (int hv = 0; hv < 2; hv++) {
                    if (!failed) {  // the vote keeps `failed` warp-uniform for tcgen05.ld
                        const bool late = (P.force_late && j == 1 && hv == 0) ||
                                          !mbar_wait_or_abort(done0 + 8u * uint32_t(hv), uint32_t((j - 1) & 1), spins, fail);
                        if (__any_sync(0xffffffffu, late)) {
                            failed = true;
                            *fail = 1;
                        }
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (!failed) epilogue(hv, x0_prev, ok_prev, nv_prev);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && !failed) mbar_arrive(accfree0 + 8u * uint32_t(hv));
                }
            }
            x0_prev = x0_cur;
            ok_prev = ok_cur;
            nv_prev = nv_cur;
            x0_cur = x0_next;
            ok_cur = ok_next;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the issuer's drain wait is over; every s_fail store is visible
    if (tid == 0 && s_fail) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOz5TmemCols));
}

// ---------------------------------------------------------------- complex64, 5- and 6-target blocks
// The same splitting for complex64 states (float2): the group vector (scaled by its power of two
// nu) and the matrix rows (scaled by mu_n) are cut into three 8-bit slices on the grids 2^-8,
// 2^-16, 2^-24, which hold every bit of an FP32 value down to 2^-24 of the group's scale; the six
// products with s + t <= 2 are summed exactly in FP32 by the tensor cores into three diagonals,
// and the epilogue adds them in FP32 from the smallest (one rounding to nearest, no bias) and
// scales by mu_n nu. Error about 2^-24 of max|v| max|K~| per output, the accuracy of the FP32
// CUDA-core kernels. Tile: 128 groups; each thread owns 16 amplitudes of a group; one slice
// buffer. The template serves Q = 5: R = 64 reals, 256 threads, two CTAs per SM (75 KB, 256 TMEM
// columns each) so that one CTA's MMAs overlap the other's slicing and folding. (Written for
// Q = 6 too — R = 128, 512 threads, one CTA per SM, the first slice's N = 384 products in two
// MMAs — but 6-target blocks run in the pipelined k_dense_bz6 below.)
constexpr int kBzNS = 3;   // slices per operand
constexpr int kBzND = 3;   // diagonals s + t <= 2
template <int Q>
struct Bz {
    static constexpr int D = 1 << Q;                                   // amplitudes per group
    static constexpr int R = 2 * D;                                    // reals per group
    static constexpr int Threads = Q == 5 ? 256 : 512;
    static constexpr int Tpg = Threads / kOzTG;                        // threads per group
    static constexpr int Amps = D / Tpg;                               // 16
    static constexpr uint32_t Sbo = (R / 8) * 128;
    static constexpr size_t Slice = size_t(kOzTG) * R * 2;
    static constexpr size_t ABuf = kBzNS * Slice;
    static constexpr size_t Mat = size_t(kBzNS) * R * R * 2;          // [B_0; B_1; B_2]
    static constexpr int TmemCols = Q == 5 ? 256 : 512;
    static constexpr size_t OffA = 0;
    static constexpr size_t OffMat = OffA + ABuf;
    static constexpr size_t OffMu = OffMat + Mat;
    static constexpr size_t OffNu = OffMu + R * 4;
    static constexpr size_t Smem = OffNu + size_t(Tpg) * kOzTG * 4;
    static constexpr int MinBlocks = Q == 5 ? 2 : 1;
    static_assert(kBzND * R <= TmemCols, "accumulators fit the TMEM allocation");
    static_assert(Amps == 16, "sixteen amplitudes per thread");
};
template <int Q>
struct BzParams {
    IndexPlan ip;
    uint64_t offs[1 << Q];
    uint64_t n_groups;
    long long wait_spins;    // try_wait attempts of each accumulator wait before it gives up
    int force_late;          // test hook: the first accumulator wait reports a timeout at once
};

// the three slices of x * inv (|x * inv| <= 1, real and imaginary part of one amplitude at once,
// as packed pairs): multiples of 2^-8, 2^-16, 2^-24
__device__ __forceinline__ void slice3x2(float2 x, float2 inv, float2 (&a)[kBzNS]) {
    x = __fmul2_rn(x, inv);
    a[0] = grid_round2<0>(x);
    const float2 r = rsub2(x, a[0]);
    a[1] = grid_round2<1>(r);
    a[2] = grid_round2<2>(rsub2(r, a[1]));
}

template <int Q>
__device__ __forceinline__ uint64_t bz_desc(uint32_t saddr) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((kOzLbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((Bz<Q>::Sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

template <int Q, bool kPairs>
__global__ void __launch_bounds__(Bz<Q>::Threads, Bz<Q>::MinBlocks) k_dense_bz(float2* __restrict__ psi,
                                                                               const unsigned char* __restrict__ dmat,
                                                                               const __grid_constant__ BzParams<Q> P,
                                                                               int* err) {
    using B = Bz<Q>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar, drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid & (kOzTG - 1), h = tid >> 7;  // thread (g, h): amplitudes 16h .. 16h + 15 of group g
    const float* mu = reinterpret_cast<const float*>(smem + B::OffMu);
    float* nu_part = reinterpret_cast<float*>(smem + B::OffNu);
    unsigned char* ab = smem + B::OffA;

    for (int i = tid; i < int((B::Mat + B::R * 4) / 16); i += B::Threads)
        reinterpret_cast<uint4*>(smem + B::OffMat)[i] = reinterpret_cast<const uint4*>(dmat)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)));
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(B::TmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    auto group_x0 = [&](uint64_t j) {
        const uint64_t gi = (blockIdx.x + j * gridDim.x) * kOzTG + uint64_t(g);
        return gi < P.n_groups ? expand(gi, P.ip) : ~0ull;
    };
    auto load = [&](uint64_t x0, float2 (&v)[B::Amps]) {
        if (kPairs) {  // lowest target qubit 0: adjacent 16-byte-aligned pairs, one 128-bit load each
#pragma unroll
            for (int i = 0; i < B::Amps; i += 2) {
                const float4 w = x0 != ~0ull ? *reinterpret_cast<const float4*>(psi + x0 + P.offs[B::Amps * h + i])
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                v[i] = make_float2(w.x, w.y);
                v[i + 1] = make_float2(w.z, w.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < B::Amps; i++)
                v[i] = x0 != ~0ull ? psi[x0 + P.offs[B::Amps * h + i]] : make_float2(0.f, 0.f);
        }
    };
    auto slice = [&](const float2 (&v)[B::Amps]) {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < B::Amps; i++) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
        nu_part[h * kOzTG + g] = m;
        group_set_sync<B::Threads>(warp);  // a group's threads are in the warps with the same warp mod 4
        m = nu_part[g];
#pragma unroll
        for (int t = 1; t < B::Tpg; t++) m = fmaxf(m, nu_part[t * kOzTG + g]);
        const float nv = pow2_ceil(m);
        const float inv = __uint_as_float((254u - (__float_as_uint(nv) >> 23)) << 23);
#pragma unroll
        for (int c = 0; c < B::Amps / 4; c++) {  // 4 amplitudes = K columns 32h + 8c .. +7
            uint32_t pk[kBzNS][4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                float2 a[kBzNS];  // (real, imaginary) slices
                slice3x2(v[4 * c + i], dup2(inv), a);
#pragma unroll
                for (int s2 = 0; s2 < kBzNS; s2++) pk[s2][i] = pack_bf16(a[s2].x, a[s2].y);
            }
            const uint32_t r = uint32_t(g), k = uint32_t(32 * h + 8 * c);
            const uint32_t o = (r >> 3) * B::Sbo + (k >> 3) * kOzLbo + (r & 7) * 16;
#pragma unroll
            for (int s2 = 0; s2 < kBzNS; s2++)
                *reinterpret_cast<uint4*>(ab + s2 * B::Slice + o) = make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        return nv;
    };
    auto issue = [&]() {  // state slice s times matrix slices 0 .. 2 - s into diagonals s .. 2
        if (tid != 0) return;
        const uint32_t a0 = smem_u32(ab), m0 = smem_u32(smem + B::OffMat);
        auto prod = [&](int s2, int t0, int nt, int ks, uint32_t acc) {
            mma_bf16(tmem + uint32_t((s2 + t0) * B::R), bz_desc<Q>(a0 + uint32_t(s2 * B::Slice) + uint32_t(ks * 256)),
                     bz_desc<Q>(m0 + uint32_t(t0 * B::R / 8) * B::Sbo + uint32_t(ks * 256)), idesc(uint32_t(nt * B::R)), acc);
        };
#pragma unroll
        for (int ks = 0; ks < B::R / 16; ks++) {
            const uint32_t first = ks == 0 ? 0u : 1u;
            if (3 * B::R <= 256) {
                prod(0, 0, 3, ks, first);
            } else {  // N = 3 R above 256: slices 0-1, then slice 2
                prod(0, 0, 2, ks, first);
                prod(0, 2, 1, ks, first);
            }
            prod(1, 0, 2, ks, 1u);
            prod(2, 0, 1, ks, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    };
    auto epilogue = [&](uint64_t x0, float nv) {
        const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(32 * h);
#pragma unroll
        for (int c = 0; c < B::Amps / 2; c++) {  // 4 output reals = 2 amplitudes per step
            uint32_t r[kBzND][4];
#pragma unroll
            for (int d = 0; d < kBzND; d++)
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3])
                             : "r"(lane_base + uint32_t(d * B::R + 4 * c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float2 o[2];  // two amplitudes: columns (2i, 2i + 1) = (real, imaginary), as pairs
#pragma unroll
            for (int i = 0; i < 2; i++) {
                auto col = [&](int d) { return make_float2(__uint_as_float(r[d][2 * i]), __uint_as_float(r[d][2 * i + 1])); };
                const float2 sm = __fadd2_rn(__fadd2_rn(col(2), col(1)), col(0));
                o[i] = __fmul2_rn(sm, __fmul2_rn(*reinterpret_cast<const float2*>(mu + 32 * h + 4 * c + 2 * i), dup2(nv)));
            }
            if (x0 != ~0ull) {
                if (kPairs) {
                    *reinterpret_cast<float4*>(psi + x0 + P.offs[B::Amps * h + 2 * c]) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                } else {
                    psi[x0 + P.offs[B::Amps * h + 2 * c]] = o[0];
                    psi[x0 + P.offs[B::Amps * h + 2 * c + 1]] = o[1];
                }
            }
        }
    };

    float2 vcur[B::Amps], vnext[B::Amps];
    uint64_t x0_cur = 0, x0_prev = 0;
    float nv_prev = 1.f;
    bool failed = false;  // a commit wait ran out in this warp, or s_fail was seen (warp-uniform)
    if (my_tiles > 0) {
        x0_cur = group_x0(0);
        load(x0_cur, vcur);
    }
    for (uint64_t j = 0; j <= my_tiles && my_tiles > 0; j++) {
        uint64_t x0_next = 0;
        if (j + 1 < my_tiles) {
            x0_next = group_x0(j + 1);
            load(x0_next, vnext);
        }
        // tile j + 2 into L2, so that next tile's loads find it there (Q = 6, one CTA per SM; with
        // two CTAs per SM (Q = 5) the loads already overlap the other CTA's work, and the prefetch
        // measured 1 % slower)
        if (Q == 6 && j + 2 < my_tiles) {
            const uint64_t xp = group_x0(j + 2);
            if (xp != ~0ull) {
#pragma unroll
                for (int i = 0; i < B::Amps; i += (kPairs ? 2 : 1)) prefetch_l2(psi + xp + P.offs[B::Amps * h + i]);
            }
        }
        if (j >= 1) {
            if (!failed) {  // every thread waits itself; the vote reconverges the warp for tcgen05.ld
                const bool late = (P.force_late && j == 1) || !mbar_wait(smem_u32(&mbar), uint32_t((j - 1) & 1), P.wait_spins);
                if (__any_sync(0xffffffffu, late)) {
                    failed = true;
                    s_fail = 1;
                }
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!failed) epilogue(x0_prev, nv_prev);
        }
        float nv_cur = 1.f;
        if (j < my_tiles) nv_cur = slice(vcur);  // the buffer was read by the MMAs of tile j - 1 (done)
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // slices of tile j written; accumulators of tile j - 1 read
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (s_fail) failed = true;  // read by a converged warp: stays warp-uniform
        if (j < my_tiles && !failed) issue();
        x0_prev = x0_cur;
        nv_prev = nv_cur;
        x0_cur = x0_next;
#pragma unroll
        for (int i = 0; i < B::Amps; i++) vcur[i] = vnext[i];
    }
    __syncthreads();  // every thread's s_fail store is visible
    if (s_fail && tid == 0) {
        atomicExch(err, 1);
        // bounded: the MMAs this thread issued finish before TMEM is freed (a commit to a barrier
        // of its own tracks every one of them)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&drain_bar)));
        mbar_wait(smem_u32(&drain_bar), 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(B::TmemCols));
}

// ---------------------------------------------------------------- complex64, 6 targets, pipelined
// 64 x 64 complex blocks (R = 128 reals, K = 128: eight K-steps) with the 5-target kernel's
// pipeline. The outputs are split into two halves of 64 reals (amplitudes 0..31 and 32..63), each
// with its stacked matrix slices [B_0h; B_1h; B_2h] (192 x 128 bf16), three diagonals in its own
// 192 TMEM columns and its own commit barrier; the MMAs of a half are, per K-step, slice 0 times
// all three matrix slices (N = 192, diagonals 0..2), slice 1 times two (N = 128, diagonals 1, 2)
// and slice 2 times one (N = 64, diagonal 2). Sixteen worker warps (four threads per group, each
// owning eight amplitudes of either half) load, slice and sum; one more warp issues the MMAs. The
// state slices are double-buffered: buffer 0 holds its three slices in shared memory, buffer 1
// its slice 0 in shared memory and slices 1 and 2 as the MMA's A operand in TMEM, in the 64-column
// gaps after each half's accumulators (2 x (192 + 64) = all 512 columns; shared memory
// 3 x 32 + 32 + 96 KB of matrix slices; the row scales are read from global memory). Hand-offs,
// bounded waits and the recovery on a timeout are those of the 5-target kernel.
constexpr int kBz6D = 64;                                      // amplitudes per group
constexpr int kBz6R = 2 * kBz6D;                               // 128 reals
constexpr int kBz6Workers = 512;
constexpr int kBz6WorkerWarps = kBz6Workers / 32;
constexpr int kBz6Threads = kBz6Workers + 32;
constexpr int kBz6TPG = kBz6Workers / kOzTG;                   // 4 threads per group
constexpr int kBz6Amps = kBz6D / kBz6TPG;                      // 16 amplitudes per thread
constexpr uint32_t kBz6Sbo = (kBz6R / 8) * 128;                // 2048
constexpr size_t kBz6Slice = size_t(kOzTG) * kBz6R * 2;        // 32 KB
constexpr int kBz6HalfRows = kBzNS * (kBz6R / 2);              // 192 rows per half stack
constexpr size_t kBz6Half = size_t(kBz6HalfRows) * kBz6R * 2;  // 48 KB
constexpr size_t kBz6Mat = 2 * kBz6Half;                       // 96 KB
constexpr int kBz6TmemCols = 512;
constexpr uint32_t kBz6HalfCol = 256;
constexpr uint32_t kBz6ACol = kBzND * (kBz6R / 2);             // 192: the A slice of buffer 1 in half h's gap
constexpr size_t kOff6A0 = 0;                                  // buffer 0: slices 0..2
constexpr size_t kOff6A1 = kBzNS * kBz6Slice;                  // buffer 1: slice 0
constexpr size_t kOff6Mat = kOff6A1 + kBz6Slice;
constexpr size_t kOff6NuPart = kOff6Mat + kBz6Mat;
constexpr size_t kBz6Smem = kOff6NuPart + size_t(kBz6TPG) * kOzTG * 4;
static_assert(kBz6ACol + kBz6R / 2 <= kBz6HalfCol, "a half's accumulators and one A slice fit its 256 TMEM columns");
// with the 1 KB of static shared memory (the barriers, padded to the dynamic array's alignment)
static_assert(kBz6Smem + 1024 <= 227 * 1024, "shared memory of one CTA");

struct Bz6Params {
    IndexPlan ip;
    uint64_t offs[kBz6D];    // s(w), targets ascending
    uint64_t n_groups;
    long long wait_spins;    // try_wait attempts of each pipeline wait before it gives up
    int force_late;          // test hook: a worker's first accumulator wait reports a timeout at once
};

__device__ __forceinline__ uint64_t sdesc6(uint32_t saddr) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((kOzLbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((kBz6Sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

template <bool kPairs>
__global__ void __launch_bounds__(kBz6Threads, 1) k_dense_bz6(float2* __restrict__ psi,
                                                              const unsigned char* __restrict__ dmat,
                                                              const __grid_constant__ Bz6Params P, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[7];  // full[0..1], accfree[0..1], done[0..1], drain
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the row scales stay in global memory (512 bytes, read through L1): shared memory is full
    const float* __restrict__ mu = reinterpret_cast<const float*>(dmat + kBz6Mat);
    float* nu_part = reinterpret_cast<float*>(smem + kOff6NuPart);
    const uint32_t full0 = smem_u32(&bars[0]), accfree0 = smem_u32(&bars[2]), done0 = smem_u32(&bars[4]);
    const uint32_t drain = smem_u32(&bars[6]);
    volatile int* fail = &s_fail;

    for (int i = tid; i < int(kBz6Mat / 16); i += kBz6Threads)
        reinterpret_cast<uint4*>(smem + kOff6Mat)[i] = reinterpret_cast<const uint4*>(dmat)[i];
    if (tid == 0) {
        for (int i = 0; i < 4; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8u * i), "r"(kBz6WorkerWarps));
        for (int i = 4; i < 7; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * i));
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kBz6TmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long spins = P.wait_spins;

    if (warp >= kBz6WorkerWarps) {
        // ---------------------------------------------------------- MMA issuer (one thread)
        if (warp == kBz6WorkerWarps && lane == 0) {
            const uint64_t a0 = sdesc6(smem_u32(smem + kOff6A0)), a1 = sdesc6(smem_u32(smem + kOff6A1));
            const uint64_t mbase = sdesc6(smem_u32(smem + kOff6Mat));
            for (uint64_t j = 0; j < my_tiles; j++) {
                const uint32_t b = uint32_t(j & 1);
                if (!mbar_wait_or_abort(full0 + 8u * b, uint32_t((j >> 1) & 1), spins, fail)) {
                    *fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool stop = false;
#pragma unroll 1
                for (int hv = 0; hv < 2; hv++) {
                    if (j >= 1 && !mbar_wait_or_abort(accfree0 + 8u * hv, uint32_t((j - 1) & 1), spins, fail)) {
                        *fail = 1;
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dh = tmem + kBz6HalfCol * uint32_t(hv);
                    const uint64_t bdh = mbase + uint64_t(hv * (kBz6Half >> 4));
                    // state slice s2 of buffer b times matrix slices 0 .. nt - 1 into diagonals s2..
                    auto prod = [&](int s2, int nt, int ks, uint32_t acc) {
                        const uint32_t d = dh + uint32_t(s2 * (kBz6R / 2));
                        const uint64_t bd = bdh + uint64_t((ks * 256) >> 4);
                        const uint32_t id = idesc(uint32_t(nt * (kBz6R / 2)));
                        if (b == 0)
                            mma_bf16(d, a0 + uint64_t((s2 * kBz6Slice + ks * 256) >> 4), bd, id, acc);
                        else if (s2 == 0)
                            mma_bf16(d, a1 + uint64_t((ks * 256) >> 4), bd, id, acc);
                        else
                            mma_bf16_tmem_a(d, tmem + kBz6HalfCol * uint32_t(s2 - 1) + kBz6ACol + uint32_t(ks * 8), bd,
                                            id, acc);
                    };
#pragma unroll
                    for (int ks = 0; ks < kBz6R / 16; ks++) {
                        prod(0, 3, ks, ks > 0 ? 1u : 0u);  // starts diagonals 0..2 at the first K-step
                        prod(1, 2, ks, 1u);
                        prod(2, 1, ks, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        done0 + 8u * uint32_t(hv)));
                }
                if (stop) break;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain));
            if (!mbar_wait(drain, 0)) *fail = 1;
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- workers
        // thread (g, q): group g of the tile (= TMEM lane); amplitudes 8q..8q+7 (half 0) and
        // 32+8q..32+8q+7 (half 1), held as v[0..7] and v[8..15]
        const int g = tid & (kOzTG - 1), q = tid >> 7;
        // s(w) of amplitude i, w = (i / 8) * 32 + 8 q + i % 8: s(8q) once per thread plus a
        // parameter at a compile-time index
        const uint64_t qoff = P.offs[8 * q];
        auto off = [&](int i) { return qoff + P.offs[(i >> 3) * 32 + (i & 7)]; };
        const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;
        const uint64_t gx = expand(uint64_t(g) < P.n_groups ? uint64_t(g) : P.n_groups - 1, P.ip);
        auto group_x0 = [&](uint64_t j, bool& valid) {
            const uint64_t t = blockIdx.x + j * gridDim.x;
            valid = t * kOzTG + uint64_t(g) < P.n_groups;
            return expand(t * kOzTG, P.ip) | gx;
        };
        auto load = [&](uint64_t x0, float2 (&v)[kBz6Amps]) {
            if (kPairs) {  // lowest target qubit 0: amplitudes 2k, 2k + 1 adjacent, one 128-bit load
#pragma unroll
                for (int i = 0; i < kBz6Amps; i += 2) {
                    const float4 w4 = __ldcg(reinterpret_cast<const float4*>(psi + x0 + off(i)));
                    v[i] = make_float2(w4.x, w4.y);
                    v[i + 1] = make_float2(w4.z, w4.w);
                }
            } else {
#pragma unroll
                for (int i = 0; i < kBz6Amps; i++) v[i] = __ldcg(psi + x0 + off(i));
            }
        };
        // slices of this thread's amplitudes into buffer b (a warp that has given up, `store`
        // false and warp-uniform, writes nothing)
        auto slice = [&](uint32_t b, const float2 (&v)[kBz6Amps], bool store) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < kBz6Amps; i++) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
            nu_part[q * kOzTG + g] = m;
            group_set_sync<kBz6Workers>(warp);
            m = nu_part[g];
#pragma unroll
            for (int t = 1; t < kBz6TPG; t++) m = fmaxf(m, nu_part[t * kOzTG + g]);
            const float nv = pow2_ceil(m);
            if (!store) return nv;
            const float inv = __uint_as_float((254u - (__float_as_uint(nv) >> 23)) << 23);
#pragma unroll
            for (int c = 0; c < 4; c++) {  // 4 amplitudes = K columns kb .. kb + 7
                uint32_t pk[kBzNS][4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    float2 a[kBzNS];
                    slice3x2(v[4 * c + i], dup2(inv), a);
#pragma unroll
                    for (int s2 = 0; s2 < kBzNS; s2++) pk[s2][i] = pack_bf16(a[s2].x, a[s2].y);
                }
                const uint32_t kb = uint32_t((c >> 1) * (kBz6R / 2) + 16 * q + 8 * (c & 1));
                const uint32_t r = uint32_t(g);
                const uint32_t o = (r >> 3) * kBz6Sbo + (kb >> 3) * kOzLbo + (r & 7) * 16;
                if (b == 0) {
#pragma unroll
                    for (int s2 = 0; s2 < kBzNS; s2++)
                        *reinterpret_cast<uint4*>(smem + kOff6A0 + s2 * kBz6Slice + o) =
                            make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
                } else {
                    *reinterpret_cast<uint4*>(smem + kOff6A1 + o) = make_uint4(pk[0][0], pk[0][1], pk[0][2], pk[0][3]);
#pragma unroll
                    for (int s2 = 1; s2 < kBzNS; s2++)
                        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(
                                         tmem + lane_off + kBz6HalfCol * uint32_t(s2 - 1) + kBz6ACol + kb / 2),
                                     "r"(pk[s2][0]), "r"(pk[s2][1]), "r"(pk[s2][2]), "r"(pk[s2][3]));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (b != 0) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            return nv;
        };
        // half hv's accumulators -> outputs of this thread's 8 amplitudes of that half
        auto epilogue = [&](int hv, uint64_t x0, bool valid, float nv) {
            const uint32_t lane_base = tmem + lane_off + kBz6HalfCol * uint32_t(hv) + uint32_t(16 * q);
#pragma unroll
            for (int c = 0; c < 4; c++) {  // 4 output reals = 2 amplitudes per step
                uint32_t r[kBzND][4];
#pragma unroll
                for (int d = 0; d < kBzND; d++)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3])
                                 : "r"(lane_base + uint32_t(d * (kBz6R / 2) + 4 * c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float2 o[2];
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    auto col = [&](int d) { return make_float2(__uint_as_float(r[d][2 * i]), __uint_as_float(r[d][2 * i + 1])); };
                    const float2 sm = __fadd2_rn(__fadd2_rn(col(2), col(1)), col(0));
                    o[i] = __fmul2_rn(sm, __fmul2_rn(__ldg(reinterpret_cast<const float2*>(mu + (kBz6R / 2) * hv + 16 * q + 4 * c + 2 * i)),
                                                     dup2(nv)));
                }
                if (valid) {
                    const int i0 = 8 * hv + 2 * c;  // this thread's amplitude index of the pair
                    if (kPairs) {
                        __stcg(reinterpret_cast<float4*>(psi + x0 + off(i0)), make_float4(o[0].x, o[0].y, o[1].x, o[1].y));
                    } else {
                        psi[x0 + off(i0)] = o[0];
                        psi[x0 + off(i0 + 1)] = o[1];
                    }
                }
            }
        };

        float2 v[kBz6Amps];
        uint64_t x0_cur = 0, x0_prev = 0;
        bool ok_cur = false, ok_prev = false;
        float nv_prev = 1.f;
        bool failed = false;
        if (my_tiles > 0) {
            x0_cur = group_x0(0, ok_cur);
            load(x0_cur, v);
        }
        for (uint64_t j = 0; j <= my_tiles && my_tiles > 0; j++) {
            if (j + 2 < my_tiles) {  // tile j + 2 into L2 (see the 5-target kernel)
                bool ok_pf;
                const uint64_t xp = group_x0(j + 2, ok_pf);
#pragma unroll
                for (int i = 0; i < kBz6Amps; i += (kPairs ? 2 : 1)) prefetch_l2(psi + xp + off(i));
            }
            float nv_cur = 1.f;
            if (j < my_tiles) {
                // buffer j & 1 was last read by the MMAs of tile j - 2, which finished before
                // this warp summed half 1 of that tile
                if (__any_sync(0xffffffffu, *fail != 0)) failed = true;
                nv_cur = slice(uint32_t(j & 1), v, !failed);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0 && !failed) mbar_arrive(full0 + 8u * uint32_t(j & 1));
            }
            uint64_t x0_next = 0;
            bool ok_next = false;
            if (j + 1 < my_tiles) {
                x0_next = group_x0(j + 1, ok_next);
                load(x0_next, v);
            }
            if (j >= 1) {
#pragma unroll
                for (int hv = 0; hv < 2; hv++) {
                    if (!failed) {
                        const bool late = (P.force_late && j == 1 && hv == 0) ||
                                          !mbar_wait_or_abort(done0 + 8u * uint32_t(hv), uint32_t((j - 1) & 1), spins, fail);
                        if (__any_sync(0xffffffffu, late)) {
                            failed = true;
                            *fail = 1;
                        }
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (!failed) epilogue(hv, x0_prev, ok_prev, nv_prev);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && !failed) mbar_arrive(accfree0 + 8u * uint32_t(hv));
                }
            }
            x0_prev = x0_cur;
            ok_prev = ok_cur;
            nv_prev = nv_cur;
            x0_cur = x0_next;
            ok_cur = ok_next;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_fail) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBz6TmemCols));
}

// Per device (the current one at launch): SM count, the device-side error flag, and whether the
// shared-memory limits of each kernel family have been raised there (function attributes are per
// device context).
constexpr int kOzMaxDevices = 64;
struct OzDevice {
    int sms = 0;
    int* err = nullptr;
    bool attr4 = false, attr5 = false, attr_bz5 = false, attr_bz6 = false;
};
OzDevice g_oz_dev[kOzMaxDevices];
std::mutex g_oz_mu;
std::atomic<long long> g_oz_wait_spins{kOzSpinLimit};
std::atomic<int> g_oz_force_late{0};

OzDevice& oz_init() {
    int dev = 0;
    QS_TRY_CUDA(cudaGetDevice(&dev));
    QS_REQUIRE(dev >= 0 && dev < kOzMaxDevices, "device index out of range");
    std::lock_guard<std::mutex> lk(g_oz_mu);
    OzDevice& d = g_oz_dev[dev];
    if (!d.sms) {
        int sms = 0;
        QS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (!d.err) {
            QS_TRY_CUDA(dev_malloc(&d.err, sizeof(int)));
            QS_TRY_CUDA(cudaMemset(d.err, 0, sizeof(int)));
        }
        d.sms = sms;
    }
    return d;
}

// the real form of K~ (16 x 16 complex): row n = 2z + c_out, column k = 2w + c_in
double real_form(const std::vector<cplx>& K, int n, int k) {
    const cplx e = K[size_t(n >> 1) * kOzD + size_t(k >> 1)];
    if ((n & 1) == 0) return (k & 1) == 0 ? e.real() : -e.imag();
    return (k & 1) == 0 ? e.imag() : e.real();
}

uint16_t bf16_bits_exact(double v) {
    const float f = float(v);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return uint16_t(u >> 16);  // v has at most 8 significant bits: the low half is zero
}

}  // namespace

size_t oz4_matrix_bytes() { return kOzMat + kOzR * 4; }

// Stacked bf16 slices of the scaled real form, K-major core-matrix layout, then the row scales.
void prepare_oz4_matrix(const std::vector<cplx>& K, unsigned char* host_out) {
    QS_REQUIRE(K.size() == size_t(kOzD) * kOzD, "tensor-core double-float path takes 4-target matrices");
    std::memset(host_out, 0, oz4_matrix_bytes());
    float* mu = reinterpret_cast<float*>(host_out + kOzMat);
    double magic[kOzNS];
    for (int t = 0; t < kOzNS; t++) magic[t] = 1.5 * std::ldexp(1.0, 52 - 8 * (t + 1));
    for (int n = 0; n < kOzR; n++) {
        double m = 0.0;
        for (int k = 0; k < kOzR; k++) m = std::max(m, std::fabs(real_form(K, n, k)));
        double scale = 1.0;
        if (m > 0.0) {
            int e = 0;
            const double f = std::frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
            scale = f == 0.5 ? m : std::ldexp(1.0, e);
        }
        mu[n] = float(scale);
        for (int k = 0; k < kOzR; k++) {
            double r = real_form(K, n, k) / scale;  // exact (power of two), |r| <= 1
            for (int t = 0; t < kOzNS; t++) {
                // r rounded to a multiple of u = 2^-8(t+1): (r + c) - c with c = 1.5 * 2^52 * u
                // (|r| is far below 2^51 u, so the sum stays in c's binade; exact in FP64)
                const double a = (r + magic[t]) - magic[t];
                r -= a;
                const int row = t * kOzR + n;
                const size_t off = size_t(row >> 3) * kOzSbo + size_t(k >> 3) * kOzLbo + size_t(row & 7) * 16 +
                                   size_t(k & 7) * 2;
                const uint16_t bits = bf16_bits_exact(a);
                std::memcpy(host_out + off, &bits, 2);
            }
        }
    }
}

// y = K v on every group of the 4 targets (ascending) of a double-float state.
void launch_dense_oz4(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                      const std::vector<int>& cvals, const void* dmat, cudaStream_t st, bool ieee_in) {
    QS_REQUIRE(targets.size() == size_t(kOzQ), "tensor-core double-float path takes 4 targets");
    QS_REQUIRE(std::is_sorted(targets.begin(), targets.end()), "targets must be ascending");
    OzDevice& D = oz_init();
    if (!D.attr4) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz4<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOzSmem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz4<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOzSmem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz4<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOzSmem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz4<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOzSmem)));
        D.attr4 = true;
    }
    std::vector<int> fixed(targets);
    uint64_t setmask = 0;
    for (size_t j = 0; j < controls.size(); j++) {
        fixed.push_back(controls[j]);
        if (cvals[j]) setmask |= 1ull << controls[j];
    }
    OzParams P;
    P.ip = make_index_plan(n, fixed, setmask);
    for (int w = 0; w < kOzD; w++) {
        uint64_t o = 0;
        for (int j = 0; j < kOzQ; j++)
            if ((w >> j) & 1) o |= 1ull << targets[j];
        P.offs[w] = o;
    }
    P.wait_spins = g_oz_wait_spins.load();
    P.force_late = g_oz_force_late.load();
    P.n_groups = P.ip.n_iter;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, 2 * uint64_t(D.sms))));
    // lowest target qubit 0 (and a 32-byte-aligned state): each thread's amplitudes come in
    // adjacent 32-byte-aligned pairs
    QS_REQUIRE(!ieee_in || controls.empty(), "an IEEE-input block rewrites every amplitude (no controls)");
    const bool pairs = targets[0] == 0 && (reinterpret_cast<uintptr_t>(psi) & 31) == 0;
    auto kern = pairs ? (ieee_in ? k_dense_oz4<true, true> : k_dense_oz4<true, false>)
                      : (ieee_in ? k_dense_oz4<false, true> : k_dense_oz4<false, false>);
    kern<<<grid, kOzThreads, kOzSmem, st>>>(reinterpret_cast<float4*>(psi), static_cast<const unsigned char*>(dmat), P,
                                            D.err);
    QS_TRY_CUDA(cudaGetLastError());
}

size_t oz5_matrix_bytes() { return kOz5Mat + kOz5R * 4; }

// Two stacked half matrices (output reals 0..31 and 32..63), each [B_0; ...; B_5] of the scaled
// real form's rows in that half (192 x 64 bf16, K-major core-matrix layout), then the 64 row
// scales.
void prepare_oz5_matrix(const std::vector<cplx>& K, unsigned char* host_out) {
    QS_REQUIRE(K.size() == size_t(kOz5D) * kOz5D, "5-target tensor-core path takes 32 x 32 matrices");
    std::memset(host_out, 0, oz5_matrix_bytes());
    float* mu = reinterpret_cast<float*>(host_out + kOz5Mat);
    double magic[kOzNS];
    for (int t = 0; t < kOzNS; t++) magic[t] = 1.5 * std::ldexp(1.0, 52 - 8 * (t + 1));
    auto rf = [&](int n, int k) {
        const cplx e = K[size_t(n >> 1) * kOz5D + size_t(k >> 1)];
        if ((n & 1) == 0) return (k & 1) == 0 ? e.real() : -e.imag();
        return (k & 1) == 0 ? e.imag() : e.real();
    };
    for (int n = 0; n < kOz5R; n++) {
        double m = 0.0;
        for (int k = 0; k < kOz5R; k++) m = std::max(m, std::fabs(rf(n, k)));
        double scale = 1.0;
        if (m > 0.0) {
            int e = 0;
            const double f = std::frexp(m, &e);
            scale = f == 0.5 ? m : std::ldexp(1.0, e);
        }
        mu[n] = float(scale);
        const int hv = n / kOz5D, nl = n % kOz5D;
        for (int k = 0; k < kOz5R; k++) {
            double r = rf(n, k) / scale;
            for (int t = 0; t < kOzNS; t++) {
                const double a = (r + magic[t]) - magic[t];
                r -= a;
                const int row = t * kOz5D + nl;
                const size_t off = size_t(hv) * kOz5Half + size_t(row >> 3) * kOz5Sbo + size_t(k >> 3) * kOzLbo +
                                   size_t(row & 7) * 16 + size_t(k & 7) * 2;
                const uint16_t bits = bf16_bits_exact(a);
                std::memcpy(host_out + off, &bits, 2);
            }
        }
    }
}

void launch_dense_oz5(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                      const std::vector<int>& cvals, const void* dmat, cudaStream_t st, bool ieee_in) {
    QS_REQUIRE(targets.size() == size_t(kOz5Q), "5-target tensor-core path takes 5 targets");
    QS_REQUIRE(std::is_sorted(targets.begin(), targets.end()), "targets must be ascending");
    OzDevice& D = oz_init();
    if (!D.attr5) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz5<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOz5Smem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz5<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOz5Smem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz5<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOz5Smem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz5<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOz5Smem)));
        D.attr5 = true;
    }
    std::vector<int> fixed(targets);
    uint64_t setmask = 0;
    for (size_t i = 0; i < controls.size(); i++) {
        fixed.push_back(controls[i]);
        if (cvals[i]) setmask |= 1ull << controls[i];
    }
    Oz5Params P;
    P.ip = make_index_plan(n, fixed, setmask);
    P.n_groups = P.ip.n_iter;
    P.wait_spins = g_oz_wait_spins.load();
    P.force_late = g_oz_force_late.load();
    for (int w = 0; w < kOz5D; w++) {
        uint64_t o = 0;
        for (int j = 0; j < kOz5Q; j++)
            if ((w >> j) & 1) o |= 1ull << targets[j];
        P.offs[w] = o;
    }
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(D.sms))));
    QS_REQUIRE(!ieee_in || controls.empty(), "an IEEE-input block rewrites every amplitude (no controls)");
    const bool pairs = targets[0] == 0 && (reinterpret_cast<uintptr_t>(psi) & 31) == 0;
    auto kern = pairs ? (ieee_in ? k_dense_oz5<true, true> : k_dense_oz5<true, false>)
                      : (ieee_in ? k_dense_oz5<false, true> : k_dense_oz5<false, false>);
    kern<<<grid, kOz5Threads, kOz5Smem, st>>>(reinterpret_cast<float4*>(psi), static_cast<const unsigned char*>(dmat), P,
                                              D.err);
    QS_TRY_CUDA(cudaGetLastError());
}

size_t bz_matrix_bytes(int q) { return q == 5 ? Bz<5>::Mat + Bz<5>::R * 4 : kBz6Mat + kBz6R * 4; }

// [B_0; B_1; B_2] (3 R x R bf16, K-major core-matrix layout) of the row-scaled real form of a
// 2^q x 2^q matrix (for q = 6 stacked per output half: [B_00; B_10; B_20; B_01; B_11; B_21]), then
// the R row scales.
void prepare_bz_matrix(int q, const std::vector<cplx>& K, unsigned char* host_out) {
    QS_REQUIRE(q == 5 || q == 6, "complex64 tensor-core path takes 5 or 6 targets");
    const int D = 1 << q, R = 2 * D;
    const size_t sbo = size_t(R / 8) * 128;
    QS_REQUIRE(K.size() == size_t(D) * D, "matrix size does not match the target count");
    std::memset(host_out, 0, bz_matrix_bytes(q));
    float* mu = reinterpret_cast<float*>(host_out + size_t(kBzNS) * R * R * 2);
    double magic[kBzNS];
    for (int t = 0; t < kBzNS; t++) magic[t] = 1.5 * std::ldexp(1.0, 52 - 8 * (t + 1));
    auto rf = [&](int n, int k) {
        const cplx e = K[size_t(n >> 1) * D + size_t(k >> 1)];
        if ((n & 1) == 0) return (k & 1) == 0 ? e.real() : -e.imag();
        return (k & 1) == 0 ? e.imag() : e.real();
    };
    for (int n = 0; n < R; n++) {
        double m = 0.0;
        for (int k = 0; k < R; k++) m = std::max(m, std::fabs(rf(n, k)));
        double scale = 1.0;
        if (m > 0.0) {
            int e = 0;
            const double f = std::frexp(m, &e);
            scale = f == 0.5 ? m : std::ldexp(1.0, e);
        }
        mu[n] = float(scale);
        for (int k = 0; k < R; k++) {
            double r = rf(n, k) / scale;
            for (int t = 0; t < kBzNS; t++) {
                const double a = (r + magic[t]) - magic[t];
                r -= a;
                // q = 5: [B_0; B_1; B_2]; q = 6: per output half h, [B_0h; B_1h; B_2h]
                const int row = q == 5 ? t * R + n : (n / (R / 2)) * (kBzNS * (R / 2)) + t * (R / 2) + n % (R / 2);
                const size_t off = size_t(row >> 3) * sbo + size_t(k >> 3) * kOzLbo + size_t(row & 7) * 16 +
                                   size_t(k & 7) * 2;
                const uint16_t bits = bf16_bits_exact(a);
                std::memcpy(host_out + off, &bits, 2);
            }
        }
    }
}

template <int Q>
void launch_bz_t(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                 const std::vector<int>& cvals, const void* dmat, cudaStream_t st) {
    using B = Bz<Q>;
    OzDevice& D = oz_init();
    bool& attr = Q == 5 ? D.attr_bz5 : D.attr_bz6;
    if (!attr) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_bz<Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(B::Smem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_bz<Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(B::Smem)));
        attr = true;
    }
    std::vector<int> fixed(targets);
    uint64_t setmask = 0;
    for (size_t i = 0; i < controls.size(); i++) {
        fixed.push_back(controls[i]);
        if (cvals[i]) setmask |= 1ull << controls[i];
    }
    BzParams<Q> P;
    P.ip = make_index_plan(n, fixed, setmask);
    P.wait_spins = g_oz_wait_spins.load();
    P.force_late = g_oz_force_late.load();
    P.n_groups = P.ip.n_iter;
    for (int w = 0; w < B::D; w++) {
        uint64_t o = 0;
        for (int j = 0; j < Q; j++)
            if ((w >> j) & 1) o |= 1ull << targets[j];
        P.offs[w] = o;
    }
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const unsigned grid =
        unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(B::MinBlocks) * uint64_t(D.sms))));
    if (targets[0] == 0 && (reinterpret_cast<uintptr_t>(psi) & 15) == 0)
        k_dense_bz<Q, true><<<grid, B::Threads, B::Smem, st>>>(reinterpret_cast<float2*>(psi),
                                                               static_cast<const unsigned char*>(dmat), P, D.err);
    else
        k_dense_bz<Q, false><<<grid, B::Threads, B::Smem, st>>>(reinterpret_cast<float2*>(psi),
                                                                static_cast<const unsigned char*>(dmat), P, D.err);
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_dense_bz(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                     const std::vector<int>& cvals, const void* dmat, cudaStream_t st) {
    QS_REQUIRE(targets.size() == 5 || targets.size() == 6, "complex64 tensor-core path takes 5 or 6 targets");
    QS_REQUIRE(std::is_sorted(targets.begin(), targets.end()), "targets must be ascending");
    if (targets.size() == 5) {
        launch_bz_t<5>(psi, n, targets, controls, cvals, dmat, st);
        return;
    }
    OzDevice& D = oz_init();
    if (!D.attr_bz6) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_bz6<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBz6Smem)));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_bz6<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBz6Smem)));
        D.attr_bz6 = true;
    }
    std::vector<int> fixed(targets);
    uint64_t setmask = 0;
    for (size_t i = 0; i < controls.size(); i++) {
        fixed.push_back(controls[i]);
        if (cvals[i]) setmask |= 1ull << controls[i];
    }
    Bz6Params P;
    P.ip = make_index_plan(n, fixed, setmask);
    P.n_groups = P.ip.n_iter;
    P.wait_spins = g_oz_wait_spins.load();
    P.force_late = g_oz_force_late.load();
    for (int w = 0; w < kBz6D; w++) {
        uint64_t o = 0;
        for (int j = 0; j < 6; j++)
            if ((w >> j) & 1) o |= 1ull << targets[j];
        P.offs[w] = o;
    }
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(D.sms))));
    const bool pairs = targets[0] == 0 && (reinterpret_cast<uintptr_t>(psi) & 15) == 0;
    auto kern = pairs ? k_dense_bz6<true> : k_dense_bz6<false>;
    kern<<<grid, kBz6Threads, kBz6Smem, st>>>(reinterpret_cast<float2*>(psi), static_cast<const unsigned char*>(dmat), P,
                                              D.err);
    QS_TRY_CUDA(cudaGetLastError());
}

// device-side error recorded by a tensor-core kernel on the current device (a bounded wait ran
// out); cleared on read
bool oz_error_pending() {
    int dev = 0;
    QS_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kOzMaxDevices) return false;
    int* flag = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_oz_mu);
        flag = g_oz_dev[dev].err;
    }
    if (!flag) return false;
    int e = 0;
    QS_TRY_CUDA(cudaMemcpy(&e, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) QS_TRY_CUDA(cudaMemset(flag, 0, sizeof(int)));
    return e != 0;
}

// test hooks: try_wait attempts of the tensor-core kernels' accumulator and pipeline waits (< 0:
// the default limit), and whether their first accumulator wait reports a timeout at once
void oz_set_wait_spins(long long spins) { g_oz_wait_spins.store(spins < 0 ? kOzSpinLimit : spins); }
void oz_set_force_late(bool on) { g_oz_force_late.store(on ? 1 : 0); }

}  // namespace qs
