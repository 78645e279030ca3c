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
// D_0..D_6, one per d; they are combined exactly from the smallest (each D_d is a multiple of
// the unit in the last place of the partial sum below it, so Fast2Sum is error-free) into a
// double-float value and scaled back by mu_n nu. What is dropped (slice remainders below
// 2^-48 and the products with s + t >= 7) bounds the error at about 2^-45 of max|v| max|K~|
// per output, the accuracy of the double-float CUDA-core kernels.
//
// Tile: 128 groups (the MMA's M = 128, TMEM lane = group), K = 32 real inputs. The stacked
// matrix slices [B_0; ...; B_5] (192 x 32) let one MMA per state slice s and K-step cover all
// its products: columns (s + t) * 32 of the accumulator block receive A_s B_t, so a single
// MMA with N = 32 * min(6, 7 - s) feeds diagonals s..min(s + 5, 6).
//
// Pipeline: two CTAs per SM (256 threads, ~95 KB of shared memory and 256 TMEM columns
// each), so that one CTA's tensor-core and memory phases overlap the other's CUDA-core work.
// Within a CTA: slice tile j, start its MMAs, start the cp.async loads of tile j + 1, then
// read the accumulators (TMEM -> double-float -> shared staging) and store tile j coalesced.
// Every mbarrier wait is bounded; on expiry the kernel records an error, waits (bounded) for
// its MMAs and frees TMEM.
#include <algorithm>
#include <cmath>
#include <cstring>

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
constexpr int kOzElemsPerThread = kOzTG * kOzD / kOzThreads;   // 8 loads / stores per tile
constexpr uint32_t kOzSbo = (kOzR / 8) * 128;                  // 8-row group stride (K-major)
constexpr uint32_t kOzLbo = 128;
constexpr size_t kOzSlice = size_t(kOzTG) * kOzR * 2;          // one state slice, bf16
constexpr size_t kOzABuf = kOzNS * kOzSlice;                   // 48 KB
constexpr size_t kOzRaw = size_t(kOzTG) * kOzD * 16;           // 32 KB of double-float amplitudes
constexpr size_t kOzMat = size_t(kOzNS) * kOzR * kOzR * 2;     // 12 KB
constexpr int kOzAccCols = kOzND * kOzR;                       // 224 columns per accumulator set
constexpr int kOzTmemCols = 256;                               // one set, rounded to a power of 2
constexpr long long kOzSpinLimit = 1ll << 22;

static_assert(kOzABuf >= kOzRaw, "output staging reuses a slice buffer");
static_assert(kOzAccCols <= kOzTmemCols, "accumulators fit the TMEM allocation");

// shared-memory plan (bytes), ~95 KB: two CTAs per SM
constexpr size_t kOffRaw = 0;                           // 32 KB
constexpr size_t kOffA = kOffRaw + kOzRaw;              // 48 KB (slices, then output staging)
constexpr size_t kOffMat = kOffA + kOzABuf;             // 12 KB
constexpr size_t kOffMu = kOffMat + kOzMat;             // 32 floats
constexpr size_t kOffNu = kOffMu + kOzR * 4;            // 128 floats
constexpr size_t kOffNuPart = kOffNu + kOzTG * 4;       // 2 x 128 floats
constexpr size_t kOffX0 = kOffNuPart + 2 * kOzTG * 4;   // 2 x 128 uint64
constexpr size_t kOzSmem = kOffX0 + 2 * kOzTG * 8;

struct OzParams {
    IndexPlan ip;            // 4 targets (and controls) inserted
    uint64_t offs[kOzD];     // s(w), targets ascending
    uint64_t n_groups;
    int low;                 // targets 0..low-1 are qubits 0..low-1 (coalescing)
    int swz;                 // swizzle shift of the staging slots: max(0, 3 - low)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major core-matrix offset of bf16 element (row r, column k), K = 32
__device__ __forceinline__ uint32_t kmaj(uint32_t r, uint32_t k) {
    return (r >> 3) * kOzSbo + (k >> 3) * kOzLbo + (r & 7) * 16 + (k & 7) * 2;
}
// raw / staging slot of (group g, amplitude w): w-major, XOR-swizzled in 16-byte units so that
// eight consecutive lanes hit eight bank groups both when they share w (consecutive g) and when
// they run over the 2^low low amplitudes of 8 / 2^low groups (the coalesced load order)
__device__ __forceinline__ uint32_t raw_slot(uint32_t g, uint32_t w, int swz) {
    return w * kOzTG + (g ^ ((w << swz) & 7));
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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long spins = 0; spins < kOzSpinLimit; spins++) {
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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// value rounded to a multiple of 2^-8(s+1) (|x| <= 2^(14-8s)); the magic constant is
// 1.5 * 2^(23 - 8(s+1)), the sum lands in its binade and the low bits are rounded off
template <int S>
__device__ __forceinline__ float grid_round(float x) {
    constexpr float c = 1.5f * float(1 << 15) / float(1ull << (8 * S));
    return __fsub_rn(__fadd_rn(x, c), c);
}

// the six slices of x = (h + l) * inv_nu, each exact in bf16 (see the header comment)
__device__ __forceinline__ void slice6(float h, float l, float inv_nu, float (&a)[kOzNS]) {
    h = __fmul_rn(h, inv_nu);
    l = __fmul_rn(l, inv_nu);
    a[0] = grid_round<0>(h);
    float r = __fsub_rn(h, a[0]);
    a[1] = grid_round<1>(r);
    r = __fsub_rn(r, a[1]);
    a[2] = grid_round<2>(r);
    r = __fadd_rn(__fsub_rn(r, a[2]), l);  // rounding error below 2^-49
    a[3] = grid_round<3>(r);
    r = __fsub_rn(r, a[3]);
    a[4] = grid_round<4>(r);
    a[5] = grid_round<5>(__fsub_rn(r, a[4]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// (a + b) exactly as (s, t) when a is a multiple of ulp(b) or |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    t = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float pow2_ceil(float m) {
    // smallest power of two >= m for m > 0 (1 for m == 0), exponent kept in range
    if (!(m > 0.f)) return 1.f;
    uint32_t e = ((__float_as_uint(m) + 0x007FFFFFu) >> 23) & 0xFFu;
    e = e < 1u ? 1u : (e > 253u ? 253u : e);
    return __uint_as_float(e << 23);
}

__global__ void __launch_bounds__(kOzThreads, 2) k_dense_oz4(float4* __restrict__ psi, const unsigned char* __restrict__ dmat,
                                                             const __grid_constant__ OzParams P, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid & (kOzTG - 1), h = tid >> 7;  // group and amplitude half of this thread
    const int swz = P.swz;
    float4* raw = reinterpret_cast<float4*>(smem + kOffRaw);
    unsigned char* abuf = smem + kOffA;
    const float* mu = reinterpret_cast<const float*>(smem + kOffMu);
    float* nu = reinterpret_cast<float*>(smem + kOffNu);
    float* nu_part = reinterpret_cast<float*>(smem + kOffNuPart);
    uint64_t* x0s = reinterpret_cast<uint64_t*>(smem + kOffX0);

    // matrix slices (stacked, already in the K-major layout) and row scales, once per CTA
    for (int i = tid; i < int((kOzMat + kOzR * 4) / 16); i += kOzThreads)
        reinterpret_cast<uint4*>(smem + kOffMat)[i] = reinterpret_cast<const uint4*>(dmat)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
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

    // this thread's loads / stores of a tile: element e -> (group, amplitude) with consecutive e
    // at consecutive addresses where the low targets allow it; fixed for every tile
    uint32_t el_g[kOzElemsPerThread], el_slot[kOzElemsPerThread];
    uint64_t el_off[kOzElemsPerThread];
    {
        const uint32_t lowmask = (1u << P.low) - 1u;
#pragma unroll
        for (int i = 0; i < kOzElemsPerThread; i++) {
            const uint32_t e = uint32_t(tid + i * kOzThreads);
            const uint32_t wl = e & lowmask, rest = e >> P.low;
            const uint32_t gg = rest & (kOzTG - 1), w = ((rest >> 7) << P.low) | wl;
            el_g[i] = gg;
            el_slot[i] = raw_slot(gg, w, swz);
            el_off[i] = P.offs[w];
        }
    }
    auto fill_x0 = [&](uint64_t j) {
        const uint64_t tile = blockIdx.x + j * gridDim.x;
        if (tid < kOzTG) {
            const uint64_t gi = tile * kOzTG + tid;
            x0s[(j & 1) * kOzTG + tid] = gi < P.n_groups ? expand(gi, P.ip) : ~0ull;
        }
    };
    auto load = [&](uint64_t j) {  // cp.async of tile j into raw (x0 list ready)
        const uint64_t* x = x0s + (j & 1) * kOzTG;
        const uint32_t base = smem_u32(raw);
#pragma unroll
        for (int i = 0; i < kOzElemsPerThread; i++) {
            const uint64_t x0 = x[el_g[i]];
            const bool ok = x0 != ~0ull;
            cp_async16(base + el_slot[i] * 16, ok ? psi + x0 + el_off[i] : psi, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto slice = [&](uint64_t j) {  // raw -> state slices in abuf, scales nu; x0 list of tile j + 1
        if (j + 1 < my_tiles) fill_x0(j + 1);
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < kOzAmpsPerThread; i++) {
            const float4 v = raw[raw_slot(g, h * kOzAmpsPerThread + i, swz)];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.z)));
        }
        nu_part[h * kOzTG + g] = m;
        __syncthreads();
        m = fmaxf(nu_part[g], nu_part[kOzTG + g]);
        const float nv = pow2_ceil(m);
        if (h == 0) nu[g] = nv;
        const float inv = __uint_as_float((254u - (__float_as_uint(nv) >> 23)) << 23);
        // two passes of 4 amplitudes = K columns 16h + 8c .. 16h + 8c + 7: one 16-byte chunk per slice
#pragma unroll
        for (int c = 0; c < 2; c++) {
            uint32_t pk[kOzNS][4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float4 v = raw[raw_slot(g, h * kOzAmpsPerThread + 4 * c + i, swz)];
                float ar[kOzNS], ai[kOzNS];
                slice6(v.x, v.y, inv, ar);
                slice6(v.z, v.w, inv, ai);
#pragma unroll
                for (int s = 0; s < kOzNS; s++) pk[s][i] = pack_bf16(ar[s], ai[s]);
            }
            const uint32_t off = kmaj(uint32_t(g), uint32_t(16 * h + 8 * c));
#pragma unroll
            for (int s = 0; s < kOzNS; s++)
                *reinterpret_cast<uint4*>(abuf + s * kOzSlice + off) = make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    auto issue = [&]() {  // MMAs of the tile into the accumulator set
        if (tid != 0) return;
        const uint32_t a0 = smem_u32(abuf), m0 = smem_u32(smem + kOffMat);
        // state slice s times matrix slices t = t0 .. t0 + nt - 1 into diagonals s + t
        auto prod = [&](int s, int t0, int nt, int ks, uint32_t acc) {
            mma_bf16(tmem + uint32_t((s + t0) * kOzR), sdesc(a0 + uint32_t(s * kOzSlice) + uint32_t(ks * 256)),
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
            for (int s = 2; s < kOzNS; s++) prod(s, 0, kOzND - s < kOzNS ? kOzND - s : kOzNS, ks, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    };
    auto epilogue = [&]() {  // accumulators -> double-float outputs in the staging area (abuf)
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        const float nv = nu[g];
        float4* stg = reinterpret_cast<float4*>(abuf);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const int col0 = 16 * h + 8 * c;  // 8 output reals = 4 amplitudes
            uint32_t r[kOzND][8];
#pragma unroll
            for (int d = 0; d < kOzND; d++) {
                const uint32_t taddr = tmem + lane_base + uint32_t(d * kOzR + col0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3]), "=r"(r[d][4]),
                               "=r"(r[d][5]), "=r"(r[d][6]), "=r"(r[d][7])
                             : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 4; i++) {
                float o[4];
#pragma unroll
                for (int cc = 0; cc < 2; cc++) {
                    const int col = 2 * i + cc;
                    float sm = __uint_as_float(r[kOzND - 1][col]), lo = 0.f, t;
#pragma unroll
                    for (int d = kOzND - 2; d >= 0; d--) {
                        fast_two_sum(__uint_as_float(r[d][col]), sm, sm, t);
                        lo = __fadd_rn(lo, t);
                    }
                    const float sc = __fmul_rn(mu[col0 + col], nv);
                    fast_two_sum(__fmul_rn(sm, sc), __fmul_rn(lo, sc), o[2 * cc], o[2 * cc + 1]);
                }
                stg[raw_slot(g, (col0 >> 1) + i, swz)] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    };
    auto store = [&](uint64_t j) {  // staging -> the state, coalesced
        const uint64_t* x = x0s + (j & 1) * kOzTG;
        const float4* stg = reinterpret_cast<const float4*>(abuf);
#pragma unroll
        for (int i = 0; i < kOzElemsPerThread; i++) {
            const uint64_t x0 = x[el_g[i]];
            if (x0 != ~0ull) psi[x0 + el_off[i]] = stg[el_slot[i]];
        }
    };

    if (my_tiles > 0) {
        fill_x0(0);
        __syncthreads();
        load(0);
    }
    for (uint64_t j = 0; j < my_tiles; j++) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();  // raw holds tile j; the staging area of tile j - 1 has been stored
        slice(j);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue();
        if (j + 1 < my_tiles) load(j + 1);  // raw is free: fetch the next tile while the tensor cores work
        if (tid == 0 && !mbar_wait(smem_u32(&mbar), uint32_t(j & 1))) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        epilogue();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        store(j);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (s_fail && tid == 0) {
        atomicExch(err, 1);
        mbar_wait(smem_u32(&mbar), 0);  // bounded: let the MMAs in flight finish before TMEM is freed
        mbar_wait(smem_u32(&mbar), 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
}

int g_oz_sms = 0;
int* g_oz_err = nullptr;

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
                const double u = std::ldexp(1.0, -8 * (t + 1));
                const double a = std::nearbyint(r / u) * u;
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
                      const std::vector<int>& cvals, const void* dmat, cudaStream_t st) {
    QS_REQUIRE(targets.size() == size_t(kOzQ), "tensor-core double-float path takes 4 targets");
    QS_REQUIRE(std::is_sorted(targets.begin(), targets.end()), "targets must be ascending");
    if (!g_oz_sms) {
        int dev = 0;
        QS_TRY_CUDA(cudaGetDevice(&dev));
        QS_TRY_CUDA(cudaDeviceGetAttribute(&g_oz_sms, cudaDevAttrMultiProcessorCount, dev));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_oz4, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kOzSmem)));
        QS_TRY_CUDA(cudaMalloc(&g_oz_err, sizeof(int)));
        QS_TRY_CUDA(cudaMemset(g_oz_err, 0, sizeof(int)));
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
    int low = 0;
    while (low < kOzQ && targets[low] == low) low++;
    P.low = low;
    P.swz = low >= 3 ? 0 : 3 - low;
    P.n_groups = P.ip.n_iter;
    const uint64_t n_tiles = (P.n_groups + kOzTG - 1) / kOzTG;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, 2 * uint64_t(g_oz_sms))));
    k_dense_oz4<<<grid, kOzThreads, kOzSmem, st>>>(reinterpret_cast<float4*>(psi),
                                                   static_cast<const unsigned char*>(dmat), P, g_oz_err);
    QS_TRY_CUDA(cudaGetLastError());
}

// device-side error recorded by the kernel (a bounded wait ran out); cleared on read
bool oz_error_pending() {
    if (!g_oz_err) return false;
    int e = 0;
    QS_TRY_CUDA(cudaMemcpy(&e, g_oz_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) QS_TRY_CUDA(cudaMemset(g_oz_err, 0, sizeof(int)));
    return e != 0;
}

}  // namespace qs
