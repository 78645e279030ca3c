// Fused 6-qubit dense blocks on a complex64 state with the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in TMEM).
//
// A fused block applies a 64 x 64 complex gate matrix K~ to 2^(n-6) vectors of 64 amplitudes
// (Eq. update_mat with m = 6): a dense (64 x 64) . (64 x 2^(n-6)) contraction. As a real GEMM,
//     [Re y; Im y] = [[Kr, -Ki], [Ki, Kr]] [Re v; Im v]   (128 x 128 times 128 x groups).
// A tile holds 32 groups: the CTA gathers their 64 amplitudes (coalesced over the groups),
// splits every FP32 value x into a TF32 head h (low 13 mantissa bits cleared) and the FP32
// remainder l = x - h, and computes D = Ah Bh + Ah Bl + Al Bh with 48 MMAs (M = 128, N = 32,
// K = 8 each) into TMEM ("3xTF32": FP32-class accuracy from TF32 tensor cores). The gather of
// tile t+1 overlaps the MMAs of tile t; the epilogue reads D from TMEM, stages it in shared
// memory and stores the 64 outputs of each group coalesced over the groups. The remainders are
// rounded to TF32 (nearest-even) before the tensor cores read them, so the error is unbiased
// (truncation alone would shrink the norm by ~2^-22 per block).
//
// Operands sit in shared memory K-major without swizzle: 8-row x 16-byte core matrices, LBO =
// 128 B between core matrices along K, SBO = 4096 B between 8-row groups. Every mbarrier wait is
// bounded; on expiry the kernel records an error, waits (bounded) for its MMAs and frees TMEM.
#include <algorithm>
#include <cstring>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;            // 2 x 64 real rows
constexpr int kTcK = 128;            // 2 x 64 real columns
constexpr int kTcN = 32;             // groups per tile
constexpr int kTcKSteps = kTcK / 8;  // MMAs of K = 8 per product
constexpr uint32_t kTcSbo = (kTcK / 4) * 128;  // 4096
constexpr uint32_t kTcLbo = 128;
constexpr int kTmemCols = 2 * kTcN;  // two accumulator buffers
constexpr long long kTcSpinLimit = 1ll << 22;

// shared-memory plan (bytes)
constexpr size_t kOffAh = 0;                                   // 128 x 128 x 4 = 64 KB
constexpr size_t kOffAl = kOffAh + size_t(kTcM) * kTcK * 4;    // 64 KB
constexpr size_t kOffB = kOffAl + size_t(kTcM) * kTcK * 4;     // 2 stages x (Bh, Bl) x 32 x 128 x 4 = 64 KB
constexpr size_t kBBytes = size_t(kTcN) * kTcK * 4;            // 16 KB per operand per stage
constexpr size_t kOffStage = kOffB + 4 * kBBytes;              // epilogue staging 128 x 32 x 4 = 16 KB
constexpr size_t kOffXs = kOffStage + size_t(kTcM) * kTcN * 4; // 2 x 32 x 8 B
constexpr size_t kTcSmem = kOffXs + 2 * kTcN * 8;

struct TcParams {
    IndexPlan ip;        // 6 targets inserted
    uint64_t offs[64];   // s(w)
    uint64_t n_groups;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major core-matrix offset of element (row r, column k)
__device__ __forceinline__ uint32_t kmaj(uint32_t r, uint32_t k) {
    return (r >> 3) * kTcSbo + (k >> 2) * kTcLbo + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((kTcLbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((kTcSbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;  // tcgen05 descriptor version; no swizzle, base offset 0
    return d;
}

// D F32, A and B TF32, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kTcN >> 3) << 17) | (uint32_t(kTcM >> 4) << 24);

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// the tensor cores read a TF32 operand by dropping the low 13 mantissa bits (toward zero); the
// remainder is rounded to nearest-even here first so the split's error has no bias
__host__ __device__ __forceinline__ uint32_t tf32_rne_bits(uint32_t u) {
    return (u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
}
__device__ __forceinline__ float tf32_rne(float x) { return __uint_as_float(tf32_rne_bits(__float_as_uint(x))); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    long long spins = 0;
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (++spins > kTcSpinLimit) return false;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_dense_tc6(float2* __restrict__ psi, const float* __restrict__ Ah,
                                                             const float* __restrict__ Al,
                                                             const __grid_constant__ TcParams P, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sAh = smem + kOffAh;
    unsigned char* sAl = smem + kOffAl;
    float* stage = reinterpret_cast<float*>(smem + kOffStage);
    uint64_t* xs = reinterpret_cast<uint64_t*>(smem + kOffXs);
    // matrix operands, once per CTA
    for (int i = tid; i < kTcM * kTcK; i += kTcThreads) {
        const uint32_t r = i / kTcK, k = i % kTcK;
        *reinterpret_cast<float*>(sAh + kmaj(r, k)) = Ah[i];
        *reinterpret_cast<float*>(sAl + kmaj(r, k)) = Al[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint64_t n_tiles = (P.n_groups + kTcN - 1) / kTcN;
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    // gather tile `t` (local index j) into stage buffer b
    auto gather = [&](uint64_t j, int b) {
        const uint64_t tile = blockIdx.x + j * gridDim.x;
        uint64_t* x = xs + b * kTcN;
        if (tid < kTcN) {
            const uint64_t gidx = tile * kTcN + tid;
            x[tid] = gidx < P.n_groups ? expand(gidx, P.ip) : ~0ull;
        }
        __syncthreads();
        unsigned char* bh = smem + kOffB + size_t(b) * 2 * kBBytes;
        unsigned char* bl = bh + kBBytes;
        // 32 groups x 64 amplitudes; consecutive threads take consecutive groups
        for (int e = tid; e < kTcN * 64; e += kTcThreads) {
            const int g = e % kTcN, w = e / kTcN;
            const uint64_t x0 = x[g];
            const float2 v = x0 != ~0ull ? psi[x0 + P.offs[w]] : make_float2(0.f, 0.f);
            const float hr = tf32_head(v.x), hi = tf32_head(v.y);
            *reinterpret_cast<float*>(bh + kmaj(g, w)) = hr;
            *reinterpret_cast<float*>(bl + kmaj(g, w)) = tf32_rne(v.x - hr);
            *reinterpret_cast<float*>(bh + kmaj(g, 64 + w)) = hi;
            *reinterpret_cast<float*>(bl + kmaj(g, 64 + w)) = tf32_rne(v.y - hi);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    // 3xTF32 product of stage buffer b into accumulator buffer b, completion on mbar[b]
    auto issue = [&](int b) {
        if (tid != 0) return;
        const uint32_t d = tmem + uint32_t(b * kTcN);
        const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl);
        const uint32_t bh = smem_u32(smem + kOffB + size_t(b) * 2 * kBBytes), bl = bh + uint32_t(kBBytes);
        for (int ks = 0; ks < kTcKSteps; ks++) {
            const uint32_t off = uint32_t(ks) * 2 * kTcLbo;  // 8 K-elements = 2 core matrices
            mma_tf32(d, sdesc(ah + off), sdesc(bl + off), ks > 0 ? 1u : 0u);
            mma_tf32(d, sdesc(al + off), sdesc(bh + off), 1u);
            mma_tf32(d, sdesc(ah + off), sdesc(bh + off), 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[b])));
    };
    // read accumulator buffer b, store the tile's outputs
    auto epilogue = [&](int b) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3, half = warp >> 2;  // lane quarter, column half
        uint32_t r[16];
        const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(b * kTcN + half * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = q * 32 + lane;
#pragma unroll
        for (int j = 0; j < 16; j++) stage[row * kTcN + half * 16 + j] = __uint_as_float(r[j]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        const uint64_t* x = xs + b * kTcN;
        for (int e = tid; e < kTcN * 64; e += kTcThreads) {
            const int g = e % kTcN, z = e / kTcN;
            const uint64_t x0 = x[g];
            if (x0 != ~0ull) psi[x0 + P.offs[z]] = make_float2(stage[z * kTcN + g], stage[(64 + z) * kTcN + g]);
        }
        __syncthreads();
    };

    if (my_tiles > 0) {
        gather(0, 0);
        __syncthreads();
        issue(0);
    }
    for (uint64_t j = 0; j < my_tiles; j++) {
        const int b = int(j & 1);
        if (j + 1 < my_tiles) {
            gather(j + 1, b ^ 1);  // overlaps the MMAs of tile j
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue(b ^ 1);
        }
        if (!mbar_wait(smem_u32(&mbar[b]), uint32_t((j >> 1) & 1))) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        epilogue(b);
    }
    if (s_fail) {
        if (tid == 0) atomicExch(err, 1);
        // let every committed MMA finish before TMEM is released (bounded)
        mbar_wait(smem_u32(&mbar[0]), 0);
        mbar_wait(smem_u32(&mbar[1]), 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

int g_tc_sms = 0;
int* g_tc_err = nullptr;

}  // namespace

// y = K v on every group of the 6 targets (K: 64 x 64 complex, FP64), complex64 state.
// Ah/Al: device buffer of 2 x 128 x 128 floats prepared by prepare_tc6_matrix (or staged here).
void prepare_tc6_matrix(const std::vector<cplx>& K, float* host_out /* 2 * 128 * 128 */) {
    float* ah = host_out;
    float* al = host_out + kTcM * kTcK;
    for (int m = 0; m < kTcM; m++)
        for (int k = 0; k < kTcK; k++) {
            const int z = m & 63, w = k & 63;
            const cplx e = K[size_t(z) * 64 + w];
            double v;
            if (m < 64) v = k < 64 ? e.real() : -e.imag();
            else v = k < 64 ? e.imag() : e.real();
            const float f = float(v);
            uint32_t u;
            std::memcpy(&u, &f, 4);
            u &= 0xFFFFE000u;
            float h;
            std::memcpy(&h, &u, 4);
            ah[m * kTcK + k] = h;
            const float rem = float(v - double(h));
            uint32_t ru;
            std::memcpy(&ru, &rem, 4);
            ru = tf32_rne_bits(ru);
            std::memcpy(&al[m * kTcK + k], &ru, 4);
        }
}

size_t tc6_matrix_bytes() { return size_t(2) * kTcM * kTcK * sizeof(float); }

void launch_dense_tc6(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                      const std::vector<int>& cvals, const float* dmat, cudaStream_t st) {
    QS_REQUIRE(targets.size() == 6, "tensor-core path takes 6 targets");
    if (!g_tc_sms) {
        int dev = 0;
        QS_TRY_CUDA(cudaGetDevice(&dev));
        QS_TRY_CUDA(cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev));
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_tc6, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem)));
        QS_TRY_CUDA(cudaMalloc(&g_tc_err, sizeof(int)));
        QS_TRY_CUDA(cudaMemset(g_tc_err, 0, sizeof(int)));
    }
    std::vector<int> fixed(targets);
    uint64_t setmask = 0;
    for (size_t j = 0; j < controls.size(); j++) {
        fixed.push_back(controls[j]);
        if (cvals[j]) setmask |= 1ull << controls[j];
    }
    TcParams P;
    P.ip = make_index_plan(n, fixed, setmask);
    for (int w = 0; w < 64; w++) {
        uint64_t o = 0;
        for (int j = 0; j < 6; j++)
            if ((w >> j) & 1) o |= 1ull << targets[j];
        P.offs[w] = o;
    }
    P.n_groups = P.ip.n_iter;
    const uint64_t n_tiles = (P.n_groups + kTcN - 1) / kTcN;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(g_tc_sms))));
    k_dense_tc6<<<grid, kTcThreads, kTcSmem, st>>>(reinterpret_cast<float2*>(psi), dmat, dmat + kTcM * kTcK, P,
                                                   g_tc_err);
    QS_TRY_CUDA(cudaGetLastError());
}

// device-side error recorded by the tensor-core kernel (a bounded wait ran out); cleared on read
bool tc_error_pending() {
    if (!g_tc_err) return false;
    int e = 0;
    QS_TRY_CUDA(cudaMemcpy(&e, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) QS_TRY_CUDA(cudaMemset(g_tc_err, 0, sizeof(int)));
    return e != 0;
}

}  // namespace qs
