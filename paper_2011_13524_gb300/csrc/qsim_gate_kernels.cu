// Gate-update kernels (Sec. 4.3.2): dense gate matrices on 1..6 targets with controls,
// diagonal gates, phases on a subspace, Pauli strings and SWAPs, for complex64 and
// complex128 states. All work in place on the state vector.
//
// Every kernel enumerates the 2^(n - fixed) elements x0 of B(0) (Eq. update_mat) with
// the fixed bits (targets, controls) inserted at their positions; consecutive threads
// take consecutive x0, so for every target position a warp's accesses to each of the
// 2^m amplitudes of its groups form contiguous runs (coalesced for low and high targets
// alike). Grids are a multiple of the SM count, each thread striding over the range.
#include <algorithm>

#include "qsim_kernels.cuh"

namespace qs {

namespace {

constexpr int kThreads = 256;

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

unsigned grid_for(uint64_t work, int per_thread = 1) {
    const uint64_t want = (work + uint64_t(kThreads) * per_thread - 1) / (uint64_t(kThreads) * per_thread);
    const uint64_t cap = uint64_t(sm_count()) * 16;  // 16 resident-ish CTAs per SM, then stride
    return unsigned(std::max<uint64_t>(1, std::min(want, cap)));
}

// ------------------------------------------------------------------ dense, registers
template <typename R, int M>
struct DenseRegParams {
    IndexPlan ip;
    uint64_t offs[1 << M];
    typename CT<R>::type K[(1 << M) * (1 << M)];
};

template <typename R, int M>
__global__ void __launch_bounds__(kThreads) k_dense_reg(typename CT<R>::type* __restrict__ psi,
                                                        const __grid_constant__ DenseRegParams<R, M> P) {
    using C = typename CT<R>::type;
    constexpr int D = 1 << M;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t x0 = expand(i, P.ip);
        C v[D];
#pragma unroll
        for (int w = 0; w < D; w++) v[w] = psi[x0 + P.offs[w]];
#pragma unroll
        for (int z = 0; z < D; z++) {
            C acc = cmul(P.K[z * D], v[0]);
#pragma unroll
            for (int w = 1; w < D; w++) acc = cfma(P.K[z * D + w], v[w], acc);
            psi[x0 + P.offs[z]] = acc;
        }
    }
}

// ------------------------------------------------------------------ dense, shared-memory tile
// For 4..6 targets: a CTA stages G groups of 2^M amplitudes in shared memory (coalesced
// loads: consecutive threads read consecutive x0), then thread (rc, g) forms 8 output rows
// of group g from the staged vector and the gate matrix held in shared memory.
struct DenseSmemParams {
    IndexPlan ip;
    uint64_t offs[64];
};

template <typename R, int M>
__global__ void __launch_bounds__(kThreads) k_dense_smem(typename CT<R>::type* __restrict__ psi,
                                                         const typename CT<R>::type* __restrict__ Kg,
                                                         const __grid_constant__ DenseSmemParams P) {
    using C = typename CT<R>::type;
    constexpr int D = 1 << M;
    constexpr int RC = D / 8;          // row chunks of 8
    constexpr int G = kThreads / RC;   // groups per tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Ks = reinterpret_cast<C*>(smem_raw);
    C* tile = Ks + D * D;              // tile[w * G + g]
    uint64_t* xs = reinterpret_cast<uint64_t*>(tile + D * G);
    for (int e = threadIdx.x; e < D * D; e += kThreads) Ks[e] = Kg[e];
    const int g = threadIdx.x % G, rc = threadIdx.x / G;
    const uint64_t n_tiles = (P.ip.n_iter + G - 1) / G;
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint64_t base = t * G;
        __syncthreads();  // previous tile fully consumed
        if (threadIdx.x < G) {
            const uint64_t i = base + threadIdx.x;
            xs[threadIdx.x] = i < P.ip.n_iter ? expand(i, P.ip) : ~0ull;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < D * G; e += kThreads) {
            const int w = e / G, gg = e % G;
            const uint64_t x0 = xs[gg];
            if (x0 != ~0ull) tile[e] = psi[x0 + P.offs[w]];
        }
        __syncthreads();
        const uint64_t x0 = xs[g];
        if (x0 != ~0ull) {
            C acc[8];
#pragma unroll
            for (int r = 0; r < 8; r++) acc[r] = cmake<C>(0.0, 0.0);
#pragma unroll 4
            for (int w = 0; w < D; w++) {
                const C v = tile[w * G + g];
#pragma unroll
                for (int r = 0; r < 8; r++) acc[r] = cfma(Ks[(rc * 8 + r) * D + w], v, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < 8; r++) psi[x0 + P.offs[rc * 8 + r]] = acc[r];
        }
    }
}

// ------------------------------------------------------------------ diagonal
struct DiagParams {
    IndexPlan ip;  // controls only
    int32_t m;
    int32_t tpos[QS_MAX_TARGETS];
    double2 d[1 << QS_MAX_TARGETS];
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_diag(typename CT<R>::type* __restrict__ psi,
                                                   const __grid_constant__ DiagParams P) {
    using C = typename CT<R>::type;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t x = expand(i, P.ip);
        int r = 0;
#pragma unroll 1
        for (int j = 0; j < P.m; j++) r |= int((x >> P.tpos[j]) & 1) << j;
        const double2 dd = P.d[r];
        psi[x] = cmul(cmake<C>(dd.x, dd.y), psi[x]);
    }
}

// ------------------------------------------------------------------ phase on a subspace
// psi_x *= phase for every x whose fixed bits match; mode 0 general, 1..3 = i^mode (exact).
struct PhaseParams {
    IndexPlan ip;
    double2 phase;
    int32_t mode;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_phase(typename CT<R>::type* __restrict__ psi,
                                                    const __grid_constant__ PhaseParams P) {
    using C = typename CT<R>::type;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const C ph = cmake<C>(P.phase.x, P.phase.y);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t x = expand(i, P.ip);
        const C v = psi[x];
        psi[x] = P.mode == 0 ? cmul(ph, v) : mul_ipow(v, P.mode);
    }
}

// ------------------------------------------------------------------ Pauli string
// P|y> = i^{#Y} (-1)^{popcount(y & z)} |y ^ x>: pairs (y, y ^ x) with the pivot bit (lowest
// bit of x) clear; controls fixed. x == 0: sign flips where popcount(y & z) is odd.
struct PauliParams {
    IndexPlan ip;
    uint64_t xmask, zmask;
    int32_t nY;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_pauli(typename CT<R>::type* __restrict__ psi,
                                                    const __grid_constant__ PauliParams P) {
    using C = typename CT<R>::type;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t y = expand(i, P.ip);
        if (P.xmask == 0) {
            if (parity64(y & P.zmask)) psi[y] = mul_ipow(psi[y], 2);
            continue;
        }
        const uint64_t y2 = y ^ P.xmask;
        const C a = psi[y], b = psi[y2];
        // new psi[y2] = ph s(y) a ; new psi[y] = ph s(y2) b
        psi[y2] = mul_ipow(a, P.nY + 2 * parity64(y & P.zmask));
        psi[y] = mul_ipow(b, P.nY + 2 * parity64(y2 & P.zmask));
    }
}

// ------------------------------------------------------------------ SWAP
// fixed bits: a = 1, b = 0 (+ controls); swap psi[x] <-> psi[x ^ (a | b)].
struct SwapParams {
    IndexPlan ip;
    uint64_t flip;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_swap(typename CT<R>::type* __restrict__ psi,
                                                   const __grid_constant__ SwapParams P) {
    using C = typename CT<R>::type;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t x = expand(i, P.ip);
        const C a = psi[x], b = psi[x ^ P.flip];
        psi[x] = b;
        psi[x ^ P.flip] = a;
    }
}

// ------------------------------------------------------------------ basis state
template <typename R>
__global__ void k_set_basis(typename CT<R>::type* __restrict__ psi, uint64_t N, uint64_t j) {
    using C = typename CT<R>::type;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
        psi[i] = cmake<C>(i == j ? 1.0 : 0.0, 0.0);
}

// ------------------------------------------------------------------ launch helpers
template <typename R, int M>
void launch_dense_reg(const Op& op, const IndexPlan& ip, void* psi, cudaStream_t st) {
    using C = typename CT<R>::type;
    DenseRegParams<R, M> P;
    P.ip = ip;
    constexpr int D = 1 << M;
    for (int w = 0; w < D; w++) {
        uint64_t o = 0;
        for (int j = 0; j < M; j++)
            if ((w >> j) & 1) o |= 1ull << op.targets[j];
        P.offs[w] = o;
    }
    for (int e = 0; e < D * D; e++) {
        C c;
        c.x = R(op.data[e].real());
        c.y = R(op.data[e].imag());
        P.K[e] = c;
    }
    k_dense_reg<R, M><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), P);
}

template <typename R, int M>
void launch_dense_smem(const Op& op, const IndexPlan& ip, void* psi, const void* dK, cudaStream_t st) {
    using C = typename CT<R>::type;
    constexpr int D = 1 << M;
    constexpr int G = kThreads / (D / 8);
    DenseSmemParams P;
    P.ip = ip;
    for (int w = 0; w < D; w++) {
        uint64_t o = 0;
        for (int j = 0; j < M; j++)
            if ((w >> j) & 1) o |= 1ull << op.targets[j];
        P.offs[w] = o;
    }
    const size_t smem = sizeof(C) * (D * D + D * G) + sizeof(uint64_t) * G;
    static bool attr_set = false;
    if (!attr_set) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_smem<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        attr_set = true;
    }
    const uint64_t n_tiles = (ip.n_iter + G - 1) / G;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(sm_count()) * 4)));
    k_dense_smem<R, M><<<grid, kThreads, smem, st>>>(reinterpret_cast<C*>(psi), reinterpret_cast<const C*>(dK), P);
}

}  // namespace

template <typename R>
static void launch_typed(const Op& op, void* psi, int n, cudaStream_t st, void* stage) {
    using C = typename CT<R>::type;
    std::vector<int> fixed;
    uint64_t setmask = 0;
    for (size_t j = 0; j < op.controls.size(); j++) {
        fixed.push_back(op.controls[j]);
        if (op.cvals[j]) setmask |= 1ull << op.controls[j];
    }
    switch (op.kind) {
        case OpKind::Dense: {
            const int m = int(op.targets.size());
            for (int t : op.targets) fixed.push_back(t);
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            if (m == 1) return launch_dense_reg<R, 1>(op, ip, psi, st);
            if (m == 2) return launch_dense_reg<R, 2>(op, ip, psi, st);
            if (m == 3) return launch_dense_reg<R, 3>(op, ip, psi, st);
            if (m == 4 && sizeof(R) == 4) return launch_dense_reg<R, 4>(op, ip, psi, st);
            // the shared-memory kernels read the matrix from device memory: either the
            // caller's copy (already in the state's element type) or the state's staging
            // buffer, refilled by a copy queued on the same stream before the launch
            const void* dK = op.dmat;
            if (!dK) {
                QS_REQUIRE(stage != nullptr, "no staging buffer for a wide dense gate");
                const int D = 1 << m;
                std::vector<C> hk(size_t(D) * D);
                for (size_t e = 0; e < hk.size(); e++) {
                    hk[e].x = R(op.data[e].real());
                    hk[e].y = R(op.data[e].imag());
                }
                QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), hk.size() * sizeof(C), cudaMemcpyHostToDevice, st));
                dK = stage;
            }
            if (m == 4) return launch_dense_smem<R, 4>(op, ip, psi, dK, st);
            if (m == 5) return launch_dense_smem<R, 5>(op, ip, psi, dK, st);
            if (m == 6) return launch_dense_smem<R, 6>(op, ip, psi, dK, st);
            throw Error{QS_ERR_UNSUPPORTED, "dense gates act on at most 6 targets"};
        }
        case OpKind::Diag: {
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            DiagParams P;
            P.ip = ip;
            P.m = int(op.targets.size());
            for (int j = 0; j < P.m; j++) P.tpos[j] = op.targets[j];
            for (size_t e = 0; e < op.data.size(); e++) P.d[e] = make_double2(op.data[e].real(), op.data[e].imag());
            k_diag<R><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), P);
            return;
        }
        case OpKind::Phase: {
            if (op.phase == cplx(1.0, 0.0)) return;
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            PhaseParams P;
            P.ip = ip;
            P.phase = make_double2(op.phase.real(), op.phase.imag());
            P.mode = 0;
            if (op.phase == cplx(0.0, 1.0)) P.mode = 1;
            if (op.phase == cplx(-1.0, 0.0)) P.mode = 2;
            if (op.phase == cplx(0.0, -1.0)) P.mode = 3;
            k_phase<R><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), P);
            return;
        }
        case OpKind::Pauli: {
            if (op.xmask == 0 && op.zmask == 0) return;
            if (op.xmask) fixed.push_back(__builtin_ctzll(op.xmask));
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            PauliParams P;
            P.ip = ip;
            P.xmask = op.xmask;
            P.zmask = op.zmask;
            P.nY = __builtin_popcountll(op.xmask & op.zmask);
            k_pauli<R><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), P);
            return;
        }
        case OpKind::Swap: {
            const int a = op.targets[0], b = op.targets[1];
            fixed.push_back(a);
            fixed.push_back(b);
            IndexPlan ip = make_index_plan(n, fixed, setmask | (1ull << a));
            SwapParams P;
            P.ip = ip;
            P.flip = (1ull << a) | (1ull << b);
            k_swap<R><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), P);
            return;
        }
    }
}

void launch_op(const Op& op, void* psi, int n, qs_dtype dt, cudaStream_t st, void* stage) {
    if (dt == QS_C64)
        launch_typed<float>(op, psi, n, st, stage);
    else
        launch_typed<double>(op, psi, n, st, stage);
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_set_basis(void* psi, int n, qs_dtype dt, uint64_t j, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    if (dt == QS_C64)
        k_set_basis<float><<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<float2*>(psi), N, j);
    else
        k_set_basis<double><<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<double2*>(psi), N, j);
    QS_TRY_CUDA(cudaGetLastError());
}

}  // namespace qs
