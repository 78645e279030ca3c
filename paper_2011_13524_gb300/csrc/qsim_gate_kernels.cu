// Gate-update kernels (Sec. 4.3.2): dense gate matrices on 1..6 targets with controls,
// diagonal gates, phases on a subspace, Pauli strings and SWAPs. Each kernel is written once
// over an arithmetic policy (qsim_arith.cuh): complex64 in FP32, complex128 in FP64, and
// complex128 held as double-float pairs on the FP32 pipes. All work in place.
//
// Every kernel enumerates the 2^(n - fixed) elements x0 of B(0) (Eq. update_mat) with
// the fixed bits (targets, controls) inserted at their positions; consecutive threads
// take consecutive x0, so for every target position a warp's accesses to each of the
// 2^m amplitudes of its groups form contiguous runs (coalesced for low and high targets
// alike). Grids are a multiple of the SM count, each thread striding over the range.
#include <algorithm>
#include <type_traits>
#include <cstring>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kThreads = 256;
// elementwise in-place passes take this many amplitudes per thread and step, so that as many
// loads are in flight before the first store (the stores alias the loaded buffer, so the
// compiler keeps the order)
constexpr int kConvUnroll = 4;

int sm_count() { return device_sms(); }

unsigned grid_for(uint64_t work) {
    const uint64_t want = (work + kThreads - 1) / kThreads;
    const uint64_t cap = uint64_t(sm_count()) * 16;  // 16 CTAs per SM, then stride
    return unsigned(std::max<uint64_t>(1, std::min(want, cap)));
}

// ------------------------------------------------------------------ dense, registers
template <typename P, int M>
struct DenseRegParams {
    IndexPlan ip;
    uint64_t offs[1 << M];
    typename P::K K[(1 << M) * (1 << M)];
};

template <typename P, int M>
__global__ void __launch_bounds__(kThreads) k_dense_reg(typename P::C* __restrict__ psi,
                                                        const __grid_constant__ DenseRegParams<P, M> Pm) {
    using C = typename P::C;
    constexpr int D = 1 << M;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Pm.ip.n_iter; i += stride) {
        const uint64_t x0 = expand(i, Pm.ip);
        C v[D];
#pragma unroll
        for (int w = 0; w < D; w++) v[w] = psi[x0 + Pm.offs[w]];
#pragma unroll
        for (int z = 0; z < D; z++) {
            typename P::Acc a = P::first(Pm.K[z * D], v[0]);
#pragma unroll
            for (int w = 1; w < D; w++) P::mac(a, Pm.K[z * D + w], v[w]);
            psi[x0 + Pm.offs[z]] = P::out(a);
        }
    }
}

// ------------------------------------------------------------------ dense, shared-memory tile
// For 4..6 targets: a CTA stages G groups of 2^M amplitudes in shared memory (coalesced
// loads: consecutive threads read consecutive x0), then thread (rc, g) forms R output rows
// of group g from the staged vector and the gate matrix held in shared memory. The tile shape
// (R rows per thread, so G = 256 R / 2^M groups per tile) is a template parameter, 4, 8 or 16;
// the autotuner times the three on this GPU per arithmetic and width and keeps the fastest
// (dense_tile_rows). Every output is the same sum in the same order whatever R is.
struct DenseSmemParams {
    IndexPlan ip;
    uint64_t offs[64];
};

template <typename P, int M, int R>
__global__ void __launch_bounds__(kThreads) k_dense_smem(typename P::C* __restrict__ psi,
                                                         const typename P::K* __restrict__ Kg,
                                                         const __grid_constant__ DenseSmemParams Pm) {
    using C = typename P::C;
    using K = typename P::K;
    constexpr int D = 1 << M;
    constexpr int RC = D / R;          // row chunks of R
    constexpr int G = kThreads / RC;   // groups per tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* Ks = reinterpret_cast<K*>(smem_raw);
    C* tile = reinterpret_cast<C*>(Ks + D * D);   // tile[w * G + g]
    uint64_t* xs = reinterpret_cast<uint64_t*>(tile + D * G);
    for (int e = threadIdx.x; e < D * D; e += kThreads) Ks[e] = Kg[e];
    const int g = threadIdx.x % G, rc = threadIdx.x / G;
    const uint64_t n_tiles = (Pm.ip.n_iter + G - 1) / G;
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint64_t base = t * G;
        __syncthreads();  // previous tile fully consumed
        if (threadIdx.x < G) {
            const uint64_t i = base + threadIdx.x;
            xs[threadIdx.x] = i < Pm.ip.n_iter ? expand(i, Pm.ip) : ~0ull;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < D * G; e += kThreads) {
            const int w = e / G, gg = e % G;
            const uint64_t x0 = xs[gg];
            if (x0 != ~0ull) tile[e] = psi[x0 + Pm.offs[w]];
        }
        __syncthreads();
        const uint64_t x0 = xs[g];
        if (x0 != ~0ull) {
            typename P::Acc acc[R];
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = P::zero();
#pragma unroll 2
            for (int w = 0; w < D; w++) {
                const C v = tile[w * G + g];
#pragma unroll
                for (int r = 0; r < R; r++) P::mac(acc[r], Ks[(rc * R + r) * D + w], v);
            }
#pragma unroll
            for (int r = 0; r < R; r++) psi[x0 + Pm.offs[rc * R + r]] = P::out(acc[r]);
        }
    }
}

// ------------------------------------------------------------------ diagonal
template <typename P>
struct DiagParams {
    IndexPlan ip;  // controls only
    int32_t m;
    int32_t tpos[QS_MAX_TARGETS];
    typename P::K d[1 << QS_MAX_TARGETS];
};

template <typename P>
__global__ void __launch_bounds__(kThreads) k_diag(typename P::C* __restrict__ psi,
                                                   const __grid_constant__ DiagParams<P> Pm) {
    using C = typename P::C;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < Pm.ip.n_iter; i0 += kConvUnroll * stride) {
        uint64_t x[kConvUnroll];
        C v[kConvUnroll];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            x[u] = i0 + u * stride < Pm.ip.n_iter ? expand(i0 + u * stride, Pm.ip) : ~0ull;
            if (x[u] != ~0ull) v[u] = __ldcg(psi + x[u]);
        }
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            if (x[u] == ~0ull) continue;
            int r = 0;
#pragma unroll 1
            for (int j = 0; j < Pm.m; j++) r |= int((x[u] >> Pm.tpos[j]) & 1) << j;
            typename P::Acc a = P::zero();
            P::mac(a, Pm.d[r], v[u]);
            psi[x[u]] = P::out(a);
        }
    }
}

// Several diagonal blocks (no controls) in one pass: psi_x *= t[r(x)] t2[r2(x)] with the product
// of their diagonals held as two tables over two sets of qubits (at most kDiagTableBits and
// kDiagTable2Bits; the second may be empty), staged in shared memory per CTA; r(x) and r2(x)
// gather those qubits' bits of x.
template <typename P>
struct DiagTableParams {
    uint64_t N;
    int32_t m, m2;
    int32_t second;  // 0: no second table; 1: general entries; 2: entries 1, i, -1, -i only
    int32_t nrun, nrun2;
    // runs of consecutive table qubits: shift (bits 0..7), width (8..15), table bit (16..23)
    uint32_t run[kDiagTableBits];
    uint32_t run2[kDiagTable2Bits];
};

// table index of x: its bits at the table's qubits, gathered run by run
__device__ __forceinline__ uint32_t gather_runs(uint64_t x, const uint32_t* run, int nrun) {
    uint32_t r = 0;
    for (int k = 0; k < nrun; k++) {
        const uint32_t c = run[k];
        r |= (uint32_t(x >> (c & 0xFFu)) & ((1u << ((c >> 8) & 0xFFu)) - 1u)) << (c >> 16);
    }
    return r;
}

// i^k (re + i im) of a double-float amplitude by selects and sign flips (exact)
__device__ __forceinline__ float4 quarter_turn(const float4& v, int k) {
    const bool sw = (k & 1) != 0;
    const uint32_t sre = (k == 1 || k == 2) ? 0x80000000u : 0u, sim = (k & 2) ? 0x80000000u : 0u;
    const float ah = sw ? v.z : v.x, al = sw ? v.w : v.y, bh = sw ? v.x : v.z, bl = sw ? v.y : v.w;
    return make_float4(__uint_as_float(__float_as_uint(ah) ^ sre), __uint_as_float(__float_as_uint(al) ^ sre),
                       __uint_as_float(__float_as_uint(bh) ^ sim), __uint_as_float(__float_as_uint(bl) ^ sim));
}

// k of an entry i^k (1, i, -1 or -i exactly): a quarter turn applied by swaps and signs
__device__ __forceinline__ int quarter_of(const float2& k) { return k.x > 0.5f ? 0 : k.y > 0.5f ? 1 : k.x < -0.5f ? 2 : 3; }
__device__ __forceinline__ int quarter_of(const double2& k) { return k.x > 0.5 ? 0 : k.y > 0.5 ? 1 : k.x < -0.5 ? 2 : 3; }
__device__ __forceinline__ int quarter_of(const float4& k) { return k.x > 0.5f ? 0 : k.z > 0.5f ? 1 : k.x < -0.5f ? 2 : 3; }

// kIeeeOut (double-float only): the products are written as IEEE complex128, RN(hi + lo) per
// component (the join of the layout-change pass), into the same 16 bytes.
// Chunks of 2^11 amplitudes, four per thread (four loads in flight): the table indices are
// gathers of the bits of x at the tables' qubits, and a gather is an OR over disjoint bit sets,
// so r(x) = r(chunk base) | r(x mod 2^11): the low part is fixed per thread and computed once,
// the high part once per chunk. One wave of CTAs (two of 512 threads per SM) that each stage
// the tables once.
constexpr int kDiagThreads = 512;
constexpr int kDiagPer = 4;
constexpr int kDiagChunkBits = 11;  // kDiagThreads x kDiagPer amplitudes per chunk
static_assert(kDiagThreads * kDiagPer == 1 << kDiagChunkBits, "chunk size");
template <typename P, bool kIeeeOut>
__global__ void __launch_bounds__(kDiagThreads, 2) k_diag_table(typename P::C* __restrict__ psi,
                                                         const typename P::K* __restrict__ table,
                                                         const __grid_constant__ DiagTableParams<P> Pm) {
    using C = typename P::C;
    extern __shared__ __align__(16) unsigned char dsm[];
    typename P::K* t = reinterpret_cast<typename P::K*>(dsm);
    const typename P::K* t2 = t + (1 << Pm.m);
    const int entries = (1 << Pm.m) + (Pm.m2 > 0 ? 1 << Pm.m2 : 0);
    for (int i = threadIdx.x; i < entries; i += blockDim.x) t[i] = table[i];
    __syncthreads();
    uint32_t rl[kDiagPer], rl2[kDiagPer];
#pragma unroll
    for (int u = 0; u < kDiagPer; u++) {
        const uint64_t j = threadIdx.x + uint64_t(u) * kDiagThreads;
        rl[u] = gather_runs(j, Pm.run, Pm.nrun);
        rl2[u] = gather_runs(j, Pm.run2, Pm.nrun2);
    }
    const uint64_t n_chunks = (Pm.N + (1ull << kDiagChunkBits) - 1) >> kDiagChunkBits;
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint64_t base = ch << kDiagChunkBits;
        const uint32_t rh = gather_runs(base, Pm.run, Pm.nrun), rh2 = gather_runs(base, Pm.run2, Pm.nrun2);
        C v[kDiagPer];
#pragma unroll
        for (int u = 0; u < kDiagPer; u++) {
            const uint64_t x = base + threadIdx.x + uint64_t(u) * kDiagThreads;
            if (x < Pm.N) v[u] = __ldcg(psi + x);
        }
#pragma unroll
        for (int u = 0; u < kDiagPer; u++) {
            const uint64_t x = base + threadIdx.x + uint64_t(u) * kDiagThreads;
            if (x >= Pm.N) continue;
            const uint32_t r = rh | rl[u], r2 = rh2 | rl2[u];
            C w = v[u];
            if (Pm.second == 2) {  // exact quarter turn, then the first table's entry
                if constexpr (std::is_same<P, DFArith>::value)
                    w = quarter_turn(w, quarter_of(t2[r2]));
                else
                    w = P::ipow(w, quarter_of(t2[r2]));
            }
            typename P::Acc a;
            if constexpr (std::is_same<P, DFArith>::value) {
                a = P::first(t[r], w);
            } else {
                a = P::zero();
                P::mac(a, t[r], w);
            }
            if (Pm.second == 1) {
                const C y = P::out(a);
                a = P::zero();
                P::mac(a, t2[r2], y);
            }
            if constexpr (kIeeeOut) {
                const float4 o = P::out(a);
                reinterpret_cast<double2*>(psi)[x] = make_double2(join_df_int(o.x, o.y), join_df_int(o.z, o.w));
            } else {
                psi[x] = P::out(a);
            }
        }
    }
}

template <typename P>
void launch_diag_table_t(const std::vector<int>& u, const std::vector<cplx>& tab, const std::vector<int>& u2,
                         const std::vector<cplx>& tab2, void* psi, int n, cudaStream_t st, void* stage,
                         bool ieee_out) {
    using K = typename P::K;
    const size_t entries = tab.size() + (u2.empty() ? 0 : tab2.size());
    const size_t bytes = entries * sizeof(K);
    constexpr size_t kMaxBytes = sizeof(K) * ((size_t(1) << kDiagTableBits) + (size_t(1) << kDiagTable2Bits));
    QS_REQUIRE(stage != nullptr && bytes <= kStageBytes && bytes <= kMaxBytes, "no staging buffer for a diagonal table");
    std::vector<K> hk(entries);
    for (size_t i = 0; i < tab.size(); i++) hk[i] = P::host_k(tab[i].real(), tab[i].imag());
    for (size_t i = tab.size(); i < entries; i++) hk[i] = P::host_k(tab2[i - tab.size()].real(), tab2[i - tab.size()].imag());
    QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), bytes, cudaMemcpyHostToDevice, st));
    QS_TRY_CUDA(cudaStreamSynchronize(st));  // hk is host memory that dies on return
    DiagTableParams<P> Pm;
    Pm.N = 1ull << n;
    Pm.m = int(u.size());
    Pm.m2 = int(u2.size());
    Pm.second = 0;
    if (!u2.empty()) {
        auto quarter = [](const cplx& z) {
            return (z.imag() == 0.0 && (z.real() == 1.0 || z.real() == -1.0)) ||
                   (z.real() == 0.0 && (z.imag() == 1.0 || z.imag() == -1.0));
        };
        Pm.second = std::all_of(tab2.begin(), tab2.end(), quarter) ? 2 : 1;
    }
    auto runs = [](const std::vector<int>& q, uint32_t* run) {  // q ascending
        int nr = 0;
        for (size_t j = 0; j < q.size();) {
            size_t k = j + 1;
            while (k < q.size() && q[k] == q[k - 1] + 1) k++;
            run[nr++] = uint32_t(q[j]) | (uint32_t(k - j) << 8) | (uint32_t(j) << 16);
            j = k;
        }
        return nr;
    };
    Pm.nrun = runs(u, Pm.run);
    Pm.nrun2 = runs(u2, Pm.run2);
    static PerDevice setup;
    static int resident_of[kMaxDevices][2];  // CTAs per SM at the largest table, without / with IEEE output
    setup.once([](int dev) {
        int* r = resident_of[dev];
        r[0] = r[1] = 1;
        QS_TRY_CUDA(cudaFuncSetAttribute(k_diag_table<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kMaxBytes)));
        QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[0], k_diag_table<P, false>, kDiagThreads, kMaxBytes));
        if constexpr (std::is_same<P, DFArith>::value) {
            QS_TRY_CUDA(cudaFuncSetAttribute(k_diag_table<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kMaxBytes)));
            QS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[1], k_diag_table<P, true>, kDiagThreads,
                                                                      kMaxBytes));
        }
    });
    const int* resident = resident_of[current_device()];
    auto kern = k_diag_table<P, false>;
    if constexpr (std::is_same<P, DFArith>::value) {
        if (ieee_out) kern = k_diag_table<P, true>;
    } else {
        QS_REQUIRE(!ieee_out, "IEEE output is a double-float layout change");
    }
    const uint64_t want = (Pm.N + (1ull << kDiagChunkBits) - 1) >> kDiagChunkBits;
    const uint64_t wave = uint64_t(sm_count()) * uint64_t(std::max(1, resident[ieee_out ? 1 : 0]));
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want, wave)));
    kern<<<grid, kDiagThreads, bytes, st>>>(reinterpret_cast<typename P::C*>(psi), static_cast<const K*>(stage), Pm);
    QS_TRY_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ phase on a subspace
// psi_x *= phase for every x whose fixed bits match; mode 0 general, 1..3 = i^mode (exact).
template <typename P>
struct PhaseParams {
    IndexPlan ip;
    typename P::K phase;
    int32_t mode;
};

template <typename P>
__global__ void __launch_bounds__(kThreads) k_phase(typename P::C* __restrict__ psi,
                                                    const __grid_constant__ PhaseParams<P> Pm) {
    using C = typename P::C;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < Pm.ip.n_iter; i0 += kConvUnroll * stride) {
        uint64_t x[kConvUnroll];
        C v[kConvUnroll];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            x[u] = i0 + u * stride < Pm.ip.n_iter ? expand(i0 + u * stride, Pm.ip) : ~0ull;
            if (x[u] != ~0ull) v[u] = __ldcg(psi + x[u]);
        }
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            if (x[u] == ~0ull) continue;
            if (Pm.mode == 0) {
                typename P::Acc a = P::zero();
                P::mac(a, Pm.phase, v[u]);
                psi[x[u]] = P::out(a);
            } else {
                psi[x[u]] = P::ipow(v[u], Pm.mode);
            }
        }
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

template <typename P>
__global__ void __launch_bounds__(kThreads) k_pauli(typename P::C* __restrict__ psi,
                                                    const __grid_constant__ PauliParams Pm) {
    using C = typename P::C;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Pm.ip.n_iter; i += stride) {
        const uint64_t y = expand(i, Pm.ip);
        if (Pm.xmask == 0) {
            if (parity64(y & Pm.zmask)) psi[y] = P::ipow(psi[y], 2);
            continue;
        }
        const uint64_t y2 = y ^ Pm.xmask;
        const C a = psi[y], b = psi[y2];
        psi[y2] = P::ipow(a, Pm.nY + 2 * parity64(y & Pm.zmask));
        psi[y] = P::ipow(b, Pm.nY + 2 * parity64(y2 & Pm.zmask));
    }
}

// ------------------------------------------------------------------ Pauli rotation
// exp(i phi P / 2) = cos(phi/2) I + i sin(phi/2) P for a Pauli string P of any length (Sec.
// 4.3.2, Pauli rotation gate), P|y> = i^nY (-1)^popc(y & zmask) |y ^ xmask>. With X or Y factors
// the update pairs y (pivot bit 0) with y ^ xmask; a Z string (or the identity) is diagonal.
template <typename P>
struct PauliRotParams {
    IndexPlan ip;
    uint64_t xmask, zmask;
    typename P::K c;      // cos(phi/2)
    typename P::K kp, km;  // +- i^(1 + nY) sin(phi/2); diagonal case: cos +- i sin
};

template <typename P>
__global__ void __launch_bounds__(kThreads) k_pauli_rot(typename P::C* __restrict__ psi,
                                                        const __grid_constant__ PauliRotParams<P> Pm) {
    using C = typename P::C;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Pm.ip.n_iter; i += stride) {
        const uint64_t y = expand(i, Pm.ip);
        if (Pm.xmask == 0) {
            psi[y] = P::out(P::first(parity64(y & Pm.zmask) ? Pm.km : Pm.kp, psi[y]));
            continue;
        }
        const uint64_t y2 = y ^ Pm.xmask;
        const C a = psi[y], b = psi[y2];
        typename P::Acc ra = P::first(Pm.c, a), rb = P::first(Pm.c, b);
        P::mac(ra, parity64(y2 & Pm.zmask) ? Pm.km : Pm.kp, b);
        P::mac(rb, parity64(y & Pm.zmask) ? Pm.km : Pm.kp, a);
        psi[y] = P::out(ra);
        psi[y2] = P::out(rb);
    }
}

// ------------------------------------------------------------------ SWAP
// fixed bits: a = 1, b = 0 (+ controls); swap psi[x] <-> psi[x ^ (a | b)].
struct SwapParams {
    IndexPlan ip;
    uint64_t flip;
};

template <typename P>
__global__ void __launch_bounds__(kThreads) k_swap(typename P::C* __restrict__ psi,
                                                   const __grid_constant__ SwapParams Pm) {
    using C = typename P::C;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Pm.ip.n_iter; i += stride) {
        const uint64_t x = expand(i, Pm.ip);
        const C a = psi[x], b = psi[x ^ Pm.flip];
        psi[x] = b;
        psi[x ^ Pm.flip] = a;
    }
}

// ------------------------------------------------------------------ basis state, layouts
template <typename P>
__global__ void k_set_basis(typename P::C* __restrict__ psi, uint64_t N, uint64_t j) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) psi[i] = P::basis(i == j);
}

// IEEE complex128 <-> double-float, in place (same 16 bytes per amplitude), with the
// integer-pipe splits of qsim_arith.cuh
// In-place layout changes, four amplitudes per thread and step (kConvUnroll).
__global__ void k_to_df(double2* __restrict__ psi, uint64_t N) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < N; i0 += kConvUnroll * stride) {
        double2 v[kConvUnroll];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++)
            if (i0 + u * stride < N) v[u] = psi[i0 + u * stride];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            if (i0 + u * stride >= N) continue;
            float4 r;
            split_double_int(v[u].x, r.x, r.y);
            split_double_int(v[u].y, r.z, r.w);
            reinterpret_cast<float4*>(psi)[i0 + u * stride] = r;
        }
    }
}
__global__ void k_from_df(double2* __restrict__ psi, uint64_t N) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < N; i0 += kConvUnroll * stride) {
        float4 v[kConvUnroll];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++)
            if (i0 + u * stride < N) v[u] = reinterpret_cast<const float4*>(psi)[i0 + u * stride];
#pragma unroll
        for (int u = 0; u < kConvUnroll; u++) {
            if (i0 + u * stride >= N) continue;
            psi[i0 + u * stride] = make_double2(join_df_int(v[u].x, v[u].y), join_df_int(v[u].z, v[u].w));
        }
    }
}

// ------------------------------------------------------------------ launch helpers
template <int M>
void fill_offs(const Op& op, uint64_t* offs) {
    for (int w = 0; w < (1 << M); w++) {
        uint64_t o = 0;
        for (int j = 0; j < M; j++)
            if ((w >> j) & 1) o |= 1ull << op.targets[j];
        offs[w] = o;
    }
}

template <typename P, int M>
void launch_dense_reg(const Op& op, const IndexPlan& ip, void* psi, cudaStream_t st) {
    DenseRegParams<P, M> Pm;
    Pm.ip = ip;
    fill_offs<M>(op, Pm.offs);
    constexpr int D = 1 << M;
    for (int e = 0; e < D * D; e++) Pm.K[e] = P::host_k(op.data[e].real(), op.data[e].imag());
    k_dense_reg<P, M><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<typename P::C*>(psi), Pm);
}

template <typename P, int M, int R>
void launch_dense_smem_r(const DenseSmemParams& Pm, void* psi, const void* dK, cudaStream_t st) {
    using C = typename P::C;
    using K = typename P::K;
    constexpr int D = 1 << M;
    constexpr int G = kThreads / (D / R);
    const size_t smem = sizeof(K) * D * D + sizeof(C) * D * G + sizeof(uint64_t) * G;
    static PerDevice setup;
    setup.once([smem](int) {
        QS_TRY_CUDA(cudaFuncSetAttribute(k_dense_smem<P, M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    });
    const uint64_t n_tiles = (Pm.ip.n_iter + G - 1) / G;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, uint64_t(sm_count()) * 4)));
    k_dense_smem<P, M, R><<<grid, kThreads, smem, st>>>(reinterpret_cast<C*>(psi), reinterpret_cast<const K*>(dK), Pm);
}

template <typename P, int M>
void launch_dense_smem(const Op& op, const IndexPlan& ip, void* psi, const void* dK, cudaStream_t st) {
    DenseSmemParams Pm;
    Pm.ip = ip;
    fill_offs<M>(op, Pm.offs);
    const Arith ar = std::is_same<P, DFArith>::value ? Arith::DF
                     : sizeof(typename P::C) == 8  ? Arith::F32
                                                    : Arith::F64;
    switch (dense_tile_rows(ar, M)) {
        case 4: return launch_dense_smem_r<P, M, 4>(Pm, psi, dK, st);
        case 16: return launch_dense_smem_r<P, M, 16>(Pm, psi, dK, st);
        default: return launch_dense_smem_r<P, M, 8>(Pm, psi, dK, st);
    }
}

template <typename P>
void launch_with(const Op& op, void* psi, int n, cudaStream_t st, void* stage, bool ieee_in) {
    using C = typename P::C;
    using K = typename P::K;
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
            // complex64 blocks of 5 or 6 targets: tensor cores, bf16 slices with exact sums
            if (sizeof(C) == 8 && (m == 5 || m == 6) && tensor_c64x_enabled()) {
                const Op os = op.dmat_oz ? op : sort_targets(op);
                const void* dK = op.dmat_oz ? op.dmat : nullptr;
                if (!dK) {
                    QS_REQUIRE(stage != nullptr && bz_matrix_bytes(m) <= kStageBytes, "no staging buffer for a wide dense gate");
                    std::vector<unsigned char> hk(bz_matrix_bytes(m));
                    prepare_bz_matrix(m, os.data, hk.data());
                    QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), hk.size(), cudaMemcpyHostToDevice, st));
                    QS_TRY_CUDA(cudaStreamSynchronize(st));  // hk is host memory that dies on return
                    dK = stage;
                }
                return launch_dense_bz(psi, n, os.targets, os.controls, os.cvals, dK, st);
            }
            // double-float blocks of 4 targets: tensor cores (targets ascending)
            if (std::is_same<P, DFArith>::value && m == 4 && tensor_c128_enabled()) {
                const Op os = op.dmat_oz ? op : sort_targets(op);
                const void* dK = op.dmat_oz ? op.dmat : nullptr;
                if (!dK) {
                    QS_REQUIRE(stage != nullptr, "no staging buffer for a wide dense gate");
                    std::vector<unsigned char> hk(oz4_matrix_bytes());
                    prepare_oz4_matrix(os.data, hk.data());
                    QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), hk.size(), cudaMemcpyHostToDevice, st));
                    QS_TRY_CUDA(cudaStreamSynchronize(st));  // hk is host memory that dies on return
                    dK = stage;
                }
                return launch_dense_oz4(psi, n, os.targets, os.controls, os.cvals, dK, st, ieee_in);
            }
            // double-float blocks of 5 targets: tensor cores, outputs in two halves
            if (std::is_same<P, DFArith>::value && m == 5 && tensor_c128_enabled()) {
                const Op os = op.dmat_oz ? op : sort_targets(op);
                const void* dK = op.dmat_oz ? op.dmat : nullptr;
                if (!dK) {
                    QS_REQUIRE(stage != nullptr && oz5_matrix_bytes() <= kStageBytes, "no staging buffer for a wide dense gate");
                    std::vector<unsigned char> hk(oz5_matrix_bytes());
                    prepare_oz5_matrix(os.data, hk.data());
                    QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), hk.size(), cudaMemcpyHostToDevice, st));
                    QS_TRY_CUDA(cudaStreamSynchronize(st));  // hk is host memory that dies on return
                    dK = stage;
                }
                return launch_dense_oz5(psi, n, os.targets, os.controls, os.cvals, dK, st, ieee_in);
            }
            if (m == 1) return launch_dense_reg<P, 1>(op, ip, psi, st);
            if (m == 2) return launch_dense_reg<P, 2>(op, ip, psi, st);
            if (m == 3) return launch_dense_reg<P, 3>(op, ip, psi, st);
            if (m == 4 && sizeof(C) == 8) return launch_dense_reg<P, 4>(op, ip, psi, st);
            // the shared-memory kernels read the matrix from device memory: either the
            // caller's copy (already in this policy's entry type) or the state's staging
            // buffer, refilled by a copy queued on the same stream before the launch
            const void* dK = op.dmat;
            if (!dK) {
                QS_REQUIRE(stage != nullptr, "no staging buffer for a wide dense gate");
                const int D = 1 << m;
                std::vector<K> hk(size_t(D) * D);
                for (size_t e = 0; e < hk.size(); e++) hk[e] = P::host_k(op.data[e].real(), op.data[e].imag());
                QS_TRY_CUDA(cudaMemcpyAsync(stage, hk.data(), hk.size() * sizeof(K), cudaMemcpyHostToDevice, st));
                QS_TRY_CUDA(cudaStreamSynchronize(st));  // hk is host memory that dies on return
                dK = stage;
            }
            if (m == 4) return launch_dense_smem<P, 4>(op, ip, psi, dK, st);
            if (m == 5) return launch_dense_smem<P, 5>(op, ip, psi, dK, st);
            if (m == 6) return launch_dense_smem<P, 6>(op, ip, psi, dK, st);
            throw Error{QS_ERR_UNSUPPORTED, "dense gates act on at most 6 targets"};
        }
        case OpKind::Diag: {
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            DiagParams<P> Pm;
            Pm.ip = ip;
            Pm.m = int(op.targets.size());
            for (int j = 0; j < Pm.m; j++) Pm.tpos[j] = op.targets[j];
            for (size_t e = 0; e < op.data.size(); e++) Pm.d[e] = P::host_k(op.data[e].real(), op.data[e].imag());
            k_diag<P><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), Pm);
            return;
        }
        case OpKind::Phase: {
            if (op.phase == cplx(1.0, 0.0)) return;
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            PhaseParams<P> Pm;
            Pm.ip = ip;
            Pm.phase = P::host_k(op.phase.real(), op.phase.imag());
            Pm.mode = 0;
            if (op.phase == cplx(0.0, 1.0)) Pm.mode = 1;
            if (op.phase == cplx(-1.0, 0.0)) Pm.mode = 2;
            if (op.phase == cplx(0.0, -1.0)) Pm.mode = 3;
            k_phase<P><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), Pm);
            return;
        }
        case OpKind::Pauli: {
            if (op.xmask == 0 && op.zmask == 0) return;
            if (op.xmask) fixed.push_back(__builtin_ctzll(op.xmask));
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            PauliParams Pm;
            Pm.ip = ip;
            Pm.xmask = op.xmask;
            Pm.zmask = op.zmask;
            Pm.nY = __builtin_popcountll(op.xmask & op.zmask);
            k_pauli<P><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), Pm);
            return;
        }
        case OpKind::PauliRot: {
            if (op.xmask) fixed.push_back(__builtin_ctzll(op.xmask));
            IndexPlan ip = make_index_plan(n, fixed, setmask);
            PauliRotParams<P> Pm;
            Pm.ip = ip;
            Pm.xmask = op.xmask;
            Pm.zmask = op.zmask;
            const double c = std::cos(op.angle / 2), sn = std::sin(op.angle / 2);
            Pm.c = P::host_k(c, 0.0);
            if (op.xmask) {
                // i^(1 + nY) sin
                const int e = (1 + __builtin_popcountll(op.xmask & op.zmask)) & 3;
                const double re = e == 0 ? sn : e == 2 ? -sn : 0.0, im = e == 1 ? sn : e == 3 ? -sn : 0.0;
                Pm.kp = P::host_k(re, im);
                Pm.km = P::host_k(-re, -im);
            } else {
                Pm.kp = P::host_k(c, sn);
                Pm.km = P::host_k(c, -sn);
            }
            k_pauli_rot<P><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), Pm);
            return;
        }
        case OpKind::Swap: {
            const int a = op.targets[0], b = op.targets[1];
            fixed.push_back(a);
            fixed.push_back(b);
            IndexPlan ip = make_index_plan(n, fixed, setmask | (1ull << a));
            SwapParams Pm;
            Pm.ip = ip;
            Pm.flip = (1ull << a) | (1ull << b);
            k_swap<P><<<grid_for(ip.n_iter), kThreads, 0, st>>>(reinterpret_cast<C*>(psi), Pm);
            return;
        }
    }
}

}  // namespace

// the double-float launch of op reads every amplitude once in a kernel that can take the IEEE
// layout itself: an uncontrolled dense block of 4 or 5 targets on the tensor cores
bool takes_ieee_in(const Op& op) {
    const size_t m = op.targets.size();
    return op.kind == OpKind::Dense && op.controls.empty() && (m == 4 || m == 5) && tensor_c128_enabled();
}

void launch_op_arith(const Op& op, void* psi, int n, Arith ar, cudaStream_t st, void* stage, bool ieee_in) {
    QS_REQUIRE(!ieee_in || ar == Arith::DF, "IEEE input is a double-float layout change");
    if (ieee_in && !takes_ieee_in(op)) {
        launch_to_df(psi, n, st);
        ieee_in = false;
    }
    switch (ar) {
        case Arith::F32: launch_with<NativeArith<float>>(op, psi, n, st, stage, false); break;
        case Arith::F64: launch_with<NativeArith<double>>(op, psi, n, st, stage, false); break;
        case Arith::DF: launch_with<DFArith>(op, psi, n, st, stage, ieee_in); break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

bool diag_split_add(DiagSplit& sp, const std::vector<int>& qubits) {
    auto joined = [&](const std::vector<int>& u) {
        std::vector<int> w(u);
        for (int q : qubits)
            if (std::find(w.begin(), w.end(), q) == w.end()) w.push_back(q);
        return w;
    };
    std::vector<int> w = joined(sp.u);
    if (w.size() <= size_t(kDiagTableBits)) {
        sp.u.swap(w);
        sp.side.push_back(0);
        return true;
    }
    w = joined(sp.u2);
    if (w.size() <= size_t(kDiagTable2Bits)) {
        sp.u2.swap(w);
        sp.side.push_back(1);
        return true;
    }
    return false;
}

// Diagonal ops (uncontrolled diagonals, on their targets, and phases, on their control qubits'
// values) applied as one pass: the product of their diagonals as two tables over the two qubit
// sets of diag_split_add.
void launch_diag_run(const Op* ops, size_t count, void* psi, int n, Arith ar, cudaStream_t st, void* stage,
                     bool ieee_out) {
    auto qubits = [](const Op& op) -> const std::vector<int>& {
        return op.kind == OpKind::Phase ? op.controls : op.targets;
    };
    DiagSplit sp;
    for (size_t i = 0; i < count; i++) {
        QS_REQUIRE((ops[i].kind == OpKind::Diag && ops[i].controls.empty()) || ops[i].kind == OpKind::Phase,
                   "diagonal run of uncontrolled diagonals and phases");
        QS_REQUIRE(diag_split_add(sp, qubits(ops[i])), "diagonal run on too many qubits");
    }
    std::sort(sp.u.begin(), sp.u.end());
    std::sort(sp.u2.begin(), sp.u2.end());
    std::vector<cplx> tab(size_t(1) << sp.u.size(), cplx(1.0, 0.0)), tab2(size_t(1) << sp.u2.size(), cplx(1.0, 0.0));
    for (size_t i = 0; i < count; i++) {
        const std::vector<int>& u = sp.side[i] ? sp.u2 : sp.u;
        std::vector<cplx>& t = sp.side[i] ? tab2 : tab;
        std::vector<int> pos;  // bit of the table index for each qubit of op i
        for (int q : qubits(ops[i])) pos.push_back(int(std::find(u.begin(), u.end(), q) - u.begin()));
        for (size_t r = 0; r < t.size(); r++) {
            size_t ri = 0;
            for (size_t j = 0; j < pos.size(); j++) ri |= ((r >> pos[j]) & 1) << j;
            if (ops[i].kind == OpKind::Phase) {
                bool match = true;
                for (size_t j = 0; j < pos.size(); j++) match = match && int((ri >> j) & 1) == ops[i].cvals[j];
                if (match) t[r] *= ops[i].phase;
            } else {
                t[r] *= ops[i].data[ri];
            }
        }
    }
    switch (ar) {
        case Arith::F32:
            launch_diag_table_t<NativeArith<float>>(sp.u, tab, sp.u2, tab2, psi, n, st, stage, ieee_out);
            break;
        case Arith::F64:
            launch_diag_table_t<NativeArith<double>>(sp.u, tab, sp.u2, tab2, psi, n, st, stage, ieee_out);
            break;
        case Arith::DF: launch_diag_table_t<DFArith>(sp.u, tab, sp.u2, tab2, psi, n, st, stage, ieee_out); break;
    }
}

void launch_op(const Op& op, void* psi, int n, qs_dtype dt, cudaStream_t st, void* stage) {
    launch_op_arith(op, psi, n, dt == QS_C64 ? Arith::F32 : Arith::F64, st, stage);
}

void launch_set_basis_arith(void* psi, int n, Arith ar, uint64_t j, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    switch (ar) {
        case Arith::F32:
            k_set_basis<NativeArith<float>><<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<float2*>(psi), N, j);
            break;
        case Arith::F64:
            k_set_basis<NativeArith<double>><<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<double2*>(psi), N, j);
            break;
        case Arith::DF:
            k_set_basis<DFArith><<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<float4*>(psi), N, j);
            break;
    }
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_set_basis(void* psi, int n, qs_dtype dt, uint64_t j, cudaStream_t st) {
    launch_set_basis_arith(psi, n, dt == QS_C64 ? Arith::F32 : Arith::F64, j, st);
}

void launch_to_df(void* psi, int n, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    k_to_df<<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<double2*>(psi), N);
    QS_TRY_CUDA(cudaGetLastError());
}

void launch_from_df(void* psi, int n, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    k_from_df<<<grid_for(N), kThreads, 0, st>>>(reinterpret_cast<double2*>(psi), N);
    QS_TRY_CUDA(cudaGetLastError());
}

Op sort_targets(const Op& op) {
    const int m = int(op.targets.size());
    std::vector<int> perm(m);
    for (int j = 0; j < m; j++) perm[j] = j;
    std::sort(perm.begin(), perm.end(), [&](int a, int b) { return op.targets[a] < op.targets[b]; });
    Op r = op;
    for (int j = 0; j < m; j++) r.targets[j] = op.targets[perm[j]];
    if (op.kind == OpKind::Dense) {
        const int D = 1 << m;
        auto old_index = [&](int x) {  // bit j of the new local index is bit perm[j] of the old one
            int o = 0;
            for (int j = 0; j < m; j++)
                if ((x >> j) & 1) o |= 1 << perm[j];
            return o;
        };
        for (int z = 0; z < D; z++)
            for (int w = 0; w < D; w++) r.data[size_t(z) * D + w] = op.data[size_t(old_index(z)) * D + old_index(w)];
    }
    r.dmat = nullptr;
    r.dmat_oz = false;
    return r;
}

// matrix entries in the form a policy's kernels read from device memory
size_t kernel_entry_bytes(Arith ar) { return ar == Arith::F32 ? 8 : 16; }
void encode_entries(Arith ar, const std::vector<cplx>& m, unsigned char* dst) {
    for (size_t e = 0; e < m.size(); e++) {
        if (ar == Arith::F32) {
            float2 k = NativeArith<float>::host_k(m[e].real(), m[e].imag());
            std::memcpy(dst + 8 * e, &k, 8);
        } else if (ar == Arith::F64) {
            double2 k = NativeArith<double>::host_k(m[e].real(), m[e].imag());
            std::memcpy(dst + 16 * e, &k, 16);
        } else {
            float4 k = DFArith::host_k(m[e].real(), m[e].imag());
            std::memcpy(dst + 16 * e, &k, 16);
        }
    }
}

}  // namespace qs
