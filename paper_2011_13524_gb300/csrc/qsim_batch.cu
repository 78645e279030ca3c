// Batched execution of many small parametric circuits in one persistent kernel launch,
// replayed from a CUDA graph: for every (circuit, observable) pair the energy
// E = <psi|H|psi> and the adjoint gradient dE/dtheta (reverse sweep of Sec. 4.4 parametric
// circuits, rotation convention exp(+i theta P / 2) of the paper's gate table), complex64
// storage with compensated FP32 products summed in FP64.
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
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kBT = 1024;        // threads per CTA
constexpr int kLocal = 13;       // qubits per shared-memory chunk
constexpr int kChunk = 1 << kLocal;
constexpr int kMaxBatchQubits = 24;

enum BKind : uint8_t { BK_RX = 0, BK_RY = 1, BK_RZ = 2, BK_CZ = 3, BK_CNOT = 4, BK_H = 5, BK_X = 6, BK_Y = 7, BK_Z = 8 };

struct BGate {
    uint8_t kind;
    uint8_t a;      // local bit of the target (CNOT: target)
    uint8_t b;      // local bit of the second qubit (CZ) or control (CNOT)
    uint8_t pad;
    int32_t slot;   // angle slot in the item's angle array (rotations), -1 otherwise
    int32_t grad;   // gradient index (parametric rotations), -1 otherwise
};

struct BPass {
    int32_t g0, g1;               // gate range
    uint32_t tab_lo[128];         // local index bits 0..6 -> address bits
    uint32_t tab_hi[64];          // local index bits 7..12 -> address bits
    uint32_t nonlocal;            // qubits outside the window (address bits fixed per chunk)
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

struct BatchDev {
    const BItem* items;
    const int32_t* order;
    const BPass* passes;
    const BGate* gates;
    const BTerm* terms;
    const float2* cs;             // (cos, sin) of theta/2 per angle slot
    float2* ws;                   // per-CTA workspace: psi and lambda, 2^maxn each
    uint64_t ws_stride;           // amplitudes per buffer
    double* energy;
    double* grad;
    int32_t count;
    int32_t want_grad;
    unsigned int* counter;
};

__device__ __forceinline__ uint32_t insert0(uint32_t i, int b) {
    const uint32_t lo = i & ((1u << b) - 1u);
    return ((i ^ lo) << 1) | lo;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// apply gate g (or its adjoint) to a chunk of `size` amplitudes in shared memory
__device__ void apply_local(float2* s, int size, const BGate& g, float2 cs, bool adjoint) {
    const float c = cs.x, sn = adjoint ? -cs.y : cs.y;
    switch (g.kind) {
        case BK_RX: case BK_RY: case BK_RZ: case BK_H: case BK_X: case BK_Y: {
            const int half = size >> 1;
            for (int i = threadIdx.x; i < half; i += kBT) {
                const uint32_t i0 = insert0(i, g.a), i1 = i0 | (1u << g.a);
                const float2 u = s[i0], v = s[i1];
                float2 r0, r1;
                if (g.kind == BK_RX) {         // [[c, i s], [i s, c]]
                    r0 = make_float2(c * u.x - sn * v.y, c * u.y + sn * v.x);
                    r1 = make_float2(c * v.x - sn * u.y, c * v.y + sn * u.x);
                } else if (g.kind == BK_RY) {  // [[c, s], [-s, c]]
                    r0 = make_float2(c * u.x + sn * v.x, c * u.y + sn * v.y);
                    r1 = make_float2(c * v.x - sn * u.x, c * v.y - sn * u.y);
                } else if (g.kind == BK_RZ) {  // diag(c + i s, c - i s)
                    r0 = cmulf(make_float2(c, sn), u);
                    r1 = cmulf(make_float2(c, -sn), v);
                } else if (g.kind == BK_H) {
                    const float h = 0.70710678118654752f;
                    r0 = make_float2(h * (u.x + v.x), h * (u.y + v.y));
                    r1 = make_float2(h * (u.x - v.x), h * (u.y - v.y));
                } else if (g.kind == BK_X) {
                    r0 = v; r1 = u;
                } else {                       // Y = [[0, -i], [i, 0]]
                    r0 = make_float2(v.y, -v.x);
                    r1 = make_float2(-u.y, u.x);
                }
                s[i0] = r0;
                s[i1] = r1;
            }
            break;
        }
        case BK_Z: {
            for (int i = threadIdx.x; i < (size >> 1); i += kBT) {
                const uint32_t x = insert0(i, g.a) | (1u << g.a);
                s[x] = make_float2(-s[x].x, -s[x].y);
            }
            break;
        }
        case BK_CZ: {
            const int lo = min(g.a, g.b), hi = max(g.a, g.b);
            for (int i = threadIdx.x; i < (size >> 2); i += kBT) {
                const uint32_t x = insert0(insert0(i, lo), hi) | (1u << g.a) | (1u << g.b);
                s[x] = make_float2(-s[x].x, -s[x].y);
            }
            break;
        }
        case BK_CNOT: {  // control b, target a
            const int lo = min(g.a, g.b), hi = max(g.a, g.b);
            for (int i = threadIdx.x; i < (size >> 2); i += kBT) {
                const uint32_t x = insert0(insert0(i, lo), hi) | (1u << g.b);
                const uint32_t y = x | (1u << g.a);
                const float2 u = s[x];
                s[x] = s[y];
                s[y] = u;
            }
            break;
        }
    }
}

// this thread's share of <lam|P|psi> for the rotation axis of g on local bit a (exact products,
// double-float sums)
__device__ void grad_local(const float2* sp, const float2* sl, int size, const BGate& g, DFAcc& re, DFAcc& im) {
    const int half = size >> 1;
    for (int i = threadIdx.x; i < half; i += kBT) {
        const uint32_t i0 = insert0(i, g.a), i1 = i0 | (1u << g.a);
        const float2 a = sp[i0], b = sp[i1], la = sl[i0], lb = sl[i1];
        // P psi on the pair: X -> (b, a); Y -> (-i b, i a); Z -> (a, -b)
        float2 p0, p1;
        if (g.kind == BK_RX) { p0 = b; p1 = a; }
        else if (g.kind == BK_RY) { p0 = make_float2(b.y, -b.x); p1 = make_float2(-a.y, a.x); }
        else { p0 = a; p1 = make_float2(-b.x, -b.y); }
        // conj(l) * p = (lx px + ly py) + i (lx py - ly px)
        df_add_prod(re, la.x, p0.x); df_add_prod(re, la.y, p0.y);
        df_add_prod(im, la.x, p0.y); df_add_prod(im, -la.y, p0.x);
        df_add_prod(re, lb.x, p1.x); df_add_prod(re, lb.y, p1.y);
        df_add_prod(im, lb.x, p1.y); df_add_prod(im, -lb.y, p1.x);
    }
}

__device__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = red[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // thread 0
}

__device__ __forceinline__ uint32_t chunk_addr(const BPass& P, uint32_t base, int l) {
    return base | P.tab_lo[l & 127] | P.tab_hi[l >> 7];
}

// address base of chunk c: deposit c into the non-local bits
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

__global__ void __launch_bounds__(kBT, 1) k_batch(const BatchDev B) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* sp = reinterpret_cast<float2*>(smem);
    float2* sl = sp + kChunk;
    __shared__ double red[32];
    __shared__ int s_item;
    float2* gpsi = B.ws + uint64_t(blockIdx.x) * 2 * B.ws_stride;
    float2* glam = gpsi + B.ws_stride;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = int(atomicAdd(B.counter, 1u));
        __syncthreads();
        const int w = s_item;
        if (w >= B.count) break;
        const BItem it = B.items[B.order[w]];
        const bool resident = it.n <= kLocal;
        const int size = resident ? (1 << it.n) : kChunk;
        const uint32_t N = 1u << it.n;
        for (int j = threadIdx.x; j < it.ngrad; j += kBT) B.grad[it.grad0 + j] = 0.0;
        // ---------------- forward sweep
        for (int p = it.p0; p < it.p1; p++) {
            const BPass& P = B.passes[p];
            const uint32_t nch = resident ? 1u : (N >> kLocal);
            for (uint32_t c = 0; c < nch; c++) {
                const uint32_t base = resident ? 0u : chunk_base(P.nonlocal, c);
                if (p == it.p0) {
                    for (int l = threadIdx.x; l < size; l += kBT)
                        sp[l] = make_float2((base == 0 && l == 0) ? 1.f : 0.f, 0.f);
                } else if (!resident) {
                    for (int l = threadIdx.x; l < size; l += kBT) sp[l] = gpsi[chunk_addr(P, base, l)];
                }
                __syncthreads();
                for (int gi = P.g0; gi < P.g1; gi++) {
                    const BGate g = B.gates[gi];
                    const float2 cs = g.slot >= 0 ? B.cs[it.angle0 + g.slot] : make_float2(1.f, 0.f);
                    apply_local(sp, size, g, cs, false);
                    __syncthreads();
                }
                if (!resident)
                    for (int l = threadIdx.x; l < size; l += kBT) gpsi[chunk_addr(B.passes[p], base, l)] = sp[l];
                __syncthreads();
            }
        }
        // ---------------- lambda = H psi, E = Re <psi|lambda>
        {
            DFAcc e;
            df_zero(e);
            const float2* src = resident ? sp : gpsi;
            float2* dst = resident ? sl : glam;
            for (uint32_t y = threadIdx.x; y < N; y += kBT) {
                double re = 0.0, im = 0.0;
                for (int t = it.t0; t < it.t1; t++) {
                    const BTerm T = B.terms[t];
                    const uint32_t y2 = y ^ T.xmask;
                    float2 v = src[y2];
                    v = mul_ipow(v, T.nY + 2 * (__popc(y2 & T.zmask) & 1));
                    re = fma(T.coef, double(v.x), re);
                    im = fma(T.coef, double(v.y), im);
                }
                const float2 lam = make_float2(float(re), float(im));
                dst[y] = lam;
                const float2 ps = src[y];
                df_add_prod(e, ps.x, lam.x);
                df_add_prod(e, ps.y, lam.y);
            }
            const double E = block_sum_d(df_value(e), red);
            if (threadIdx.x == 0) B.energy[B.order[w]] = E;
            __syncthreads();
        }
        if (!B.want_grad) continue;
        // ---------------- reverse sweep
        for (int p = it.p1 - 1; p >= it.p0; p--) {
            const BPass& P = B.passes[p];
            const uint32_t nch = resident ? 1u : (N >> kLocal);
            for (uint32_t c = 0; c < nch; c++) {
                const uint32_t base = resident ? 0u : chunk_base(P.nonlocal, c);
                if (!resident) {
                    for (int l = threadIdx.x; l < size; l += kBT) {
                        const uint32_t a = chunk_addr(P, base, l);
                        sp[l] = gpsi[a];
                        sl[l] = glam[a];
                    }
                }
                __syncthreads();
                for (int gi = P.g1 - 1; gi >= P.g0; gi--) {
                    const BGate g = B.gates[gi];
                    const float2 cs = g.slot >= 0 ? B.cs[it.angle0 + g.slot] : make_float2(1.f, 0.f);
                    if (g.grad >= 0) {
                        DFAcc re, im;
                        df_zero(re);
                        df_zero(im);
                        grad_local(sp, sl, size, g, re, im);
                        // dE/dtheta = -Im <lambda|P|psi>
                        const double v = block_sum_d(df_value(im), red);
                        if (threadIdx.x == 0) B.grad[it.grad0 + g.grad] -= v;
                        __syncthreads();
                    }
                    apply_local(sp, size, g, cs, true);
                    apply_local(sl, size, g, cs, true);
                    __syncthreads();
                }
                if (!resident) {
                    for (int l = threadIdx.x; l < size; l += kBT) {
                        const uint32_t a = chunk_addr(P, base, l);
                        gpsi[a] = sp[l];
                        glam[a] = sl[l];
                    }
                }
                __syncthreads();
            }
        }
    }
}

// (cos, sin) of theta/2 for every angle slot
__global__ void k_angles(const double* __restrict__ theta, float2* __restrict__ cs, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double s, c;
        sincos(0.5 * theta[i], &s, &c);
        cs[i] = make_float2(float(c), float(s));
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
    std::vector<qs::BGate> gates;
    std::vector<qs::BTerm> terms;
    std::vector<int32_t> angle_param;   // angle slot -> parameter index of its circuit (or -1)
    std::vector<double> angle_fixed;    // angle slot -> fixed angle (when not parametric)
    std::vector<int32_t> angle_item;    // angle slot -> item
    std::vector<int32_t> param0;        // item -> first parameter in the caller's theta array
    std::vector<int32_t> grad_of_item;  // item -> grad0
    // device buffers
    void* d_items = nullptr;
    void* d_order = nullptr;
    void* d_passes = nullptr;
    void* d_gates = nullptr;
    void* d_terms = nullptr;
    double* d_theta = nullptr;
    float2* d_cs = nullptr;
    float2* d_ws = nullptr;
    double* d_energy = nullptr;
    double* d_grad = nullptr;
    unsigned int* d_counter = nullptr;
    double* h_theta = nullptr;   // pinned
    double* h_energy = nullptr;  // pinned
    double* h_grad = nullptr;    // pinned
    int grid = 0;
    size_t smem = 0;
    uint64_t ws_stride = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    int device = 0;
};

namespace qs {
namespace {

// split one circuit into passes over windows of <= kLocal qubits
void plan_passes(const qs_circuit& c, const std::vector<BGate>& gl, const std::vector<uint32_t>& gmask,
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
        bp.g0 = int(b.gates.size());
        for (int gi : p.gates) {
            BGate g = gl[gi];
            g.a = local(g.a);
            if (g.kind == BK_CZ || g.kind == BK_CNOT) g.b = local(g.b);
            b.gates.push_back(g);
        }
        bp.g1 = int(b.gates.size());
        b.passes.push_back(bp);
    }
    it.p1 = int(b.passes.size());
}

void free_batch(qs_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    void* dev[] = {b->d_items, b->d_order, b->d_passes, b->d_gates, b->d_terms, b->d_theta,
                   b->d_cs, b->d_ws, b->d_energy, b->d_grad, b->d_counter};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (b->h_theta) cudaFreeHost(b->h_theta);
    if (b->h_energy) cudaFreeHost(b->h_energy);
    if (b->h_grad) cudaFreeHost(b->h_grad);
}

template <typename T>
void upload(void** d, const std::vector<T>& h) {
    const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    QS_TRY_CUDA(cudaMalloc(d, bytes));
    if (!h.empty()) QS_TRY_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// enqueue one batch evaluation on `st` (used directly and under graph capture)
void enqueue(qs_batch* b, cudaStream_t st) {
    QS_TRY_CUDA(cudaMemcpyAsync(b->d_theta, b->h_theta, sizeof(double) * std::max(1, b->total_angles),
                                cudaMemcpyHostToDevice, st));
    k_angles<<<std::max(1, std::min(1024, (b->total_angles + 255) / 256)), 256, 0, st>>>(b->d_theta, b->d_cs,
                                                                                          b->total_angles);
    QS_TRY_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st));
    BatchDev B;
    B.items = static_cast<const BItem*>(b->d_items);
    B.order = static_cast<const int32_t*>(b->d_order);
    B.passes = static_cast<const BPass*>(b->d_passes);
    B.gates = static_cast<const BGate*>(b->d_gates);
    B.terms = static_cast<const BTerm*>(b->d_terms);
    B.cs = b->d_cs;
    B.ws = b->d_ws;
    B.ws_stride = b->ws_stride;
    B.energy = b->d_energy;
    B.grad = b->d_grad;
    B.count = b->count;
    B.want_grad = 1;
    B.counter = b->d_counter;
    k_batch<<<b->grid, kBT, b->smem, st>>>(B);
    QS_TRY_CUDA(cudaGetLastError());
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
        QS_REQUIRE(c.n >= 1 && c.n <= kMaxBatchQubits, "batched circuits have 1..24 qubits");
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
        int slots = 0;
        for (int i = 0; i < c.n_gates; i++) {
            const qs_gate& g = c.gates[i];
            check_qubits(c.n, g.targets, g.m, g.controls, g.mc);
            BGate bg;
            std::memset(&bg, 0, sizeof(bg));
            bg.slot = -1;
            bg.grad = -1;
            bg.a = uint8_t(g.targets[0]);
            uint32_t m = 1u << g.targets[0];
            QS_REQUIRE(g.kind == QS_GATE_NAMED, "batched circuits take named gates only");
            switch (g.named) {
                case QS_NAMED_RX:
                case QS_NAMED_RY:
                case QS_NAMED_RZ:
                    QS_REQUIRE(g.mc == 0 && g.m == 1, "batched rotations act on one qubit, uncontrolled");
                    bg.kind = g.named == QS_NAMED_RX ? BK_RX : g.named == QS_NAMED_RY ? BK_RY : BK_RZ;
                    bg.slot = slots++;
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
        }
        plan_passes(c, gl, gm, *b, it);
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
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    QS_TRY_CUDA(cudaGetDevice(&b->device));
    int sms = 1;
    QS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, std::min(sms, count));
    b->smem = 2 * sizeof(float2) * kChunk;
    b->ws_stride = b->max_n > kLocal ? (uint64_t(1) << b->max_n) : 1;
    try {
        upload(&b->d_items, b->items);
        upload(&b->d_order, b->order);
        upload(&b->d_passes, b->passes);
        upload(&b->d_gates, b->gates);
        upload(&b->d_terms, b->terms);
        QS_TRY_CUDA(cudaMalloc(&b->d_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMalloc(&b->d_cs, sizeof(float2) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMalloc(&b->d_ws, sizeof(float2) * 2 * b->ws_stride * b->grid));
        QS_TRY_CUDA(cudaMalloc(&b->d_energy, sizeof(double) * count));
        QS_TRY_CUDA(cudaMalloc(&b->d_grad, sizeof(double) * std::max(1, b->total_grads)));
        QS_TRY_CUDA(cudaMalloc(&b->d_counter, sizeof(unsigned int)));
        QS_TRY_CUDA(cudaMallocHost(&b->h_theta, sizeof(double) * std::max(1, b->total_angles)));
        QS_TRY_CUDA(cudaMallocHost(&b->h_energy, sizeof(double) * count));
        QS_TRY_CUDA(cudaMallocHost(&b->h_grad, sizeof(double) * std::max(1, b->total_grads)));
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
    if (workspace_bytes) *workspace_bytes = sizeof(float2) * 2 * b->ws_stride * b->grid;
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
        if (!b->exec) {
            QS_TRY_CUDA(cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking));
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
    std::memcpy(energies, b->h_energy, sizeof(double) * b->count);
    if (b->total_grads) std::memcpy(grads, b->h_grad, sizeof(double) * b->total_grads);
    BATCH_END
}

qs_status qs_batch_destroy(qs_batch* b) {
    BATCH_BEGIN
    if (!b) return QS_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
    BATCH_END
}

}  // extern "C"
