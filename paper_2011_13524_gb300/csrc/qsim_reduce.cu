// Reductions over a state vector (Sec. 4.2.2 squared norm and inner product, Sec. 4.5
// Pauli-observable expectation and transition amplitude) and the out-of-place product
// lambda = O psi used by the adjoint gradient.
//
// Sums are deterministic: every block writes its partial sums to its own slot, and one
// block adds the slots in a fixed order. Accumulation is FP64 for both storage types;
// complex64 amplitudes are widened to double before they are multiplied.
//
// Expectation: the terms of O = sum_P alpha_P P are grouped by their flip mask f (the
// X-or-Y positions). Group f = 0 is diagonal: sum_y w(y) |psi_y|^2 with
// w(y) = sum_P alpha_P (-1)^{popcount(y & z_P)}. A group f != 0 visits each pair
// (y, y ^ f) once, with A = conj(psi_{y^f}) psi_y:
//   <psi|P|psi> restricted to the pair = i^{#Y} (s(y) A + s(y^f) conj(A)).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

#include "qsim_arith.cuh"

namespace qs {

namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxTermsPerLaunch = 48;
static_assert(kHeavyChunkTerms <= kMaxTermsPerLaunch, "heavy chunks must fit one launch");

int sms() { return device_sms(); }

unsigned red_grid(uint64_t work) {
    const uint64_t want = (work + kRedThreads * 4 - 1) / (kRedThreads * 4);
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(sms()) * 4)));
}

// Block partial of (re, im) pairs into part[2*blockIdx.x + {0,1}].
__device__ __forceinline__ void write_partial2(double re, double im, double* part) {
    __shared__ double sh[kRedThreads / 32];
    const double r = block_sum<kRedThreads>(re, sh);
    const double i = block_sum<kRedThreads>(im, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r;
        part[2 * blockIdx.x + 1] = i;
    }
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const C* __restrict__ psi, uint64_t N, double* part) {
    double acc = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < N; x += stride) {
        const double2 v = widen(psi[x]);
        acc = fma(v.x, v.x, acc);
        acc = fma(v.y, v.y, acc);
    }
    write_partial2(acc, 0.0, part);
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_inner(const C* __restrict__ a, const C* __restrict__ b, uint64_t N,
                                                       double* part) {
    double re = 0.0, im = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < N; x += stride) {
        const double2 u = widen(a[x]), v = widen(b[x]);
        re = fma(u.x, v.x, re);
        re = fma(u.y, v.y, re);
        im = fma(u.x, v.y, im);
        im = fma(-u.y, v.x, im);
    }
    write_partial2(re, im, part);
}

struct TermParams {
    uint64_t xmask;          // group flip mask
    IndexPlan ip;            // pivot bit inserted (f != 0) or plain range (f == 0)
    int32_t nterms;
    double coef[kMaxTermsPerLaunch];
    uint64_t zmask[kMaxTermsPerLaunch];
    int32_t nY[kMaxTermsPerLaunch];
};

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_expect_group(const C* __restrict__ psi,
                                                              const __grid_constant__ TermParams P, double* part) {
    double re = 0.0, im = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.ip.n_iter; i += stride) {
        const uint64_t y = expand(i, P.ip);
        if (P.xmask == 0) {
            const double2 v = widen(psi[y]);
            const double p = fma(v.x, v.x, v.y * v.y);
            double w = 0.0;
            for (int t = 0; t < P.nterms; t++) w += parity64(y & P.zmask[t]) ? -P.coef[t] : P.coef[t];
            re = fma(w, p, re);
        } else {
            const uint64_t y2 = y ^ P.xmask;
            const double2 a = widen(psi[y]), b = widen(psi[y2]);
            const double Ar = fma(b.x, a.x, b.y * a.y);   // A = conj(b) a
            const double Ai = fma(b.x, a.y, -b.y * a.x);
            for (int t = 0; t < P.nterms; t++) {
                const int s1 = parity64(y & P.zmask[t]);
                const int s2 = parity64(y2 & P.zmask[t]);
                // s1 A + s2 conj(A): equal signs -> 2 s Re A ; opposite -> 2 i s Im A
                double ur, ui;
                const double sg = s1 ? -2.0 : 2.0;
                if (s1 == s2) { ur = sg * Ar; ui = 0.0; } else { ur = 0.0; ui = sg * Ai; }
                double vr, vi;  // multiply by i^{nY}
                switch (P.nY[t] & 3) {
                    case 0: vr = ur; vi = ui; break;
                    case 1: vr = -ui; vi = ur; break;
                    case 2: vr = -ur; vi = -ui; break;
                    default: vr = ui; vi = -ur; break;
                }
                re = fma(P.coef[t], vr, re);
                im = fma(P.coef[t], vi, im);
            }
        }
    }
    write_partial2(re, im, part);
}

// <lam| P |psi> = sum_y conj(lam_y) i^{#Y} s(y ^ f) psi_{y ^ f}
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_transition(const C* __restrict__ lam, const C* __restrict__ psi,
                                                            uint64_t N, uint64_t xmask, uint64_t zmask, int nY,
                                                            double* part) {
    double re = 0.0, im = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; y < N; y += stride) {
        const uint64_t y2 = y ^ xmask;
        const double2 l = widen(lam[y]);
        double2 p = widen(psi[y2]);
        p = mul_ipow(p, nY + 2 * parity64(y2 & zmask));
        re = fma(l.x, p.x, re);
        re = fma(l.y, p.y, re);
        im = fma(l.x, p.y, im);
        im = fma(-l.y, p.x, im);
    }
    write_partial2(re, im, part);
}

// <bra| sum_t coef_t P_t |ket> over the terms of one flip group: sum_y conj(bra_y) coef_t i^nY_t
// (-1)^popc(x & z_t) ket_x with x = y ^ xmask (P_t |x> lands on |y>)
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_transition_group(const C* __restrict__ bra, const C* __restrict__ ket,
                                                                  uint64_t N, const __grid_constant__ TermParams P,
                                                                  double* part) {
    double re = 0.0, im = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; y < N; y += stride) {
        const uint64_t x = y ^ P.xmask;
        const double2 b = widen(bra[y]), k = widen(ket[x]);
        const double vr = fma(b.x, k.x, b.y * k.y), vi = fma(b.x, k.y, -b.y * k.x);  // conj(b) k
        for (int t = 0; t < P.nterms; t++) {
            const double w = parity64(x & P.zmask[t]) ? -P.coef[t] : P.coef[t];
            const double ur = w * vr, ui = w * vi;
            switch (P.nY[t] & 3) {
                case 0: re += ur; im += ui; break;
                case 1: re -= ui; im += ur; break;
                case 2: re -= ur; im -= ui; break;
                default: re += ui; im -= ur; break;
            }
        }
    }
    write_partial2(re, im, part);
}

// sum of |psi_x|^2 over the x whose measured bits are fixed: i runs over the free qubits, its
// bits deposited at their positions, the measured ones set from `set`
struct FreeBits {
    uint64_t set;
    int32_t nfree;
    int8_t pos[64];
};
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_norm2_sub(const C* __restrict__ psi, const __grid_constant__ FreeBits F,
                                                           double* part) {
    double acc = 0.0;
    const uint64_t n_iter = 1ull << F.nfree;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_iter; i += stride) {
        uint64_t x = F.set;
        for (int j = 0; j < F.nfree; j++) x |= ((i >> j) & 1ull) << F.pos[j];
        const double2 v = widen(psi[x]);
        acc = fma(v.x, v.x, acc);
        acc = fma(v.y, v.y, acc);
    }
    write_partial2(acc, 0.0, part);
}

// sampling, step 1: probability mass of each chunk of 2^chunk_log amplitudes (one block each)
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_chunk_mass(const C* __restrict__ psi, uint64_t N, int chunk_log,
                                                            double* mass) {
    const uint64_t base = uint64_t(blockIdx.x) << chunk_log;
    const uint64_t end = N < base + (1ull << chunk_log) ? N : base + (1ull << chunk_log);
    double acc = 0.0;
    for (uint64_t x = base + threadIdx.x; x < end; x += blockDim.x) {
        const double2 v = widen(psi[x]);
        acc = fma(v.x, v.x, acc);
        acc = fma(v.y, v.y, acc);
    }
    __shared__ double sh[kRedThreads / 32];
    const double r = block_sum<kRedThreads>(acc, sh);
    if (threadIdx.x == 0) mass[blockIdx.x] = r;
}

// sampling, step 2: one warp per sample finds, inside its chunk, the first x whose running mass
// (lanes own consecutive stretches, summed in order) exceeds the residual target
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_sample_find(const C* __restrict__ psi, uint64_t N, int chunk_log,
                                                             const uint64_t* __restrict__ chunk,
                                                             const double* __restrict__ resid, int count,
                                                             uint64_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int s = int((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (s >= count) return;
    const uint64_t base = chunk[s] << chunk_log;
    const uint64_t len = N - base < (1ull << chunk_log) ? N - base : (1ull << chunk_log);
    const uint64_t per = (len + 31) / 32;
    const uint64_t lo = len < uint64_t(lane) * per ? len : uint64_t(lane) * per;
    const uint64_t hi = len < lo + per ? len : lo + per;
    auto mass = [&](uint64_t x) {
        const double2 v = widen(psi[base + x]);
        return fma(v.x, v.x, v.y * v.y);
    };
    double own = 0.0;
    for (uint64_t x = lo; x < hi; x++) own += mass(x);
    double incl = own;  // inclusive scan over lanes, in lane order
    for (int d = 1; d < 32; d <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const double r = resid[s];
    const unsigned over = __ballot_sync(0xffffffffu, incl > r);
    const unsigned nonzero = __ballot_sync(0xffffffffu, own > 0.0);
    // the lane whose stretch crosses r; past the end (rounding) the last lane with mass
    const int L = over ? __ffs(over) - 1 : (nonzero ? 31 - __clz(nonzero) : 31);
    if (lane == L) {
        double acc = incl - own;
        uint64_t pick = hi > lo ? hi - 1 : lo, last = pick;
        bool found = false;
        for (uint64_t x = lo; x < hi; x++) {
            const double m = mass(x);
            if (m > 0.0) last = x;
            acc += m;
            if (acc > r) {
                pick = x;
                found = true;
                break;
            }
        }
        out[s] = base + (found ? pick : last);
    }
}

// sum of `nslots` (re, im) partials in a fixed order -> out[0..1]
__global__ void __launch_bounds__(kRedThreads) k_final2(const double* __restrict__ part, int nslots, double* out) {
    __shared__ double sh[kRedThreads / 32];
    double re = 0.0, im = 0.0;
    for (int j = threadIdx.x; j < nslots; j += kRedThreads) {
        re += part[2 * j];
        im += part[2 * j + 1];
    }
    const double r = block_sum<kRedThreads>(re, sh);
    const double i = block_sum<kRedThreads>(im, sh);
    if (threadIdx.x == 0) {
        out[0] = r;
        out[1] = i;
    }
}

// lambda_y = sum_groups sum_terms coef * i^{#Y} s(y ^ f) psi_{y ^ f}
struct ObsDevTerm {
    uint64_t xmask, zmask;
    double coef;
    int32_t nY, pad;
};

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_apply_obs(const C* __restrict__ psi, C* __restrict__ lam, uint64_t N,
                                                           const ObsDevTerm* __restrict__ terms, int nterms) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; y < N; y += stride) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < nterms; t++) {
            const ObsDevTerm T = terms[t];
            const uint64_t y2 = y ^ T.xmask;
            double2 p = widen(psi[y2]);
            p = mul_ipow(p, T.nY + 2 * parity64(y2 & T.zmask));
            re = fma(T.coef, p.x, re);
            im = fma(T.coef, p.y, im);
        }
        lam[y] = narrow<C>(re, im);
    }
}

// double-float states: the same sum in double-float arithmetic on the FP32 pipes (exact
// products with the split coefficient, compensated sums)
struct ObsDevTermDF {
    uint64_t xmask, zmask;
    float ch, cl;  // coefficient = ch + cl
    int32_t nY, pad;
};

__global__ void __launch_bounds__(kRedThreads) k_apply_obs_df(const float4* __restrict__ psi, float4* __restrict__ lam,
                                                              uint64_t N, const ObsDevTermDF* __restrict__ terms,
                                                              int nterms) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; y < N; y += stride) {
        DFArith::Acc a = DFArith::zero();
        for (int t = 0; t < nterms; t++) {
            const ObsDevTermDF T = terms[t];
            const uint64_t y2 = y ^ T.xmask;
            const float4 v = DFArith::ipow(psi[y2], T.nY + 2 * parity64(y2 & T.zmask));
            DFArith::dprod(a.rs, a.rc, T.ch, T.cl, v.x, v.y);
            DFArith::dprod(a.is, a.ic, T.ch, T.cl, v.z, v.w);
        }
        lam[y] = DFArith::out(a);
    }
}

// ---------------------------------------------------------------- host side
// calls f(C*) with the state's buffer typed by its arithmetic layout
template <typename F>
void with_type(Arith ar, const void* p, F&& f) {
    switch (ar) {
        case Arith::F32: f(reinterpret_cast<const float2*>(p)); break;
        case Arith::F64: f(reinterpret_cast<const double2*>(p)); break;
        case Arith::DF: f(reinterpret_cast<const float4*>(p)); break;
    }
}
void ensure_scratch(qs_state* s, size_t part_doubles) {
    Scratch& sc = s->scratch;
    if (sc.part_cap < part_doubles) {
        if (sc.d_part) {
            QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
            dev_free(sc.d_part);
            sc.d_part = nullptr;
            sc.part_cap = 0;
        }
        QS_TRY_CUDA(dev_malloc(&sc.d_part, part_doubles * sizeof(double)));
        sc.part_cap = part_doubles;
    }
    if (!sc.h_out) {
        QS_TRY_CUDA(host_malloc_pinned(&sc.h_out, 16 * sizeof(double)));
        sc.out_cap = 16;
    }
}

// final reduce of nslots partials into d_part[out_off..], copy 2 doubles to host, sync
void finish2(qs_state* s, int nslots, double out[2]) {
    double* d_out = s->scratch.d_part + s->scratch.part_cap - 2;
    k_final2<<<1, kRedThreads, 0, s->stream>>>(s->scratch.d_part, nslots, d_out);
    QS_TRY_CUDA(cudaGetLastError());
    QS_TRY_CUDA(cudaMemcpyAsync(s->scratch.h_out, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = s->scratch.h_out[0];
    out[1] = s->scratch.h_out[1];
}

}  // namespace

std::vector<PauliGroup> group_observable(const qs_pauli_obs* obs, int n) {
    QS_REQUIRE(obs != nullptr, "null observable");
    QS_REQUIRE(obs->n_terms >= 0, "negative term count");
    QS_REQUIRE(obs->n_terms == 0 || (obs->coef && obs->x_mask && obs->z_mask), "null observable arrays");
    const uint64_t lim = n >= 64 ? ~0ull : ((1ull << n) - 1);
    std::map<uint64_t, size_t> idx;
    std::vector<PauliGroup> groups;
    for (int t = 0; t < obs->n_terms; t++) {
        QS_REQUIRE((obs->x_mask[t] & ~lim) == 0 && (obs->z_mask[t] & ~lim) == 0, "Pauli term acts on a qubit >= n");
        auto it = idx.find(obs->x_mask[t]);
        if (it == idx.end()) {
            idx[obs->x_mask[t]] = groups.size();
            groups.push_back(PauliGroup{obs->x_mask[t], {}, {}});
            it = idx.find(obs->x_mask[t]);
        }
        groups[it->second].coef.push_back(obs->coef[t]);
        groups[it->second].zmask.push_back(obs->z_mask[t]);
    }
    return groups;
}

void reduce_norm2(qs_state* s, double* out) {
    const uint64_t N = 1ull << s->n;
    const unsigned g = red_grid(N);
    ensure_scratch(s, 2 * g + 2);
    with_type(arith_of(s), s->data, [&](auto p) { k_norm2<<<g, kRedThreads, 0, s->stream>>>(p, N, s->scratch.d_part); });
    QS_TRY_CUDA(cudaGetLastError());
    double r[2];
    finish2(s, int(g), r);
    *out = r[0];
}

void reduce_inner(const qs_state* a, const qs_state* b, double out[2]) {
    qs_state* s = const_cast<qs_state*>(a);
    const uint64_t N = 1ull << s->n;
    const unsigned g = red_grid(N);
    ensure_scratch(s, 2 * g + 2);
    if (b->stream != s->stream) {
        // order b's pending work before the read on a's stream
        QS_TRY_CUDA(cudaStreamSynchronize(b->stream));
    }
    QS_REQUIRE(arith_of(a) == arith_of(b), "states in different layouts");
    with_type(arith_of(a), a->data, [&](auto pa) {
        using CP = decltype(pa);
        k_inner<<<g, kRedThreads, 0, s->stream>>>(pa, reinterpret_cast<CP>(b->data), N, s->scratch.d_part);
    });
    QS_TRY_CUDA(cudaGetLastError());
    finish2(s, int(g), out);
}

// Launches of one expectation: the tile passes, then one launch per heavy chunk. With a cap on
// the block partials the grids shrink proportionally (the kernels loop over their work).
struct ExpectLaunches {
    std::vector<unsigned> pass_grid, heavy_grid;  // a diagonal observable: its one streaming pass in pass_grid
    size_t slots = 0;
};
ExpectLaunches expectation_launches(const ExpectPlan& plan, int n, Arith ar, size_t cap) {
    ExpectLaunches L;
    if (plan.diag) L.pass_grid.push_back(expect_diag_grid(n, ar));
    for (const TileParams& P : plan.passes) L.pass_grid.push_back(expect_pass_grid(P, ar));
    for (const HeavyChunk& h : plan.heavy) L.heavy_grid.push_back(red_grid((1ull << n) >> (h.g->xmask ? 1 : 0)));
    size_t tot = 0;
    for (unsigned g : L.pass_grid) tot += g;
    for (unsigned g : L.heavy_grid) tot += g;
    if (tot > cap) {
        const size_t nl = L.pass_grid.size() + L.heavy_grid.size();
        QS_REQUIRE(nl <= cap, "observable needs more kernel launches than the partial-sum scratch holds");
        const size_t per = cap / nl;
        for (unsigned& g : L.pass_grid) g = unsigned(std::min<size_t>(g, per));
        for (unsigned& g : L.heavy_grid) g = unsigned(std::min<size_t>(g, per));
    }
    for (unsigned g : L.pass_grid) L.slots += g;
    for (unsigned g : L.heavy_grid) L.slots += g;
    return L;
}

void launch_expectation(const ExpectPlan& plan, const ExpectLaunches& L, const void* psi, int n, Arith ar,
                        cudaStream_t st, double* part) {
    size_t slots = 0;
    if (plan.diag) {
        launch_expect_diag(plan.dp, psi, ar, part, L.pass_grid[0], st);
        return;
    }
    for (size_t p = 0; p < plan.passes.size(); p++) {
        launch_expect_pass(plan.passes[p], psi, ar, part + 2 * slots, L.pass_grid[p], st);
        slots += L.pass_grid[p];
    }
    for (size_t h = 0; h < plan.heavy.size(); h++) {
        const HeavyChunk& c = plan.heavy[h];
        TermParams P;
        P.xmask = c.g->xmask;
        std::vector<int> fixed;
        if (P.xmask) fixed.push_back(__builtin_ctzll(P.xmask));
        P.ip = make_index_plan(n, fixed, 0);
        P.nterms = int(c.t1 - c.t0);
        for (size_t t = c.t0; t < c.t1; t++) {
            P.coef[t - c.t0] = c.g->coef[t];
            P.zmask[t - c.t0] = c.g->zmask[t];
            P.nY[t - c.t0] = __builtin_popcountll(c.g->xmask & c.g->zmask[t]);
        }
        with_type(ar, psi, [&](auto p) { k_expect_group<<<L.heavy_grid[h], kRedThreads, 0, st>>>(p, P, part + 2 * slots); });
        QS_TRY_CUDA(cudaGetLastError());
        slots += L.heavy_grid[h];
    }
}

void reduce_expectation(qs_state* s, const qs_pauli_obs* obs, double out[2]) {
    const std::vector<PauliGroup> groups = group_observable(obs, s->n);
    if (groups.empty()) {
        out[0] = out[1] = 0.0;
        return;
    }
    const ExpectPlan plan = plan_expectation(groups, s->n);
    const ExpectLaunches L = expectation_launches(plan, s->n, arith_of(s), size_t(1) << 40);
    ensure_scratch(s, 2 * L.slots + 2);
    launch_expectation(plan, L, s->data, s->n, arith_of(s), s->stream, s->scratch.d_part);
    finish2(s, int(L.slots), out);
}

void reduce_pauli_transition(qs_state* lam, const qs_state* psi, uint64_t xmask, uint64_t zmask, double out[2]) {
    const uint64_t N = 1ull << lam->n;
    const unsigned g = red_grid(N);
    ensure_scratch(lam, 2 * g + 2);
    const int nY = __builtin_popcountll(xmask & zmask);
    QS_REQUIRE(arith_of(lam) == arith_of(psi), "states in different layouts");
    with_type(arith_of(lam), lam->data, [&](auto pl) {
        using CP = decltype(pl);
        k_transition<<<g, kRedThreads, 0, lam->stream>>>(pl, reinterpret_cast<CP>(psi->data), N, xmask, zmask, nY,
                                                         lam->scratch.d_part);
    });
    QS_TRY_CUDA(cudaGetLastError());
    finish2(lam, int(g), out);
}

void reduce_transition(const qs_state* bra, const qs_pauli_obs* obs, const qs_state* ket, double out[2]) {
    qs_state* s = const_cast<qs_state*>(bra);
    const std::vector<PauliGroup> groups = group_observable(obs, s->n);
    const uint64_t N = 1ull << s->n;
    QS_REQUIRE(arith_of(bra) == arith_of(ket), "states in different layouts");
    if (ket->stream != s->stream) QS_TRY_CUDA(cudaStreamSynchronize(ket->stream));
    if (groups.empty()) {
        out[0] = out[1] = 0.0;
        return;
    }
    const Arith ar = arith_of(s);
    const ExpectPlan plan = plan_transition(groups, s->n);
    std::vector<unsigned> grids;
    size_t slots_needed = 0;
    for (const TileParams& P : plan.passes) {
        grids.push_back(trans_pass_grid(P, ar));
        slots_needed += grids.back();
    }
    const unsigned gr = red_grid(N);
    slots_needed += size_t(gr) * plan.heavy.size();
    ensure_scratch(s, 2 * slots_needed + 2);
    size_t slots = 0;
    for (size_t p = 0; p < plan.passes.size(); p++) {
        launch_transition_pass(plan.passes[p], bra->data, ket->data, ar, s->scratch.d_part + 2 * slots, grids[p],
                               s->stream);
        slots += grids[p];
    }
    // flip groups wider than a tile: one pass each
    for (const HeavyChunk& c : plan.heavy) {
        TermParams P;
        P.xmask = c.g->xmask;
        P.ip = make_index_plan(s->n, {}, 0);
        P.nterms = int(c.t1 - c.t0);
        for (size_t t = c.t0; t < c.t1; t++) {
            P.coef[t - c.t0] = c.g->coef[t];
            P.zmask[t - c.t0] = c.g->zmask[t];
            P.nY[t - c.t0] = __builtin_popcountll(c.g->xmask & c.g->zmask[t]);
        }
        double* part = s->scratch.d_part + 2 * slots;
        with_type(ar, s->data, [&](auto pb) {
            using CP = decltype(pb);
            k_transition_group<<<gr, kRedThreads, 0, s->stream>>>(pb, reinterpret_cast<CP>(ket->data), N, P, part);
        });
        QS_TRY_CUDA(cudaGetLastError());
        slots += gr;
    }
    finish2(s, int(slots), out);
}

void reduce_marginal(const qs_state* st, const int32_t* measured, double* out) {
    qs_state* s = const_cast<qs_state*>(st);
    FreeBits F;
    F.set = 0;
    F.nfree = 0;
    for (int q = 0; q < s->n; q++) {
        QS_REQUIRE(measured[q] >= 0 && measured[q] <= 2, "measured values must be 0, 1 or 2 (any)");
        if (measured[q] == 2) F.pos[F.nfree++] = int8_t(q);
        else if (measured[q] == 1) F.set |= 1ull << q;
    }
    const uint64_t work = 1ull << F.nfree;
    const unsigned g = red_grid(work);
    ensure_scratch(s, 2 * g + 2);
    with_type(arith_of(s), s->data, [&](auto p) { k_norm2_sub<<<g, kRedThreads, 0, s->stream>>>(p, F, s->scratch.d_part); });
    QS_TRY_CUDA(cudaGetLastError());
    double r[2];
    finish2(s, int(g), r);
    *out = r[0];
}

void sample_state(const qs_state* st, int count, const double* uniforms, uint64_t* out) {
    qs_state* s = const_cast<qs_state*>(st);
    if (count == 0) return;
    for (int k = 0; k < count; k++) QS_REQUIRE(uniforms[k] >= 0.0 && uniforms[k] < 1.0, "uniforms must lie in [0, 1)");
    const uint64_t N = 1ull << s->n;
    const int chunk_log = std::min(s->n, 12);
    const uint64_t B = N >> chunk_log;
    double* d_mass = nullptr;
    uint64_t* d_chunk = nullptr;
    double* d_resid = nullptr;
    uint64_t* d_out = nullptr;
    auto cleanup = [&]() {
        if (d_mass) dev_free_async(d_mass, s->stream);
        if (d_chunk) dev_free_async(d_chunk, s->stream);
        if (d_resid) dev_free_async(d_resid, s->stream);
        if (d_out) dev_free_async(d_out, s->stream);
    };
    try {
        QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_mass), B * sizeof(double), s->stream));
        with_type(arith_of(s), s->data, [&](auto p) {
            k_chunk_mass<<<unsigned(B), kRedThreads, 0, s->stream>>>(p, N, chunk_log, d_mass);
        });
        QS_TRY_CUDA(cudaGetLastError());
        // cumulative distribution over chunks, in order, on the host
        std::vector<double> mass(B), cum(B + 1, 0.0);
        QS_TRY_CUDA(cudaMemcpyAsync(mass.data(), d_mass, B * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
        for (uint64_t b = 0; b < B; b++) cum[b + 1] = cum[b] + mass[b];
        const double total = cum[B];
        if (!(total > 0.0)) throw Error{QS_ERR_NUMERIC, "sampling a zero state"};
        std::vector<uint64_t> chunk(count);
        std::vector<double> resid(count);
        for (int k = 0; k < count; k++) {
            const double target = uniforms[k] * total;
            // first chunk whose cumulative mass exceeds the target
            uint64_t c = uint64_t(std::upper_bound(cum.begin() + 1, cum.end(), target) - (cum.begin() + 1));
            if (c >= B) {  // rounding at the top: the last chunk with mass
                c = B - 1;
                while (c > 0 && !(mass[c] > 0.0)) c--;
            }
            chunk[k] = c;
            resid[k] = target - cum[c];
        }
        QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_chunk), count * sizeof(uint64_t), s->stream));
        QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_resid), count * sizeof(double), s->stream));
        QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_out), count * sizeof(uint64_t), s->stream));
        QS_TRY_CUDA(cudaMemcpyAsync(d_chunk, chunk.data(), count * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream));
        QS_TRY_CUDA(cudaMemcpyAsync(d_resid, resid.data(), count * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        const unsigned blocks = unsigned((uint64_t(count) * 32 + kRedThreads - 1) / kRedThreads);
        with_type(arith_of(s), s->data, [&](auto p) {
            k_sample_find<<<blocks, kRedThreads, 0, s->stream>>>(p, N, chunk_log, d_chunk, d_resid, count, d_out);
        });
        QS_TRY_CUDA(cudaGetLastError());
        QS_TRY_CUDA(cudaMemcpyAsync(out, d_out, count * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
        QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void launch_apply_observable(const std::vector<PauliGroup>& groups, const void* psi, void* lam, int n, Arith ar,
                             cudaStream_t st) {
    std::vector<ObsDevTerm> terms;
    for (const auto& g : groups)
        for (size_t t = 0; t < g.coef.size(); t++)
            terms.push_back(ObsDevTerm{g.xmask, g.zmask[t], g.coef[t], __builtin_popcountll(g.xmask & g.zmask[t]), 0});
    const uint64_t N = 1ull << n;
    if (terms.empty()) {
        QS_TRY_CUDA(cudaMemsetAsync(lam, 0, N * (ar == Arith::F32 ? 8 : 16), st));
        return;
    }
    ObsDevTerm* d_terms = nullptr;
    QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_terms), terms.size() * sizeof(ObsDevTerm), st));
    QS_TRY_CUDA(cudaMemcpyAsync(d_terms, terms.data(), terms.size() * sizeof(ObsDevTerm), cudaMemcpyHostToDevice, st));
    const unsigned g = red_grid(N);
    if (ar == Arith::DF) {
        std::vector<ObsDevTermDF> tdf(terms.size());
        for (size_t t = 0; t < terms.size(); t++) {
            tdf[t].xmask = terms[t].xmask;
            tdf[t].zmask = terms[t].zmask;
            split_double(terms[t].coef, tdf[t].ch, tdf[t].cl);
            tdf[t].nY = terms[t].nY;
            tdf[t].pad = 0;
        }
        static_assert(sizeof(ObsDevTermDF) <= sizeof(ObsDevTerm), "the term buffer holds either form");
        QS_TRY_CUDA(cudaMemcpyAsync(d_terms, tdf.data(), tdf.size() * sizeof(ObsDevTermDF), cudaMemcpyHostToDevice, st));
        QS_TRY_CUDA(cudaStreamSynchronize(st));  // tdf is host memory that dies on return
        k_apply_obs_df<<<g, kRedThreads, 0, st>>>(static_cast<const float4*>(psi), static_cast<float4*>(lam), N,
                                                  reinterpret_cast<const ObsDevTermDF*>(d_terms), int(terms.size()));
    } else {
        with_type(ar, psi, [&](auto pp) {
            using C = std::remove_const_t<std::remove_pointer_t<decltype(pp)>>;
            k_apply_obs<<<g, kRedThreads, 0, st>>>(pp, reinterpret_cast<C*>(lam), N, d_terms, int(terms.size()));
        });
    }
    QS_TRY_CUDA(cudaGetLastError());
    QS_TRY_CUDA(dev_free_async(d_terms, st));
}

}  // namespace qs

// ---------------------------------------------------------------- allocation-free variant
// Scratch for qs_expectation_noalloc: the per-block partial sums live in this fixed array
// instead of memory the library allocates. Every GPU that loads the library holds it (512 KiB)
// until the process exits. Host code may not use the symbol as a pointer; the device address
// is looked up once per device with cudaGetSymbolAddress.
namespace qs {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 16;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (set up on first use there)
double* noalloc_scratch() {
    int dev = 0;
    QS_TRY_CUDA(cudaGetDevice(&dev));
    QS_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        QS_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    return g_noalloc_ptr[dev];
}
}  // namespace

size_t noalloc_scratch_doubles() { return kNoAllocScratchDoubles; }

void expectation_noalloc(const void* psi, int n, qs_dtype dt, cudaStream_t st, const qs_pauli_obs* obs,
                         double out[2]) {
    QS_REQUIRE(psi != nullptr, "null state pointer");
    QS_REQUIRE((reinterpret_cast<uintptr_t>(psi) & 15) == 0, "state pointer must be 16-byte aligned");
    QS_REQUIRE(n >= 1 && n <= QS_MAX_QUBITS, "qubit count out of range (1..34)");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    QS_REQUIRE(obs != nullptr && out != nullptr, "null observable or output");
    QS_REQUIRE(obs->n_terms >= 0, "negative term count");
    QS_REQUIRE(obs->n_terms == 0 || (obs->coef && obs->x_mask && obs->z_mask), "null observable arrays");
    const std::vector<PauliGroup> groups = group_observable(obs, n);
    if (groups.empty()) {
        out[0] = out[1] = 0.0;
        return;
    }
    const Arith ar = dt == QS_C64 ? Arith::F32 : Arith::F64;
    const ExpectPlan plan = plan_expectation(groups, n);
    // 2 doubles per block partial, plus the 2 final values at the end of the array
    const ExpectLaunches L = expectation_launches(plan, n, ar, (kNoAllocScratchDoubles - 2) / 2);
    double* scratch = noalloc_scratch();
    double* d_out = scratch + kNoAllocScratchDoubles - 2;
    launch_expectation(plan, L, psi, n, ar, st, scratch);
    const int slots = int(L.slots);
    k_final2<<<1, kRedThreads, 0, st>>>(scratch, slots, d_out);
    QS_TRY_CUDA(cudaGetLastError());
    QS_TRY_CUDA(cudaMemcpyAsync(out, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    QS_TRY_CUDA(cudaStreamSynchronize(st));
}

}  // namespace qs
