// Internal declarations shared by the translation units of libqsim_gb300.so.
// Host-side structures, launch parameter blocks passed by value to kernels, and
// the error helpers behind qs_last_error().
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qsim_gb300.h"

namespace qs {

using cplx = std::complex<double>;

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();

struct Error {
    qs_status code;
    std::string msg;
};

#define QS_TRY_CUDA(expr)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            throw ::qs::Error{e_ == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA, \
                              std::string(#expr) + ": " + cudaGetErrorString(e_)};        \
        }                                                                                 \
    } while (0)

#define QS_REQUIRE(cond, msg)                                  \
    do {                                                       \
        if (!(cond)) throw ::qs::Error{QS_ERR_INVALID_ARG, msg}; \
    } while (0)

// ------------------------------------------------------------------ state
struct Scratch {
    // Per-state reduction scratch: per-block partial sums (device) and a pinned
    // host landing area for the final values.
    double* d_part = nullptr;
    size_t part_cap = 0;  // doubles
    double* h_out = nullptr;
    size_t out_cap = 0;   // doubles
};

}  // namespace qs

struct qs_state {
    int n = 0;
    qs_dtype dt = QS_C128;
    void* data = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    qs::Scratch scratch;
    void* d_stage = nullptr;  // kStageBytes, allocated on first wide dense gate
    int df = 0;               // 1 while a complex128 buffer holds the double-float layout
    int math = -1;            // QS_MATH_* of this state, -1: the process-wide setting
    int tensor = -1;          // QS_TENSOR_* bits of this state, -1: the process-wide setting
};

namespace qs {

inline size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

// ------------------------------------------------------------------ allocations
// Every device and pinned-host allocation of the library goes through these: they count the
// allocations held, and a test hook can make one of them fail as if memory had run out
// (cudaErrorMemoryAllocation, reported as QS_ERR_OOM), to check that no call leaks on that path.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t st);
cudaError_t host_malloc_pinned_raw(void** p, size_t bytes);
cudaError_t dev_free(void* p);
cudaError_t dev_free_async(void* p, cudaStream_t st);
cudaError_t host_free_pinned(void* p);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) { return dev_malloc_raw(reinterpret_cast<void**>(p), bytes); }
template <typename T>
cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t st) {
    return dev_malloc_async_raw(reinterpret_cast<void**>(p), bytes, st);
}
template <typename T>
cudaError_t host_malloc_pinned(T** p, size_t bytes) { return host_malloc_pinned_raw(reinterpret_cast<void**>(p), bytes); }
// test hook: the allocation after `after` more successful ones fails (-1: none); allocations held
void set_alloc_failure(long long after);
long long allocations_held();

// ------------------------------------------------------------------ per-device setup
constexpr int kMaxDevices = 64;
// index of the current device (QS_ERR_INVALID_ARG beyond kMaxDevices)
int current_device();
// SM count of the current device, looked up once per device; thread-safe
int device_sms();
// Runs a setup step once for each device, with that device current: function attributes such
// as a raised shared-memory limit belong to the device context they were set in. Thread-safe.
class PerDevice {
  public:
    template <typename F>
    void once(F&& f) {
        const int dev = current_device();
        std::lock_guard<std::mutex> lk(mu_);
        if (!((done_ >> dev) & 1ull)) {
            f(dev);
            done_ |= 1ull << dev;
        }
    }

  private:
    std::mutex mu_;
    uint64_t done_ = 0;
};

// ------------------------------------------------------------------ launch plans
// Enumeration of the x0 of Eq. (update_mat): iteration index i -> bit string with zero
// bits inserted at every fixed position (targets and controls), then the control bits
// that must be 1 or'ed in.
constexpr int kMaxFixed = QS_MAX_TARGETS + QS_MAX_CONTROLS + 2;
struct IndexPlan {
    uint64_t n_iter = 0;
    uint64_t setmask = 0;
    int32_t nfix = 0;
    int32_t fixpos[kMaxFixed] = {};
};

IndexPlan make_index_plan(int n, const std::vector<int>& fixed, uint64_t setmask);

// Gate matrix as the kernels see it: targets in the caller's order (bit j <-> targets[j]),
// controls with their values, dense 2^m x 2^m FP64 matrix (row = output).
struct DenseOp {
    std::vector<int> targets;
    std::vector<int> controls;
    std::vector<int> cvals;
    std::vector<cplx> mat;  // row-major 2^m x 2^m
};

// A gate decoded into the cheapest kernel that performs it.
enum class OpKind { Dense, Diag, Phase, Pauli, Swap, PauliRot };
struct Op {
    OpKind kind = OpKind::Dense;
    std::vector<int> targets;
    std::vector<int> controls;
    std::vector<int> cvals;
    std::vector<cplx> data;   // Dense: matrix; Diag: diagonal
    cplx phase = 1.0;         // Phase: factor on the subspace where all fixed bits match
    uint64_t xmask = 0, zmask = 0;  // Pauli, PauliRot
    double angle = 0.0;             // PauliRot: exp(i angle P / 2)
    const void* dmat = nullptr;     // Dense, optional: device copy of `data` in the state's element type
    bool dmat_oz = false;           // dmat holds the sliced tensor-core form (double-float, 4 targets)
};

// gate descriptor -> dense operator on (targets, controls) (throws Error on bad input)
DenseOp dense_of_gate(const qs_gate& g, int n, const double* theta_override);
// gate descriptor -> cheapest kernel form
Op op_of_gate(const qs_gate& g, int n, const double* theta_override);
// validation of qubit lists
void check_qubits(int n, const int* t, int m, const int* c, int mc);

// Arithmetic of the gate kernels: complex64 in FP32, complex128 in FP64, or complex128 held
// as double-float pairs (float4 {re_hi, re_lo, im_hi, im_lo}) on the FP32 pipes.
enum class Arith { F32 = 0, F64 = 1, DF = 2 };
inline Arith arith_of(const qs_state* s) {
    return s->dt == QS_C64 ? Arith::F32 : (s->df ? Arith::DF : Arith::F64);
}

// ------------------------------------------------------------------ device launches
// All launches are asynchronous on `st`. psi points at 2^n amplitudes of dtype dt.
// `stage`: a device buffer of at least kStageBytes, used to hand wide dense matrices to the
// kernels when op.dmat is not set.
constexpr size_t kStageBytes = 2 * 128 * 128 * 4;  // >= 64x64 complex128 and the tensor-core form
void launch_op(const Op& op, void* psi, int n, qs_dtype dt, cudaStream_t st, void* stage);
// ieee_in (double-float arithmetic only): psi still holds IEEE complex128 and the op leaves it in
// the double-float layout, the layout change done by the op's own kernel where it reads every
// amplitude once (takes_ieee_in), else by a conversion pass before it
void launch_op_arith(const Op& op, void* psi, int n, Arith ar, cudaStream_t st, void* stage, bool ieee_in = false);
// Tile shape of the shared-memory dense kernel (4..6 targets on the CUDA cores): output rows per
// thread, 4, 8 or 16, per device, arithmetic and width; 8 until the autotuner has timed them
// (tune_dense_tile_rows) or a test has set one.
int dense_tile_rows(Arith ar, int m);
void set_dense_tile_rows(Arith ar, int m, int rows);
bool dense_tile_rows_tuned(Arith ar, int m);
bool takes_ieee_in(const Op& op);
// Consecutive uncontrolled diagonal ops (and phases) together in one pass, their product held
// as two tables: each op in turn joins the first table if the union of its qubits stays within
// kDiagTableBits, else the second if within kDiagTable2Bits; a run ends at an op that fits
// neither (diag_split_add false, split unchanged). ieee_out (double-float only): the pass
// writes its results as IEEE complex128.
constexpr int kDiagTableBits = 12;
constexpr int kDiagTable2Bits = 8;
struct DiagSplit {
    std::vector<int> u, u2;  // the two tables' qubits
    std::vector<int> side;   // per op added: 0 first table, 1 second
};
bool diag_split_add(DiagSplit& sp, const std::vector<int>& qubits);
void launch_diag_run(const Op* ops, size_t count, void* psi, int n, Arith ar, cudaStream_t st, void* stage,
                     bool ieee_out = false);
// for each op: the number of ops launched together from it (>= 1), or 0 if an earlier op's
// diagonal run covers it
std::vector<int> diag_runs(const std::vector<Op>& ops);
void launch_set_basis(void* psi, int n, qs_dtype dt, uint64_t j, cudaStream_t st);
void launch_set_basis_arith(void* psi, int n, Arith ar, uint64_t j, cudaStream_t st);
// in-place layout change of a complex128 buffer: IEEE doubles <-> double-float pairs
void launch_to_df(void* psi, int n, cudaStream_t st);
void launch_from_df(void* psi, int n, cudaStream_t st);
// gate-matrix entries in the layout the kernels of `ar` read from device memory
size_t kernel_entry_bytes(Arith ar);
void encode_entries(Arith ar, const std::vector<cplx>& m, unsigned char* dst);

// Reductions: write results into the state's scratch and copy to host; synchronise.
void reduce_norm2(qs_state* s, double* out);
void reduce_inner(const qs_state* a, const qs_state* b, double out[2]);
void reduce_expectation(qs_state* s, const qs_pauli_obs* obs, double out[2]);
// <lambda| P |psi> for a Pauli string (complex), both states same n/dtype; synchronises.
// <bra|H|ket>, (re, im)
void reduce_transition(const qs_state* bra, const qs_pauli_obs* obs, const qs_state* ket, double out[2]);
// probability of the measured values (measured[q] = 0, 1, or 2 for any) of every qubit
void reduce_marginal(const qs_state* s, const int32_t* measured, double* out);
// out[k] = first x whose cumulative probability exceeds uniforms[k] times the total
void sample_state(const qs_state* s, int count, const double* uniforms, uint64_t* out);
void reduce_pauli_transition(qs_state* lam, const qs_state* psi, uint64_t xmask, uint64_t zmask,
                             double out[2]);

// Same value as reduce_expectation for a caller-owned device buffer (IEEE layout), with the
// per-block partials in a fixed device array instead of allocated scratch; synchronises.
void expectation_noalloc(const void* psi, int n, qs_dtype dt, cudaStream_t st, const qs_pauli_obs* obs,
                         double out[2]);
size_t noalloc_scratch_doubles();

// Observable grouped by flip mask for one pass per group.
struct PauliGroup {
    uint64_t xmask;
    std::vector<double> coef;
    std::vector<uint64_t> zmask;
};
std::vector<PauliGroup> group_observable(const qs_pauli_obs* obs, int n);

// Tiled expectation passes: a pass reads the state once as tiles of 2^12 amplitude slots (the
// amplitudes whose qubits outside a set T agree; T holds qubits 0..2 and 9 others, or all qubits
// of a smaller state, whose missing tile bits are virtual and read as zero amplitudes) and
// evaluates every flip-mask group whose flip mask lies in T. Groups whose flip mask has more than
// 9 bits above qubit 2 run one launch each.
constexpr int kTileBits = 12;
constexpr int kTransBits = 11;  // tiles of the two-state transition passes
constexpr int kTileAmps = 1 << kTileBits;
constexpr int kTileThreads = 256;
constexpr int kTileLowBits = 3;
constexpr int kTileMaxGroups = 24;
constexpr int kTileMaxSlots = 128;
constexpr int kTileMaxTerms = 128;
constexpr int kTileGroupTerms = 64;
constexpr int kHeavyChunkTerms = 48;
// Group kinds: the diagonal group (16 amplitudes per thread) and flip groups (8 pair
// representatives per thread) that need Re A, Im A or both.
enum TileKind : uint8_t { kTileDiag = 0, kTileRe = 1, kTileIm = 2, kTileReIm = 3 };
struct TileGroup {
    uint32_t f = 0;          // tile-local flip mask (0: the diagonal group)
    uint32_t excl = 0;       // the 4 tile-local bits that are not thread bits, ascending, one per byte
    uint32_t imask[4] = {};  // tile-local bit of item bit i (the pivot is not an item bit)
    uint16_t slot0 = 0;      // first slot of the group
    uint8_t kind = 0;        // TileKind
    uint8_t wht = 0;         // some slot has a nonzero item mask: full Walsh-Hadamard transform
    uint8_t bstart[17] = {}; // slots of bucket k (component * 8 + item mask): [bstart[k], bstart[k + 1])
};
struct TileSlot {
    uint16_t term0 = 0, nterm = 0;
    uint16_t zthr = 0;       // Z bits over the thread bits, in thread-index order
    uint8_t bucket = 0;
    uint8_t pad = 0;         // transition slots: nY mod 4, the rotation (-i)^{nY}
};
struct TileTerm {
    uint64_t zR = 0;         // Z bits outside the tile
    double alpha = 0.0;      // coefficient with the pair factor folded in
};
struct TileParams {
    uint64_t rest_mask = 0;  // qubits outside the tile
    uint64_t n_tiles = 0;
    uint64_t dep_hi[kTileAmps / kTileThreads] = {};  // global offset of tile-local index 256 k
    int32_t b = 0, ngroups = 0, nslots = 0, nterms = 0;  // b: real tile bits (<= 12)
    uint8_t tpos[kTileBits] = {};  // tile-local bit i < b = qubit tpos[i]
    TileGroup g[kTileMaxGroups];
    TileSlot s[kTileMaxSlots];
    TileTerm t[kTileMaxTerms];
};
struct HeavyChunk {
    const PauliGroup* g;
    size_t t0, t1;
};
// Diagonal observables (every term a Z string) whose Z qubits number at most kDiagObsBits: one
// streaming read, E = sum_x c(r(x)) |psi_x|^2 with c(r) = sum_t alpha_t (-1)^{popc(r & z_t)},
// r(x) the bits of x at the union of the terms' Z qubits (Sec. 4.5 with every flip mask zero).
constexpr int kDiagObsBits = 12;
constexpr int kDiagObsMaxTerms = 128;
struct DiagObsParams {
    uint64_t N = 0;
    int32_t m = 0, nterms = 0, nrun = 0;
    uint32_t run[kDiagObsBits] = {};  // runs of consecutive union qubits: shift | width << 8 | index bit << 16
    uint32_t z[kDiagObsMaxTerms] = {};  // term t's Z qubits as bits of the table index
    double alpha[kDiagObsMaxTerms] = {};
};
struct ExpectPlan {
    std::vector<TileParams> passes;
    std::vector<uint64_t> tmask;     // qubits of each pass's tile
    std::vector<HeavyChunk> heavy;   // terms [t0, t1) of groups that fit no tile
    bool diag = false;               // a diagonal observable read in one streaming pass (dp)
    DiagObsParams dp;
};
unsigned expect_diag_grid(int n, Arith ar);
// part[2 j], part[2 j + 1] = block j's partial (real, 0) for j < grid
void launch_expect_diag(const DiagObsParams& P, const void* psi, Arith ar, double* part, unsigned grid,
                        cudaStream_t st);
ExpectPlan plan_expectation(const std::vector<PauliGroup>& groups, int n);
unsigned expect_pass_grid(const TileParams& P, Arith ar);
// Transition amplitude <bra|O|ket>: tiles of 2^11 slots of both states (qubits 0..2 plus 8
// others); flip groups with more than 8 bits above qubit 2 go to heavy.
ExpectPlan plan_transition(const std::vector<PauliGroup>& groups, int n);
unsigned trans_pass_grid(const TileParams& P, Arith ar);
void launch_transition_pass(const TileParams& P, const void* bra, const void* ket, Arith ar, double* part,
                            unsigned grid, cudaStream_t st);
// part[2 j], part[2 j + 1] = block j's partial (real, 0) for j < grid
void launch_expect_pass(const TileParams& P, const void* psi, Arith ar, double* part, unsigned grid,
                        cudaStream_t st);

// lambda <- O psi (sum of Pauli strings), out-of-place; asynchronous.
void launch_apply_observable(const std::vector<PauliGroup>& groups, const void* psi, void* lam, int n,
                             Arith ar, cudaStream_t st);

// Fused adjoint step for an uncontrolled rotation exp(i theta P/2), P = X/Y/Z (axis 1/2/3) on
// `qubit`: per-block partials of Im <lam|P|psi> into part[0..grid), then psi, lam <- R^+ psi, R^+ lam.
unsigned adj_grid(int n);
void launch_adjoint_rotation(void* psi, void* lam, int n, Arith ar, int qubit, int axis, double theta, double* part,
                             unsigned grid, cudaStream_t st);
// nr consecutive rotation steps (2..adjoint_max_rotations(ar), which is 2) on distinct qubits
// (qubit[0] first, the latest in the circuit), one pass: partials of rotation r into
// part[r grid .. (r + 1) grid).
int adjoint_max_rotations(Arith ar);
void launch_adjoint_rotations(void* psi, void* lam, int n, Arith ar, int nr, const int* qubit, const int* axis,
                              const double* theta, double* part, unsigned grid, cudaStream_t st);
// Reverse step for a run of diagonal gates on psi and lam (both multiplied by the run's inverse),
// with the gradient partials of the run's diagonal rotations exp(i theta P / 2) (P a Z string
// gz[g]) computed before: part[g * grid + block] = block's sum of (-1)^popc(x & gz[g]) Im(conj(lam_x) psi_x).
constexpr int kAdjDiagMaxF = 48;
constexpr int kAdjDiagMaxG = 24;
constexpr int kAdjDiagMaxTab = 1024;
struct AdjDiagFactor {
    uint64_t cond_mask = 0, cond_val = 0;  // applies where (x & cond_mask) == cond_val
    uint64_t zmask = 0;                    // sign (-1)^popc(x & zmask)
    uint64_t pair_mask = 0;                // sign (-1)^popc(x & (x >> pair_shift) & pair_mask): a set of
    int32_t pair_shift = 0;                //   CZ gates on qubit pairs (a, a + pair_shift), bit a set
    int32_t sign_only = 0;                 // the factor is -1 (no table)
    int32_t tab_off = -1;                  // table of 2^nq entries (or none)
    int32_t nq = 0;
    int32_t q[6] = {0, 0, 0, 0, 0, 0};     // table index bit j = bit q[j] of x
    // the same gather as runs of consecutive q (consecutive j): x bits from (run & 0xFF), width
    // (run >> 8) & 0xFF, to table index bits from run >> 16
    int32_t nrun = 0;
    uint32_t run[6] = {0, 0, 0, 0, 0, 0};
};
struct AdjDiagParams {
    uint64_t n_amp = 0;
    int32_t nf = 0, ng = 0, ntab = 0, pad = 0;
    AdjDiagFactor f[kAdjDiagMaxF];
    uint64_t gz[kAdjDiagMaxG];
};
void launch_adjoint_diag(void* psi, void* lam, int n, Arith ar, const void* tab, const AdjDiagParams& A, double* part,
                         unsigned grid, cudaStream_t st);
// out[s] = sum_j part[s * nb + j] for s < nslots (fixed order)
void launch_slot_sums(const double* part, int nslots, unsigned nb, double* out, cudaStream_t st);

// Tensor-core path for double-float complex128 dense blocks of 4 targets (tcgen05, bf16
// slices with exact FP32 accumulation).
bool tensor_c128_enabled();
// the same op with its targets ascending (matrix local bits permuted to match)
Op sort_targets(const Op& op);
// host image of the sliced operand of a 16 x 16 matrix (stacked bf16 slices, row scales)
size_t oz4_matrix_bytes();
void prepare_oz4_matrix(const std::vector<cplx>& K, unsigned char* host_out);
// ieee_in: the state is read as IEEE complex128 (no controls: every amplitude is rewritten)
void launch_dense_oz4(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                      const std::vector<int>& cvals, const void* dmat, cudaStream_t st, bool ieee_in = false);
// 5-target blocks: the same method with the outputs in two halves (two stacked half matrices)
size_t oz5_matrix_bytes();
void prepare_oz5_matrix(const std::vector<cplx>& K, unsigned char* host_out);
void launch_dense_oz5(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                      const std::vector<int>& cvals, const void* dmat, cudaStream_t st, bool ieee_in = false);
// complex64 5- and 6-target blocks: three bf16 slices per operand, exact FP32 sums, one FP32
// rounding per output
bool tensor_c64x_enabled();
size_t bz_matrix_bytes(int q);
void prepare_bz_matrix(int q, const std::vector<cplx>& K, unsigned char* host_out);
void launch_dense_bz(void* psi, int n, const std::vector<int>& targets, const std::vector<int>& controls,
                     const std::vector<int>& cvals, const void* dmat, cudaStream_t st);
bool oz_error_pending();
// test hooks of the tensor-core kernels' bounded waits: try_wait attempts before a wait gives up
// (< 0: default), and a first accumulator wait that reports a timeout at once
void oz_set_wait_spins(long long spins);
void oz_set_force_late(bool on);
// test hooks of the batch kernel's grid barrier: polls before a wait gives up (< 0: default), and
// CTA 0 not arriving at the first barrier
void batch_set_wait_polls(long long polls);
void batch_set_hold_cta(bool on);

// complex128 arithmetic mode (QS_MATH_FP64 / QS_MATH_DF)
int c128_math();

// ------------------------------------------------------------------ fusion planner
struct FusedBlock {
    std::vector<int> qubits;   // ascending
    std::vector<cplx> mat;     // 2^w x 2^w
    int n_gates = 0;
    bool diagonal = false;
    int single_gate = -1;      // index of the source gate when the block holds exactly one
};
struct FusionPlan {
    int n = 0;
    int k = 0;
    int n_source_gates = 0;
    std::vector<FusedBlock> blocks;
    std::vector<qs_gate> source;          // copies of single-gate blocks' gates
    std::vector<std::vector<double>> source_mats;
};
// theta (optional): parameter vector overriding the angles of parametric gates
// forgets the cached partitions (planning starts afresh for every circuit)
void clear_partition_cache();
FusionPlan plan_fusion(const qs_circuit* c, int k, const double* theta = nullptr);
void apply_plan(qs_state* s, const FusionPlan& p);

}  // namespace qs

struct qs_fused_circuit {
    qs::FusionPlan plan;
};
