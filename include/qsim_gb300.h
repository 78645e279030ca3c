/*
 * qsim_gb300.h -- C ABI of the GB300 (sm_103a) state-vector simulator library
 * (libqsim_gb300.so).
 *
 * The library applies quantum gates to a full 2^n-amplitude state vector held in the
 * device memory of one GPU, evaluates Pauli observables on it, and differentiates
 * parametric circuits, following the Schroedinger-method simulator of the Qulacs paper
 * (Suzuki et al., Quantum 5, 559 (2021); arXiv 2011.13524).
 *
 * Conventions shared by every call:
 *  - State layout (Sec. 4.2.1): amplitude psi_x of basis state |x> sits at index x of a
 *    contiguous array of interleaved (re, im) pairs; qubit i is bit i of x ("the right-most
 *    digit is the 0-th qubit"). QS_C128 stores two IEEE doubles per amplitude (16 bytes),
 *    QS_C64 two IEEE floats (8 bytes).
 *  - Gate matrix (Sec. 4.3.2, Eq. update_mat): a 2^m x 2^m complex matrix K~ in row-major
 *    order, row = output local index z, column = input local index w, each element two
 *    doubles (re, im); bit j of a local index corresponds to targets[j]. K need not be
 *    unitary; no call renormalises the state.
 *  - Every function returns a qs_status; QS_OK is 0. On any other value a message is
 *    available from qs_last_error() (per calling thread). No C++ exception crosses this
 *    boundary.
 *  - Calls that only launch work are asynchronous on the state's CUDA stream. Calls that
 *    return a host value (expectation, norm, inner product, gradients, get_vector)
 *    synchronise that stream before returning. Errors that kernels record on the device
 *    are reported by the next synchronising call.
 *  - Host pointers passed in are only read during the call; the library keeps no
 *    reference to them. Device memory passed to qs_wrap_state stays owned by the caller.
 */
#ifndef QSIM_GB300_H
#define QSIM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qs_status;
#define QS_OK 0
#define QS_ERR_INVALID_ARG 1 /* bad qubit index, duplicate qubit, null pointer, size out of range */
#define QS_ERR_OOM 2         /* device allocation failed; nothing was leaked */
#define QS_ERR_CUDA 3        /* a CUDA runtime call failed (message carries cudaGetErrorString) */
#define QS_ERR_UNSUPPORTED 4 /* valid request the library does not implement */
#define QS_ERR_TIMEOUT 5     /* a bounded device-side wait gave up */
#define QS_ERR_NUMERIC 6     /* a result that must be real came out with a non-zero imaginary part */

typedef int qs_dtype;
#define QS_C64 1  /* complex64 storage, FP32 gate arithmetic with FP64-built matrices, FP64-class accumulation */
#define QS_C128 2 /* complex128 storage */

/* Arithmetic used for complex128 gate updates (qs_set_c128_math, qs_state_set_arith). */
#define QS_MATH_FP64 0 /* native FP64 multiply-adds (GB300 runs FP64 at 1/64 of the FP32 rate) */
#define QS_MATH_DF 1   /* double-float (two FP32 words per double, ~2^-46 relative) on the FP32 pipes;
                          the default */

#define QS_MAX_QUBITS 34
#define QS_MAX_TARGETS 6
#define QS_MAX_CONTROLS 8

/* Gate kinds (Sec. 4.3.2 basic gates). */
#define QS_GATE_DENSE 0 /* mat = 2^m x 2^m gate matrix */
#define QS_GATE_DIAG 1  /* mat = 2^m diagonal entries, psi_x <- d[r(x)] psi_x */
#define QS_GATE_PAULI 2 /* pauli[j] in {0,1,2,3} = {I,X,Y,Z} on targets[j] */
#define QS_GATE_NAMED 3 /* named gate of the paper's gate table, see QS_NAMED_* */

/* Named gates (Sec. 4.3.4 gate table). Rotations are exp(+i theta P / 2) (the table's sign);
 * U1/U2/U3 follow OpenQASM 2; S = diag(1,i), T = diag(1,e^{i pi/4}), sqrtX/sqrtY are the
 * principal square roots of X/Y. Qubits: 1-qubit gates use targets[0]; CNOT and TOFFOLI are X
 * on targets[0] with their controls in controls[]; CZ acts on targets[0..1]; SWAP on
 * targets[0..1]; FREDKIN is SWAP on targets[0..1] with controls[0]; PAULIROT is
 * exp(i params[0] P / 2) for the Pauli string pauli[] on targets[0..m-1]. */
#define QS_NAMED_X 1
#define QS_NAMED_Y 2
#define QS_NAMED_Z 3
#define QS_NAMED_H 4
#define QS_NAMED_S 5
#define QS_NAMED_SDAG 6
#define QS_NAMED_T 7
#define QS_NAMED_TDAG 8
#define QS_NAMED_SQRTX 9
#define QS_NAMED_SQRTXDAG 10
#define QS_NAMED_SQRTY 11
#define QS_NAMED_SQRTYDAG 12
#define QS_NAMED_RX 13
#define QS_NAMED_RY 14
#define QS_NAMED_RZ 15
#define QS_NAMED_U1 16
#define QS_NAMED_U2 17
#define QS_NAMED_U3 18
#define QS_NAMED_CNOT 19
#define QS_NAMED_CZ 20
#define QS_NAMED_SWAP 21
#define QS_NAMED_TOFFOLI 22
#define QS_NAMED_FREDKIN 23
#define QS_NAMED_PAULIROT 24

/* One gate. Controls: the gate acts only on the block where qubit controls[j] holds
 * control_values[j] (Sec. 4.3.2 controlled gates, add_control_qubit); controls and targets
 * must be disjoint. param_index >= 0 marks a parametric rotation (RX, RY, RZ, PAULIROT) whose
 * angle is theta[param_index] in qs_adjoint_grad and qs_batch_run; elsewhere params[0] is used. */
typedef struct qs_gate {
    int32_t kind;
    int32_t named;
    int32_t m;                                /* number of targets, 1..QS_MAX_TARGETS */
    int32_t targets[QS_MAX_TARGETS];
    int32_t mc;                               /* number of controls, 0..QS_MAX_CONTROLS */
    int32_t controls[QS_MAX_CONTROLS];
    int32_t control_values[QS_MAX_CONTROLS];
    int32_t pauli[QS_MAX_TARGETS];
    int32_t param_index;
    int32_t reserved;
    double params[3];
    const double* mat;                        /* host pointer (DENSE, DIAG), else NULL */
} qs_gate;

/* An ordered gate array (Sec. 4.4): gates are applied first to last. */
typedef struct qs_circuit {
    int32_t n;                                /* qubits */
    int32_t n_gates;
    int32_t n_params;                         /* parameters referenced by param_index */
    int32_t reserved;
    const qs_gate* gates;                     /* host array of n_gates */
} qs_circuit;

/* O = sum_k coef[k] P_k (Sec. 4.5), P_k by masks: bit q of x_mask set for X or Y on qubit q,
 * bit q of z_mask set for Z or Y on qubit q. A term with both masks 0 is coef * identity. */
typedef struct qs_pauli_obs {
    int32_t n_terms;
    int32_t reserved;
    const double* coef;                       /* host, n_terms */
    const uint64_t* x_mask;                   /* host, n_terms */
    const uint64_t* z_mask;                   /* host, n_terms */
} qs_pauli_obs;

typedef struct qs_state qs_state;             /* opaque */
typedef struct qs_fused_circuit qs_fused_circuit; /* opaque */

/* ---------------------------------------------------------------- library */
/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char* qs_last_error(void);
/* Library version string. */
const char* qs_version(void);
/* Settings. Each call reads the settings it uses once, at entry: a state's own settings
 * (qs_state_set_arith) where it has them, else the process-wide ones below. A call is therefore
 * not affected by settings that another thread changes while it runs; a state whose settings
 * are its own is not affected by the process-wide ones at all.
 * Process-wide arithmetic for complex128 gate updates: QS_MATH_FP64 or QS_MATH_DF (default). */
qs_status qs_set_c128_math(int mode);
qs_status qs_get_c128_math(int* mode);
/* Tensor-core paths for fused dense blocks (Sec. 5.4 blocks applied by Eq. update_mat),
 * process-wide, as a bit mask:
 * QS_TENSOR_C128: complex128 blocks of 4 or 5 targets in double-float runs (QS_MATH_DF): the
 *   matrix and every 16- or 32-amplitude group are scaled by powers of two and cut into six
 *   8-bit bf16 slices (the splitting of Ozaki, Ogita, Oishi and Rump); the 26 slice products of
 *   state slice s and matrix slice t with s + t <= 6 are summed exactly in FP32 by
 *   tcgen05.mma kind::f16 and combined exactly in double-float: about 2^-45 relative error per
 *   block, the accuracy of the double-float CUDA-core kernels.
 * QS_TENSOR_C64X: complex64 blocks of 5 or 6 targets: the matrix and every 32- or 64-amplitude
 *   group cut into three 8-bit bf16 slices; the 6 products with s + t <= 2 summed exactly in
 *   FP32 by tcgen05.mma kind::f16, added in FP32 with one rounding to nearest: about 2^-24
 *   relative error per block and no drift, the accuracy of the FP32 CUDA-core kernels.
 * Unknown bits -> QS_ERR_INVALID_ARG. Process-wide default: QS_TENSOR_C128 | QS_TENSOR_C64X. */
#define QS_TENSOR_C128 2
#define QS_TENSOR_C64X 4
qs_status qs_set_tensor_cores(int mask);
qs_status qs_get_tensor_cores(int* mask);

/* ---------------------------------------------------------------- states (Sec. 4.2) */
/* Allocates a 2^n state of type dt on the current device and sets it to |0...0>
 * (Sec. 4.2.1 default initialisation). stream: a cudaStream_t (NULL = legacy default).
 * The library owns the memory; release it with qs_destroy_state. n in [1, QS_MAX_QUBITS]. */
qs_status qs_create_state(int n, qs_dtype dt, void* stream, qs_state** out);
/* Wraps caller-owned device memory of 2^n amplitudes of type dt (16-byte aligned). The
 * contents are left as they are. qs_destroy_state frees only the handle. */
qs_status qs_wrap_state(void* dev_ptr, int n, qs_dtype dt, void* stream, qs_state** out);
/* The state's own arithmetic settings: c128_math is QS_MATH_FP64 or QS_MATH_DF, tensor_mask a
 * QS_TENSOR_* mask; -1 for either makes the state follow the process-wide setting (the default
 * of a new state). Used by every later call that applies gates to this state. */
qs_status qs_state_set_arith(qs_state* s, int c128_math, int tensor_mask);
qs_status qs_state_get_arith(const qs_state* s, int* c128_math, int* tensor_mask);
/* Frees the handle (and the memory, if the library allocated it). NULL is accepted. */
qs_status qs_destroy_state(qs_state* s);
/* Reports the qubit count, dtype and device pointer of a state (any output may be NULL). */
qs_status qs_state_info(const qs_state* s, int* n, qs_dtype* dt, void** dev_ptr);
/* Changes the stream on which later calls on this state run. */
qs_status qs_set_stream(qs_state* s, void* stream);
/* Computational basis state |j> (Sec. 4.2.1 set_computational_basis); j < 2^n. */
qs_status qs_set_basis(qs_state* s, uint64_t j);
/* Copies 2^n amplitudes of the state's dtype from src (host if is_device == 0, else device). */
qs_status qs_load(qs_state* s, const void* src, int is_device);
/* Copies the state into host memory of 2^n amplitudes (Sec. 4.2.2 get_vector); synchronises. */
qs_status qs_get_vector(const qs_state* s, void* host_out);
/* dst <- src; both states must have equal n and dtype (Sec. 4.2.1 load of another state). */
qs_status qs_copy_state(const qs_state* src, qs_state* dst);
/* Waits for the state's stream and reports device-side errors. */
qs_status qs_synchronize(const qs_state* s);

/* ---------------------------------------------------------------- gates (Sec. 4.3) */
/* psi <- K psi for one gate (Eq. update_mat; controlled, diagonal, Pauli and named forms).
 * complex128 dense gates of 3 or more targets use the double-float arithmetic (with its layout
 * change in and out) when it is selected; other gates use IEEE FP64 arithmetic, one pass. */
qs_status qs_apply_gate(qs_state* s, const qs_gate* g);
/* psi <- K psi for a dense k-qubit matrix (k in 1..6), as produced by gate fusion
 * (Sec. 5.4 merge). Equivalent to qs_apply_gate with a QS_GATE_DENSE gate. */
qs_status qs_apply_fused(qs_state* s, int k, const int* targets, const double* mat);
/* Applies every gate of c in order. fusion_k = 0 applies gate by gate; 1..6 first merges
 * gates into dense blocks of at most fusion_k qubits (Sec. 5.4 merge; the planner keeps the
 * partition with fewer blocks of two: an open-block greedy one, where a gate joins the open
 * block while the union of qubits stays within the width, and a frontier-growth one, which
 * may move a block past gates on other qubits, with which it commutes); -1 picks the width
 * with qs_autotune_fusion. c->n must equal the state's n. */
qs_status qs_run_circuit(qs_state* s, const qs_circuit* c, int fusion_k);

/* Pauli rotation gate (Sec. 4.3.2): psi <- exp(i angle P / 2) psi = cos(angle/2) psi +
 * i sin(angle/2) P psi, the half-angle convention of the RX/RY/RZ table, for a Pauli string P of
 * any length given by masks as in qs_pauli_obs (bit q of x_mask: X or Y on qubit q; of z_mask:
 * Z or Y). One O(2^n) pass whatever the length. Masks naming a qubit >= n -> QS_ERR_INVALID_ARG. */
qs_status qs_apply_pauli_rotation(qs_state* s, uint64_t x_mask, uint64_t z_mask, double angle);
/* Time evolution under an observable by the first-order Trotter decomposition (Sec. 4.5,
 * observable rotation): psi <- [prod_k exp(i (angle / n_slices) alpha_k P_k)]^n_slices psi, terms
 * in the observable's order, each factor a Pauli rotation with angle 2 angle alpha_k / n_slices
 * (an identity term is a global phase). Exact for commuting terms. n_slices >= 1. */
qs_status qs_apply_observable_rotation(qs_state* s, const qs_pauli_obs* H, double angle, int n_slices);

/* ---------------------------------------------------------------- fusion (Sec. 5.4) */
/* Plans the fused circuit for width k (2..6) without applying it. */
qs_status qs_plan_fusion(const qs_circuit* c, int k, qs_fused_circuit** out);
/* The library keeps the partitions of the last 16 circuit structures it planned (the qubits of
 * each gate, the width): a circuit run again with new angles or matrices is not partitioned
 * again. This forgets them; the next run or plan of any circuit partitions it afresh. The
 * autotuner's per-kernel timings of this GPU are kept. */
qs_status qs_clear_plan_cache(void);
/* Number of blocks of a plan and, for block b, its width and targets (ascending) and its
 * FP64 matrix (2^w x 2^w complex, row-major) copied to host memory; any output may be NULL. */
qs_status qs_fused_info(const qs_fused_circuit* f, int* n_blocks, int* n_source_gates);
qs_status qs_fused_block(const qs_fused_circuit* f, int b, int* width, int* targets, double* mat);
/* Applies a plan to a state (the plan's n must match). */
qs_status qs_apply_fused_circuit(qs_state* s, const qs_fused_circuit* f);
qs_status qs_destroy_fused(qs_fused_circuit* f);

/* Kernel that performs block b of a plan on a state of type dt, and its algorithmic memory
 * traffic: the bytes of state the update must read and write (Sec. 5.1 cost model,
 * N_mem), e.g. 2 * 2^(n - controls) amplitudes for a dense block. kernel: one of QS_KERNEL_*;
 * launches: kernels launched for the block (0 for an identity). Outputs may be NULL. */
#define QS_KERNEL_DENSE_REG 0  /* dense gate matrix, 1..3 targets (1..4 for complex64), registers */
#define QS_KERNEL_DENSE_SMEM 1 /* dense gate matrix, 4..6 targets, shared-memory tiles */
#define QS_KERNEL_DIAG 2       /* diagonal gate */
#define QS_KERNEL_PHASE 3      /* phase on the subspace of fixed bits */
#define QS_KERNEL_PAULI 4      /* Pauli string (permutation with phases) */
#define QS_KERNEL_SWAP 5       /* SWAP / controlled SWAP */
#define QS_KERNEL_DENSE_DF 6   /* complex128 dense gate matrix in double-float arithmetic */
#define QS_KERNEL_DENSE_OZ 8   /* double-float complex128 block of 4 targets on the tensor cores (bf16 slices) */
#define QS_KERNEL_PAULI_ROT 9  /* Pauli rotation exp(i phi P / 2), one pass over amplitude pairs */
#define QS_KERNEL_DENSE_OZ5 10 /* double-float complex128 block of 5 targets on the tensor cores (bf16 slices) */
#define QS_KERNEL_DENSE_BZ 11  /* complex64 block of 5 or 6 targets on the tensor cores (bf16 slices) */
qs_status qs_fused_block_cost(const qs_fused_circuit* f, int b, qs_dtype dt, int* kernel, int* launches,
                              double* bytes);
/* Separate layout-change passes (0, 1 or 2) that applying the plan to a complex128 state adds
 * under the current settings: a double-float run (QS_MATH_DF) holds the state as hi/lo float
 * pairs between a change at entry and one at exit, each a full read and write of the state,
 * unless the first block is an uncontrolled 4- or 5-target tensor-core block (it reads the
 * IEEE doubles itself) or the last pass is a run of diagonal blocks (it writes IEEE doubles);
 * 0 for complex64 and FP64 runs. Block b's kernel in qs_fused_block_cost includes what it
 * folds in. */
qs_status qs_fused_layout_passes(const qs_fused_circuit* f, qs_dtype dt, int* passes);
/* Applies a plan like qs_apply_fused_circuit, recording a CUDA event on the state's stream
 * after every block; block_ms[b] receives the device time of block b. Synchronises. */
qs_status qs_apply_fused_circuit_timed(qs_state* s, const qs_fused_circuit* f, float* block_ms);
/* Fusion-width autotuner: plans c for every width 1..6, predicts each plan's device time from
 * per-kernel costs measured on this GPU (timed once per process on a scratch state of
 * min(n, 24) qubits and scaled by 2^n), and returns the fastest width in *best_k. pred_ms
 * (optional, 7 entries): index 0 = gate by gate, 1..6 = fused widths. */
qs_status qs_autotune_fusion(const qs_circuit* c, qs_dtype dt, int* best_k, double* pred_ms);
/* Tile shape of the shared-memory dense kernel (QS_KERNEL_DENSE_SMEM: 4..6 targets on the CUDA
 * cores): output rows per thread, 4, 8 or 16 (the tile holds 256 rows / 2^m groups per row of
 * threads). The autotuner times the three shapes on this GPU the first time it costs that kernel
 * for an arithmetic (complex64; complex128 FP64 or double-float, the current setting) and width
 * m, and every later launch uses the fastest; until then 8. *rows = the shape in use for dt and
 * m on the current device; *tuned (optional) = 1 when it was timed or set. The shapes give the
 * same bits (every output is the same sum in the same order). m outside 4..6 ->
 * QS_ERR_INVALID_ARG. */
qs_status qs_dense_tile_rows(qs_dtype dt, int m, int* rows, int* tuned);

/* ---------------------------------------------------------------- observables (Sec. 4.5) */
/* out[0] = sum_k coef[k] <psi|P_k|psi>, out[1] = 0 (the terms are Hermitian and the coefficients
 * real, so the sum is formed as a real number). Terms with the same X-or-Y mask form a group; one
 * read of the state evaluates every group whose mask lies in a tile of 12 qubits (qubits 0..2
 * plus up to 9 others), in double-float arithmetic with FP64-class accuracy for complex128 and
 * exact products for complex64; groups with more than 9 X/Y positions above qubit 2 take one
 * read each. Synchronises. */
qs_status qs_expectation(const qs_state* s, const qs_pauli_obs* obs, double out[2]);
/* Host only (no GPU needed): how qs_expectation reads an n-qubit state for obs. *n_passes = the
 * tiled reads; tile_masks (optional, cap entries) receives each read's tile qubits as a bit mask;
 * *n_single (optional) = the reads of single groups that fit no tile. A diagonal observable (every
 * term a Z string) whose Z qubits number at most 12 takes one streaming read instead, reported as
 * one pass whose mask is those qubits. */
qs_status qs_expectation_plan(int n, const qs_pauli_obs* obs, int* n_passes, uint64_t* tile_masks, int cap,
                              int* n_single);
/* Allocation-free expectation, for callers that cannot allocate device memory: a process whose
 * device memory is all reserved by another allocator (a framework's caching pool) or held to a
 * fixed budget, where a cudaMalloc would fail or break the budget, and loops that must not call
 * the allocator at all because cudaMalloc and cudaFree can synchronise the whole device. Same
 * value as qs_expectation (within FP64 rounding of the block count), computed from caller-owned
 * memory: dev_psi holds 2^n amplitudes of type dt in the IEEE layout (16-byte aligned), out
 * (host) receives (re, im). The paper has no counterpart; it exists for these callers only.
 * It calls no cudaMalloc, cudaFree or other allocating routine. Its per-block partial sums live
 * in one fixed 512 KiB array in device memory that every GPU loading the library keeps until the
 * process exits. The first call on a device looks up that array's address (once per device, with
 * the device current). Every call shares the
 * array and each block overwrites its own slots, so nothing needs clearing, but calls that overlap
 * on the GPU (other streams, other threads) race on it: serialise them. The launches share the
 * array's 32767 block partials (grids shrink to fit); an observable that needs more launches than
 * that is rejected with QS_ERR_INVALID_ARG before any launch. Runs on `stream`, then copies the
 * result to `out` and synchronises `stream` before returning. */
qs_status qs_expectation_noalloc(const void* dev_psi, int n, qs_dtype dt, void* stream, const qs_pauli_obs* obs,
                                 double out[2]);
/* out = <a|b> (Sec. 4.2.2 inner_product) as (re, im); same n and dtype; synchronises. */
qs_status qs_inner_product(const qs_state* a, const qs_state* b, double out[2]);
/* Transition amplitude of an observable (Sec. 4.5): out = <bra|H|ket> = sum_k coef_k
 * <bra|P_k|ket> as (re, im), FP64 sums. Both states must have the same n and dtype. */
qs_status qs_transition_amplitude(const qs_state* bra, const qs_pauli_obs* H, const qs_state* ket, double out[2]);
/* Marginal probability (Sec. 4.2.2): measured_value[q] for every qubit q is 0, 1 or 2
 * (2 = any value); out = sum of |psi_x|^2 over the x that match (not divided by the norm).
 * Other values -> QS_ERR_INVALID_ARG. */
qs_status qs_marginal_probability(const qs_state* s, const int32_t* measured_value, double* out);
/* Z-basis sampling (Sec. 4.2.2): out[k] = the first basis index x whose cumulative probability
 * sum_{y <= x} |psi_y|^2 exceeds uniforms[k] * ||psi||^2, for caller-drawn uniforms[k] in [0, 1)
 * (host arrays of count entries). The cumulative distribution is built per call from chunk
 * masses (2^n / 4096 doubles of device scratch). A zero state -> QS_ERR_NUMERIC. */
qs_status qs_sample(const qs_state* s, int count, const double* uniforms, uint64_t* out);
/* out = <psi|psi> (Sec. 4.2.2 get_squared_norm); synchronises. */
qs_status qs_norm2(const qs_state* s, double* out);

/* ---------------------------------------------------------------- adjoint gradient */
/* Energy E = <psi(theta)|H|psi(theta)>, psi(theta) = U_G ... U_1 |0...0>, and dE/dtheta_p for
 * every parameter p of c (the gates with param_index = p; a parameter shared by several gates
 * gets the sum), by the reverse-sweep adjoint method: with lambda = H psi, each gate is
 * un-applied from psi and lambda in turn and a rotation exp(i theta P / 2) contributes
 * -Im <lambda|P|psi> at its position. The paper gives the parametric circuit (Sec. 4.4) but no
 * gradient; the sign follows from its rotation convention. theta: host, c->n_params values
 * (NULL = use each gate's params[0]). grad: host, c->n_params. Uses three device buffers of
 * 2^n amplitudes of type dt on `stream`; synchronises. */
qs_status qs_adjoint_grad(const qs_circuit* c, const double* theta, const qs_pauli_obs* H,
                          qs_dtype dt, void* stream, double* energy, double* grad);

/* ---------------------------------------------------------------- batched circuits */
/* Many independent small (circuit, observable) pairs evaluated together: energies and adjoint
 * gradients of parametric circuits, the paper's variational usage (Sec. 3.1, Sec. 4.4) at the
 * scale of thousands of circuits. complex64 states (QS_C64), 4..24 qubits each; gates RX, RY,
 * RZ (parametric or fixed, uncontrolled), CZ, CNOT (one control, value 1), H, X, Y, Z.
 * qs_batch_create validates and compiles the circuits once (per-circuit passes over 13-qubit
 * windows, device copies, a workspace of two 2^max_n complex64 buffers per SM when max_n > 13);
 * counts: circuits[k] and observables[k] for k < count. */
typedef struct qs_batch qs_batch; /* opaque */
qs_status qs_batch_create(const qs_circuit* circuits, const qs_pauli_obs* observables, int count, qs_dtype dt,
                          qs_batch** out);
/* Evaluates the whole batch in one persistent kernel launch on `stream`. theta: host, the
 * parameters of every circuit concatenated in order (circuit k contributes circuits[k].n_params
 * values; NULL only if no circuit has parameters). use_graph != 0 records the launch sequence
 * (parameter upload, angle kernel, the persistent kernel, result download) into a CUDA graph on
 * the first call and replays it afterwards. energies: host, count values; grads: host, the
 * gradients concatenated like theta. Synchronises. */
qs_status qs_batch_run(qs_batch* b, const double* theta, void* stream, int use_graph, double* energies,
                       double* grads);
/* Algorithmic device-memory traffic of one qs_batch_run, in bytes: the psi and lambda buffers of
 * the circuits wider than 13 qubits that their passes read and write (the first forward pass
 * writes psi, later ones read and write it; lambda = H psi reads psi and writes lambda; each
 * reverse pass reads and writes both). Narrower circuits run in shared memory and move only
 * their results. */
qs_status qs_batch_traffic(const qs_batch* b, double* bytes);
/* Total parameters, total passes of the compiled batch and device workspace bytes (any may be NULL). */
qs_status qs_batch_info(const qs_batch* b, int* total_params, int* total_passes, size_t* workspace_bytes);
qs_status qs_batch_destroy(qs_batch* b);

/* ---------------------------------------------------------------- test hooks */
/* Sets the shared-memory dense kernel's rows per thread (4, 8 or 16; 0 = back to untuned) for dt
 * (and, for complex128, the current arithmetic setting) and m in 4..6 on the current device, as
 * if the autotuner had chosen it. Other values -> QS_ERR_INVALID_ARG. */
qs_status qs_debug_set_tile_rows(qs_dtype dt, int m, int rows);
/* Every device-side wait of the library is bounded: when one gives up, its kernel records an
 * error, stops its work, waits (bounded) for its own asynchronous operations and exits; the next
 * synchronising call (qs_synchronize, or the call itself where it synchronises) reports
 * QS_ERR_TIMEOUT, the state's contents are then undefined, and the library stays usable. These
 * process-wide hooks let a test make such a wait run out without faulting or hanging the GPU.
 * qs_debug_set_wait_limit: polls of each pipeline wait of the tensor-core kernels and of each
 *   grid-barrier wait of the batch kernel before it gives up; -1 restores the defaults (seconds).
 *   The tensor-core kernels' final waits for their own MMAs always keep the default limit.
 * qs_debug_set_fault: QS_DEBUG_NONE; QS_DEBUG_TC_LATE: the first accumulator wait of every later
 *   tensor-core kernel launch reports a timeout without waiting; QS_DEBUG_BATCH_HOLD: CTA 0 of the
 *   batch kernel does not arrive at its first grid barrier (with a small wait limit every wait
 *   there runs out). A batch's captured graph is captured again when these settings change. */
#define QS_DEBUG_NONE 0
#define QS_DEBUG_TC_LATE 1
#define QS_DEBUG_BATCH_HOLD 2
qs_status qs_debug_set_wait_limit(long long polls);
qs_status qs_debug_set_fault(int what);
/* Every device and pinned-host allocation of the library is counted. qs_debug_fail_alloc makes
 * the allocation after `after` more successful ones fail as if memory had run out (-1: none), so
 * that the failing call returns QS_ERR_OOM; *held (optional) receives the number of allocations
 * the library holds now, to check that a failed call freed everything it had allocated. */
qs_status qs_debug_fail_alloc(long long after, long long* held);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_GB300_H */
