// C ABI of libqsim_gb300.so: states, gate application, fusion plans, reductions and the
// adjoint gradient. Every entry point converts C++ errors into a qs_status and a
// thread-local message; nothing throws across the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <exception>
#include <thread>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <memory>
#include <new>
#include <string>

#include "qsim_internal.h"

namespace qs {

namespace {
thread_local std::string g_err;
// process-wide settings: the default of states without settings of their own and of calls that
// take no state
std::atomic<int> g_c128_math{QS_MATH_DF};
std::atomic<int> g_tensor{QS_TENSOR_C128 | QS_TENSOR_C64X};  // QS_TENSOR_* bits
// the settings of the call in progress on this thread (-1 outside a call), taken once at entry
thread_local int t_math = -1, t_tensor = -1;

// Snapshot of the settings for one call: the state's own where it has them, else the
// process-wide ones as they are at entry; restored on exit (calls nest inside the library).
struct SettingsScope {
    int old_math, old_tensor;
    explicit SettingsScope(const qs_state* s) : old_math(t_math), old_tensor(t_tensor) {
        t_math = (s && s->math >= 0) ? s->math : (old_math >= 0 ? old_math : g_c128_math.load());
        t_tensor = (s && s->tensor >= 0) ? s->tensor : (old_tensor >= 0 ? old_tensor : g_tensor.load());
    }
    ~SettingsScope() {
        t_math = old_math;
        t_tensor = old_tensor;
    }
    SettingsScope(const SettingsScope&) = delete;
    SettingsScope& operator=(const SettingsScope&) = delete;
};
int cur_tensor() { return t_tensor >= 0 ? t_tensor : g_tensor.load(); }
}  // namespace

bool tensor_c128_enabled() { return (cur_tensor() & QS_TENSOR_C128) != 0; }
bool tensor_c64x_enabled() { return (cur_tensor() & QS_TENSOR_C64X) != 0; }

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
int c128_math() { return t_math >= 0 ? t_math : g_c128_math.load(); }

namespace {

void check_state(const qs_state* s) { QS_REQUIRE(s != nullptr && s->data != nullptr, "null state"); }

// after a synchronisation: an error that a tensor-core kernel on this device recorded (a bounded
// wait ran out; the state's contents are then undefined) is reported once
void report_device_errors() {
    if (oz_error_pending()) throw Error{QS_ERR_TIMEOUT, "tensor-core kernel: a bounded wait ran out"};
}

void* stage_of(qs_state* s) {
    if (!s->d_stage) QS_TRY_CUDA(dev_malloc(&s->d_stage, kStageBytes));
    return s->d_stage;
}

void free_state_resources(qs_state* s) {
    if (s->scratch.d_part) dev_free(s->scratch.d_part);
    if (s->scratch.h_out) host_free_pinned(s->scratch.h_out);
    if (s->d_stage) dev_free(s->d_stage);
    if (s->owns && s->data) dev_free(s->data);
    s->scratch = Scratch{};
    s->d_stage = nullptr;
    s->data = nullptr;
}

// adjoint of an operator: conjugate transpose (Pauli strings and SWAP are Hermitian)
Op dagger(const Op& op) {
    Op r = op;
    switch (op.kind) {
        case OpKind::Dense: {
            const int D = 1 << int(op.targets.size());
            for (int z = 0; z < D; z++)
                for (int w = 0; w < D; w++) r.data[size_t(z) * D + w] = std::conj(op.data[size_t(w) * D + z]);
            r.dmat = nullptr;
            break;
        }
        case OpKind::Diag:
            for (auto& v : r.data) v = std::conj(v);
            break;
        case OpKind::Phase: r.phase = std::conj(op.phase); break;
        case OpKind::PauliRot: r.angle = -op.angle; break;
        case OpKind::Pauli:
        case OpKind::Swap: break;
    }
    return r;
}

// A complex128 run in double-float arithmetic holds the buffer in the double-float layout
// between one conversion pass at entry and one at exit; every entry point sees IEEE doubles.
bool use_df(const qs_state* s) { return s->dt == QS_C128 && c128_math() == QS_MATH_DF; }

// With `deferred`, the entry conversion is left to the first launch (launch_op_arith with
// ieee_in), and entered() marks the buffer as converted once that launch is queued; left()
// marks a last launch that wrote IEEE doubles itself.
struct DFScope {
    qs_state* s;
    bool active;
    explicit DFScope(qs_state* st, bool on, bool deferred = false) : s(st), active(on && !st->df && !deferred) {
        if (active) {
            launch_to_df(s->data, s->n, s->stream);
            s->df = 1;
        }
    }
    void entered() {
        active = true;
        s->df = 1;
    }
    void left() {
        active = false;
        s->df = 0;
    }
    ~DFScope() {
        if (active) {
            s->df = 0;
            try {
                launch_from_df(s->data, s->n, s->stream);
            } catch (...) {
            }
        }
    }
};

// One gate outside a circuit run. complex128 dense gates of three or more targets take the
// double-float arithmetic (and the tensor-core blocks) when the state's settings select it: in
// FP64 they are bound by GB300's FP64 rate, so the layout change in and out (two passes) costs
// less than the FP64 update. Other gates keep IEEE FP64 arithmetic (one pass).
void apply_single(qs_state* s, const Op& op) {
    if (use_df(s) && op.kind == OpKind::Dense && op.targets.size() >= 3) {
        DFScope df(s, true);
        launch_op_arith(op, s->data, s->n, Arith::DF, s->stream, stage_of(s));
        return;
    }
    launch_op(op, s->data, s->n, s->dt, s->stream, stage_of(s));
}

void run_gates(qs_state* s, const qs_circuit* c, const double* theta) {
    std::vector<Op> ops;
    ops.reserve(c->n_gates);
    for (int i = 0; i < c->n_gates; i++) ops.push_back(op_of_gate(c->gates[i], s->n, theta));
    DFScope df(s, use_df(s));
    for (const Op& op : ops) launch_op_arith(op, s->data, s->n, arith_of(s), s->stream, stage_of(s));
}

}  // namespace

// Kernel form of block b of a plan (a single gate keeps its own cheapest form).
Op block_op(const FusionPlan& p, size_t b) {
    const FusedBlock& fb = p.blocks[b];
    if (fb.single_gate >= 0) return op_of_gate(p.source[fb.single_gate], p.n, nullptr);
    Op op;
    op.targets = fb.qubits;
    const int D = 1 << int(fb.qubits.size());
    if (fb.diagonal) {
        op.kind = OpKind::Diag;
        op.data.resize(D);
        for (int i = 0; i < D; i++) op.data[i] = fb.mat[size_t(i) * D + i];
    } else {
        op.kind = OpKind::Dense;
        op.data = fb.mat;
    }
    return op;
}

// Algorithmic traffic of an op on a 2^n state: amplitudes the update must read and write.
void op_cost(const Op& op, int n, qs_dtype dt, int* kernel, int* launches, double* bytes) {
    const double S = double(amp_bytes(dt));
    const int mc = int(op.controls.size());
    const double touched = std::ldexp(1.0, n - mc);
    int k = QS_KERNEL_DENSE_REG, l = 1;
    double by = 2.0 * S * touched;
    switch (op.kind) {
        case OpKind::Dense: {
            const int m = int(op.targets.size());
            const bool reg = m <= 3 || (m == 4 && dt == QS_C64);
            k = reg ? QS_KERNEL_DENSE_REG : QS_KERNEL_DENSE_SMEM;
            if (dt == QS_C64 && (m == 5 || m == 6) && tensor_c64x_enabled()) k = QS_KERNEL_DENSE_BZ;
            if (dt == QS_C128 && c128_math() == QS_MATH_DF && m <= 3) k = QS_KERNEL_DENSE_DF;
            if (dt == QS_C128 && c128_math() == QS_MATH_DF && (m == 4 || m == 5) && tensor_c128_enabled())
                k = m == 4 ? QS_KERNEL_DENSE_OZ : QS_KERNEL_DENSE_OZ5;
            break;
        }
        case OpKind::Diag: k = QS_KERNEL_DIAG; break;
        case OpKind::Phase:
            k = QS_KERNEL_PHASE;
            if (op.phase == cplx(1.0, 0.0)) { l = 0; by = 0.0; }
            break;
        case OpKind::Pauli:
            k = QS_KERNEL_PAULI;
            if (op.xmask == 0 && op.zmask == 0) { l = 0; by = 0.0; }
            else if (op.xmask == 0) by = 1.5 * S * touched;   // read all, write the odd-parity half
            break;
        case OpKind::Swap: k = QS_KERNEL_SWAP; by = S * touched; break;
        case OpKind::PauliRot: k = QS_KERNEL_PAULI_ROT; break;
    }
    if (kernel) *kernel = k;
    if (launches) *launches = l;
    if (bytes) *bytes = by;
}

namespace {
// Device copies of the wide (>= 4 target) dense matrices of a plan, in the state's element
// type, uploaded once per application on the state's stream.
struct WideMats {
    void* dbuf = nullptr;
    std::vector<const void*> ptr;
};

WideMats upload_wide(qs_state* s, Arith ar, std::vector<Op>& ops) {
    WideMats w;
    w.ptr.assign(ops.size(), nullptr);
    size_t total = 0;
    std::vector<size_t> offs(ops.size(), 0);
    std::vector<char> oz(ops.size(), 0);
    for (size_t b = 0; b < ops.size(); b++) {
        if (ops[b].kind != OpKind::Dense || ops[b].targets.size() < 4) continue;
        if (ar == Arith::F32 && (ops[b].targets.size() == 5 || ops[b].targets.size() == 6) && tensor_c64x_enabled()) {
            ops[b] = sort_targets(ops[b]);
            oz[b] = char(10 + ops[b].targets.size());  // the complex64 form, 15 or 16
        }
        if (ar == Arith::DF && (ops[b].targets.size() == 4 || ops[b].targets.size() == 5) && tensor_c128_enabled()) {
            ops[b] = sort_targets(ops[b]);
            oz[b] = char(ops[b].targets.size());
        }
        offs[b] = total;
        total += oz[b] == 4 ? oz4_matrix_bytes()
                 : oz[b] == 5 ? oz5_matrix_bytes()
                 : oz[b] >= 15 ? bz_matrix_bytes(oz[b] - 10)
                              : ops[b].data.size() * kernel_entry_bytes(ar);
        total = (total + 255) & ~size_t(255);
    }
    if (!total) return w;
    std::vector<unsigned char> host(total);
    std::vector<size_t> wide;
    for (size_t b = 0; b < ops.size(); b++)
        if (ops[b].kind == OpKind::Dense && ops[b].targets.size() >= 4) wide.push_back(b);
    auto prepare = [&](size_t b) {
        if (oz[b] == 4)
            prepare_oz4_matrix(ops[b].data, host.data() + offs[b]);
        else if (oz[b] == 5)
            prepare_oz5_matrix(ops[b].data, host.data() + offs[b]);
        else if (oz[b] >= 15)
            prepare_bz_matrix(oz[b] - 10, ops[b].data, host.data() + offs[b]);
        else
            encode_entries(ar, ops[b].data, host.data() + offs[b]);
    };
    // the blocks' device forms (sliced for the tensor cores, or encoded entries) are independent:
    // several host threads for long plans
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nth = wide.size() < 8 ? 1u : std::min<unsigned>(std::min(hw, 8u), unsigned(wide.size() / 4));
    if (nth <= 1) {
        for (size_t b : wide) prepare(b);
    } else {
        std::vector<std::thread> pool;
        std::vector<std::exception_ptr> errs(nth);
        for (unsigned t = 0; t < nth; t++)
            pool.emplace_back([&, t]() {
                try {
                    for (size_t i = t; i < wide.size(); i += nth) prepare(wide[i]);
                } catch (...) {
                    errs[t] = std::current_exception();
                }
            });
        for (auto& th : pool) th.join();
        for (auto& e : errs)
            if (e) std::rethrow_exception(e);
    }
    QS_TRY_CUDA(dev_malloc_async(&w.dbuf, total, s->stream));
    QS_TRY_CUDA(cudaMemcpyAsync(w.dbuf, host.data(), total, cudaMemcpyHostToDevice, s->stream));
    cudaStreamSynchronize(s->stream);  // the host staging vector dies on return
    for (size_t b = 0; b < ops.size(); b++)
        if (ops[b].kind == OpKind::Dense && ops[b].targets.size() >= 4) {
            w.ptr[b] = static_cast<unsigned char*>(w.dbuf) + offs[b];
            ops[b].dmat = w.ptr[b];
            ops[b].dmat_oz = oz[b] != 0;
        }
    return w;
}

}  // namespace

// diagonal ops that can join a tabulated run, and the qubits they act on
bool diag_mergeable(const Op& op) {
    return (op.kind == OpKind::Diag && op.controls.empty()) || op.kind == OpKind::Phase;
}
const std::vector<int>& diag_qubits(const Op& op) { return op.kind == OpKind::Phase ? op.controls : op.targets; }

std::vector<int> diag_runs(const std::vector<Op>& ops) {
    std::vector<int> len(ops.size(), 1);
    size_t b = 0;
    while (b < ops.size()) {
        size_t e = b;
        DiagSplit sp;
        if (diag_mergeable(ops[b]) && diag_split_add(sp, diag_qubits(ops[b])))
            while (e + 1 < ops.size() && diag_mergeable(ops[e + 1]) && diag_split_add(sp, diag_qubits(ops[e + 1]))) e++;
        len[b] = int(e - b + 1);
        for (size_t i = b + 1; i <= e; i++) len[i] = 0;
        b = e + 1;
    }
    return len;
}

namespace {

// A double-float run folds the layout changes into its first and last passes where those read
// every amplitude once: a tensor-core block first (it splits the IEEE doubles as it loads them),
// a tabulated diagonal run last (it writes RN(hi + lo)).
struct LayoutFold {
    bool in = false, out = false;
    size_t last = 0;  // the last op that launches
};
LayoutFold layout_fold(const std::vector<Op>& ops, const std::vector<int>& runs) {
    LayoutFold f;
    if (ops.empty()) return f;
    for (size_t b = 0; b < ops.size(); b++)
        if (runs[b] > 0) f.last = b;
    f.in = runs[0] == 1 && takes_ieee_in(ops[0]);
    f.out = runs[f.last] > 1;
    return f;
}

void apply_plan_impl(qs_state* s, const FusionPlan& p, float* block_ms) {
    QS_REQUIRE(p.n == s->n, "plan and state have different qubit counts");
    std::vector<Op> ops;
    ops.reserve(p.blocks.size());
    for (size_t b = 0; b < p.blocks.size(); b++) ops.push_back(block_op(p, b));
    const bool df_run = use_df(s);
    WideMats wm = upload_wide(s, df_run ? Arith::DF : arith_of(s), ops);
    std::vector<cudaEvent_t> ev;
    try {
        const std::vector<int> runs = diag_runs(ops);
        const LayoutFold fold = df_run && !s->df ? layout_fold(ops, runs) : LayoutFold{};
        const bool in_fused = fold.in, out_fused = fold.out;
        const size_t last = fold.last;
        const Arith ar = df_run ? Arith::DF : arith_of(s);
        DFScope df(s, df_run, in_fused);
        if (block_ms) {
            ev.resize(ops.size() + 1);
            for (auto& e : ev) QS_TRY_CUDA(cudaEventCreate(&e));
            QS_TRY_CUDA(cudaEventRecord(ev[0], s->stream));
        }
        for (size_t b = 0; b < ops.size(); b++) {
            if (runs[b] == 1) {
                launch_op_arith(ops[b], s->data, s->n, ar, s->stream, stage_of(s), in_fused && b == 0);
                if (in_fused && b == 0) df.entered();
            } else if (runs[b] > 1) {  // diagonal blocks in one pass (its time goes to the first)
                const bool to_ieee = out_fused && b == last;
                launch_diag_run(&ops[b], size_t(runs[b]), s->data, s->n, ar, s->stream, stage_of(s), to_ieee);
                if (to_ieee) df.left();
            }
            if (block_ms) QS_TRY_CUDA(cudaEventRecord(ev[b + 1], s->stream));
        }
        if (block_ms) {
            QS_TRY_CUDA(cudaEventSynchronize(ev.back()));
            for (size_t b = 0; b < ops.size(); b++) QS_TRY_CUDA(cudaEventElapsedTime(&block_ms[b], ev[b], ev[b + 1]));
        }
    } catch (...) {
        for (auto& e : ev) cudaEventDestroy(e);
        if (wm.dbuf) dev_free_async(wm.dbuf, s->stream);
        throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (wm.dbuf) QS_TRY_CUDA(dev_free_async(wm.dbuf, s->stream));
}

}  // namespace

void apply_plan(qs_state* s, const FusionPlan& p) { apply_plan_impl(s, p, nullptr); }

// ------------------------------------------------------------------ autotuner
// Seconds per algorithmic byte of each kernel form, measured once per process and device
// on a scratch state, keyed by (device, dtype, c128 arithmetic, kernel, targets).
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, bool>, double> g_cost;

double measure_cost(int dev, qs_dtype dt, const Op& probe_op, int np_) {
    qs_state* s = nullptr;
    qs_status rc = qs_create_state(np_, dt, nullptr, &s);
    if (rc != QS_OK) throw Error{rc, std::string("autotune: ") + qs_last_error()};
    struct G {
        qs_state* s;
        ~G() { qs_destroy_state(s); }
    } g{s};
    Op op = probe_op;
    std::vector<Op> one{op};
    const Arith ar = dt == QS_C64 ? Arith::F32 : (c128_math() == QS_MATH_DF ? Arith::DF : Arith::F64);
    WideMats wm;
    if (op.kind == OpKind::Dense && op.targets.size() >= 4) {
        wm = upload_wide(s, ar, one);
        op = one[0];
    }
    cudaEvent_t e0, e1;
    QS_TRY_CUDA(cudaEventCreate(&e0));
    QS_TRY_CUDA(cudaEventCreate(&e1));
    auto time_op = [&]() {  // best of three launches after one warm-up
        float best = 1e30f;
        for (int r = 0; r < 4; r++) {
            QS_TRY_CUDA(cudaEventRecord(e0, s->stream));
            launch_op_arith(op, s->data, s->n, ar, s->stream, stage_of(s));
            QS_TRY_CUDA(cudaEventRecord(e1, s->stream));
            QS_TRY_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            QS_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best = std::min(best, ms);
        }
        return best;
    };
    // the shared-memory dense kernel's tile shape (rows per thread) for this arithmetic and
    // width, timed once per device before its cost is measured
    int kernel = 0;
    op_cost(op, np_, dt, &kernel, nullptr, nullptr);
    const int m = int(op.targets.size());
    if (kernel == QS_KERNEL_DENSE_SMEM && !dense_tile_rows_tuned(ar, m)) {
        float best_ms = 1e30f;
        int best_rows = 8;
        for (int rows : {4, 8, 16}) {
            set_dense_tile_rows(ar, m, rows);
            const float t = time_op();
            if (t < best_ms) {
                best_ms = t;
                best_rows = rows;
            }
        }
        set_dense_tile_rows(ar, m, best_rows);
    }
    const float best = time_op();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (wm.dbuf) dev_free(wm.dbuf);
    (void)dev;
    double bytes = 0;
    op_cost(op, np_, dt, nullptr, nullptr, &bytes);
    return bytes > 0 ? 1e-3 * best / bytes : 0.0;
}

// whether an op's targets include qubit 0 or 1: such blocks read and write their amplitudes in
// short contiguous runs per thread, which costs the wide kernels more than other placements
bool touches_low(const Op& op) {
    if (op.kind != OpKind::Dense && op.kind != OpKind::Diag) return false;
    for (int t : op.targets)
        if (t <= 1) return true;
    return false;
}

// representative op of the same kernel form and width as `op`, on a probe state of np_ qubits:
// low and high qubits mixed when `op` touches qubit 0 or 1, consecutive middle qubits otherwise
Op probe_like(const Op& op, int np_) {
    static const int spread[6] = {0, -1, -2, 1, -3, 2};
    const bool low = touches_low(op);
    auto q = [&](int j) { return low ? (spread[j] >= 0 ? spread[j] : np_ + spread[j]) : np_ / 2 - 3 + j; };
    Op p;
    p.kind = op.kind;
    switch (op.kind) {
        case OpKind::Dense: {
            const int m = int(op.targets.size());
            for (int j = 0; j < m; j++) p.targets.push_back(q(j));
            const int D = 1 << m;
            p.data.assign(size_t(D) * D, cplx(0.0, 0.0));
            for (int z = 0; z < D; z++)
                for (int w = 0; w < D; w++) p.data[size_t(z) * D + w] = std::polar(1.0 / std::sqrt(double(D)), 0.37 * z * w + 0.1);
            break;
        }
        case OpKind::Diag: {
            const int m = int(op.targets.size());
            for (int j = 0; j < m; j++) p.targets.push_back(q(j));
            for (int i = 0; i < (1 << m); i++) p.data.push_back(std::polar(1.0, 0.3 * i + 0.2));
            break;
        }
        case OpKind::Phase:
            p.controls = {q(0), q(1)};
            p.cvals = {1, 1};
            p.phase = -1.0;
            break;
        case OpKind::Pauli: p.xmask = 1ull << q(1); break;
        case OpKind::Swap: p.targets = {q(0), q(1)}; break;
        case OpKind::PauliRot:
            p.xmask = (1ull << q(1)) | (1ull << q(0));
            p.zmask = 1ull << q(0);
            p.angle = 0.7;
            break;
    }
    return p;
}

double predicted_seconds(const Op& op, int n, qs_dtype dt) {
    int kernel = 0, launches = 0;
    double bytes = 0;
    op_cost(op, n, dt, &kernel, &launches, &bytes);
    if (!launches) return 0.0;
    int dev = 0;
    cudaGetDevice(&dev);
    const int width = op.kind == OpKind::Dense || op.kind == OpKind::Diag ? int(op.targets.size()) : 0;
    auto key = std::make_tuple(dev, int(dt), dt == QS_C128 ? c128_math() : cur_tensor() & QS_TENSOR_C64X,
                               kernel, width, touches_low(op));
    // (the kernel id already tells the tensor-core forms apart)
    double per_byte;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_cost.find(key);
        if (it != g_cost.end()) {
            per_byte = it->second;
        } else {
            const int np_ = std::max(8, std::min(n, dt == QS_C64 ? 25 : 24));
            per_byte = measure_cost(dev, dt, probe_like(op, np_), np_);
            g_cost[key] = per_byte;
        }
    }
    return per_byte * bytes + 2e-6;  // + launch overhead
}

double predict_plan(const FusionPlan& p, qs_dtype dt) {
    double t = 0;
    for (size_t b = 0; b < p.blocks.size(); b++) t += predicted_seconds(block_op(p, b), p.n, dt);
    return t;
}

double predict_unfused(const qs_circuit* c, qs_dtype dt) {
    double t = 0;
    for (int i = 0; i < c->n_gates; i++) t += predicted_seconds(op_of_gate(c->gates[i], c->n, nullptr), c->n, dt);
    return t;
}

int autotune(const qs_circuit* c, qs_dtype dt, double* pred_ms) {
    // the plans of every width are made on host threads at once (planning is CPU work, independent
    // per width); the predictions, which may time kernels on the GPU, follow one by one
    std::vector<FusionPlan> plans(QS_MAX_TARGETS + 1);
    std::vector<std::exception_ptr> errs(QS_MAX_TARGETS + 1);
    {
        std::vector<std::thread> pool;
        for (int k = 1; k <= QS_MAX_TARGETS; k++)
            pool.emplace_back([&, k]() {
                try {
                    plans[k] = plan_fusion(c, k);
                } catch (...) {
                    errs[k] = std::current_exception();
                }
            });
        for (auto& th : pool) th.join();
    }
    for (auto& e : errs)
        if (e) std::rethrow_exception(e);
    double best = predict_unfused(c, dt);
    if (pred_ms) pred_ms[0] = 1e3 * best;
    int best_k = 0;
    for (int k = 1; k <= QS_MAX_TARGETS; k++) {
        const double t = predict_plan(plans[k], dt);
        if (pred_ms) pred_ms[k] = 1e3 * t;
        if (t < best) {
            best = t;
            best_k = k;
        }
    }
    return best_k;
}
}  // namespace

}  // namespace qs

using namespace qs;

#define API_BEGIN \
    try {         \
        clear_error();\
        SettingsScope settings_scope_(nullptr);
// a call on a state: that state's settings (where it has its own) for the whole call
#define STATE_SETTINGS(s) SettingsScope state_settings_scope_(s)
#define API_END                                  \
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

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }

const char* qs_version(void) { return "qsim_gb300 0.1 (sm_103a)"; }

qs_status qs_set_c128_math(int mode) {
    API_BEGIN
    QS_REQUIRE(mode == QS_MATH_FP64 || mode == QS_MATH_DF, "unknown complex128 arithmetic mode");
    g_c128_math.store(mode);
    API_END
}

qs_status qs_set_tensor_cores(int mask) {
    API_BEGIN
    QS_REQUIRE((mask & ~(QS_TENSOR_C128 | QS_TENSOR_C64X)) == 0, "unknown tensor-core path bits");
    g_tensor.store(mask);
    API_END
}

qs_status qs_get_tensor_cores(int* mask) {
    API_BEGIN
    QS_REQUIRE(mask != nullptr, "null output");
    *mask = g_tensor.load();
    API_END
}

qs_status qs_get_c128_math(int* mode) {
    API_BEGIN
    QS_REQUIRE(mode != nullptr, "null output");
    *mode = g_c128_math.load();
    API_END
}

qs_status qs_debug_set_wait_limit(long long polls) {
    API_BEGIN
    QS_REQUIRE(polls >= -1, "wait limit must be -1 (default) or a poll count");
    oz_set_wait_spins(polls);
    batch_set_wait_polls(polls);
    API_END
}

qs_status qs_debug_set_fault(int what) {
    API_BEGIN
    QS_REQUIRE(what == QS_DEBUG_NONE || what == QS_DEBUG_TC_LATE || what == QS_DEBUG_BATCH_HOLD,
               "unknown wait-test setting");
    oz_set_force_late(what == QS_DEBUG_TC_LATE);
    batch_set_hold_cta(what == QS_DEBUG_BATCH_HOLD);
    API_END
}

qs_status qs_debug_fail_alloc(long long after, long long* held) {
    API_BEGIN
    QS_REQUIRE(after >= -1, "allocation count must be -1 (none) or at least 0");
    set_alloc_failure(after);
    if (held) *held = allocations_held();
    API_END
}

qs_status qs_state_set_arith(qs_state* s, int c128_math_mode, int tensor_mask) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(c128_math_mode == -1 || c128_math_mode == QS_MATH_FP64 || c128_math_mode == QS_MATH_DF,
               "unknown complex128 arithmetic mode");
    QS_REQUIRE(tensor_mask == -1 || (tensor_mask & ~(QS_TENSOR_C128 | QS_TENSOR_C64X)) == 0,
               "unknown tensor-core path bits");
    s->math = c128_math_mode;
    s->tensor = tensor_mask;
    API_END
}

qs_status qs_state_get_arith(const qs_state* s, int* c128_math_mode, int* tensor_mask) {
    API_BEGIN
    check_state(s);
    if (c128_math_mode) *c128_math_mode = s->math;
    if (tensor_mask) *tensor_mask = s->tensor;
    API_END
}

qs_status qs_create_state(int n, qs_dtype dt, void* stream, qs_state** out) {
    API_BEGIN
    QS_REQUIRE(out != nullptr, "null output");
    *out = nullptr;
    QS_REQUIRE(n >= 1 && n <= QS_MAX_QUBITS, "qubit count out of range (1..34)");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    std::unique_ptr<qs_state> s(new qs_state());
    s->n = n;
    s->dt = dt;
    s->stream = static_cast<cudaStream_t>(stream);
    s->owns = true;
    QS_TRY_CUDA(cudaGetDevice(&s->device));
    const size_t bytes = (size_t(1) << n) * amp_bytes(dt);
    cudaError_t e = dev_malloc(&s->data, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->data = nullptr;
        throw Error{e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA,
                    std::string("state allocation failed: ") + cudaGetErrorString(e)};
    }
    try {
        launch_set_basis(s->data, n, dt, 0, s->stream);
    } catch (...) {
        free_state_resources(s.get());
        throw;
    }
    *out = s.release();
    API_END
}

qs_status qs_wrap_state(void* dev_ptr, int n, qs_dtype dt, void* stream, qs_state** out) {
    API_BEGIN
    QS_REQUIRE(out != nullptr, "null output");
    *out = nullptr;
    QS_REQUIRE(dev_ptr != nullptr, "null device pointer");
    QS_REQUIRE((reinterpret_cast<uintptr_t>(dev_ptr) & 15) == 0, "device pointer must be 16-byte aligned");
    QS_REQUIRE(n >= 1 && n <= QS_MAX_QUBITS, "qubit count out of range (1..34)");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    std::unique_ptr<qs_state> s(new qs_state());
    s->n = n;
    s->dt = dt;
    s->data = dev_ptr;
    s->owns = false;
    s->stream = static_cast<cudaStream_t>(stream);
    QS_TRY_CUDA(cudaGetDevice(&s->device));
    *out = s.release();
    API_END
}

qs_status qs_destroy_state(qs_state* s) {
    API_BEGIN
    if (!s) return QS_OK;
    if (s->stream || s->data) cudaStreamSynchronize(s->stream);
    free_state_resources(s);
    delete s;
    API_END
}

qs_status qs_state_info(const qs_state* s, int* n, qs_dtype* dt, void** dev_ptr) {
    API_BEGIN
    check_state(s);
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    if (dev_ptr) *dev_ptr = s->data;
    API_END
}

qs_status qs_set_stream(qs_state* s, void* stream) {
    API_BEGIN
    check_state(s);
    s->stream = static_cast<cudaStream_t>(stream);
    API_END
}

qs_status qs_set_basis(qs_state* s, uint64_t j) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(j < (1ull << s->n), "basis index out of range");
    launch_set_basis(s->data, s->n, s->dt, j, s->stream);
    API_END
}

qs_status qs_load(qs_state* s, const void* src, int is_device) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(src != nullptr, "null source");
    const size_t bytes = (size_t(1) << s->n) * amp_bytes(s->dt);
    QS_TRY_CUDA(cudaMemcpyAsync(s->data, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                s->stream));
    API_END
}

qs_status qs_get_vector(const qs_state* s, void* host_out) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(host_out != nullptr, "null output");
    const size_t bytes = (size_t(1) << s->n) * amp_bytes(s->dt);
    QS_TRY_CUDA(cudaMemcpyAsync(host_out, s->data, bytes, cudaMemcpyDeviceToHost, s->stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    report_device_errors();
    API_END
}

qs_status qs_copy_state(const qs_state* src, qs_state* dst) {
    API_BEGIN
    check_state(src);
    check_state(dst);
    QS_REQUIRE(src->n == dst->n && src->dt == dst->dt, "states differ in qubit count or dtype");
    if (src->stream != dst->stream) QS_TRY_CUDA(cudaStreamSynchronize(src->stream));
    const size_t bytes = (size_t(1) << src->n) * amp_bytes(src->dt);
    QS_TRY_CUDA(cudaMemcpyAsync(dst->data, src->data, bytes, cudaMemcpyDeviceToDevice, dst->stream));
    API_END
}

qs_status qs_synchronize(const qs_state* s) {
    API_BEGIN
    check_state(s);
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    QS_TRY_CUDA(cudaGetLastError());
    report_device_errors();
    API_END
}

qs_status qs_apply_gate(qs_state* s, const qs_gate* g) {
    API_BEGIN
    STATE_SETTINGS(s);
    check_state(s);
    QS_REQUIRE(g != nullptr, "null gate");
    apply_single(s, op_of_gate(*g, s->n, nullptr));
    API_END
}

qs_status qs_apply_fused(qs_state* s, int k, const int* targets, const double* mat) {
    API_BEGIN
    STATE_SETTINGS(s);
    check_state(s);
    QS_REQUIRE(targets != nullptr && mat != nullptr, "null targets or matrix");
    QS_REQUIRE(k >= 1 && k <= QS_MAX_TARGETS, "fused width must be in 1..6");
    qs_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = QS_GATE_DENSE;
    g.m = k;
    for (int j = 0; j < k; j++) g.targets[j] = targets[j];
    g.mat = mat;
    g.param_index = -1;
    apply_single(s, op_of_gate(g, s->n, nullptr));
    API_END
}

qs_status qs_run_circuit(qs_state* s, const qs_circuit* c, int fusion_k) {
    API_BEGIN
    STATE_SETTINGS(s);
    check_state(s);
    QS_REQUIRE(c != nullptr, "null circuit");
    QS_REQUIRE(c->n == s->n, "circuit and state have different qubit counts");
    QS_REQUIRE(c->n_gates >= 0 && (c->n_gates == 0 || c->gates), "null gate array");
    QS_REQUIRE(fusion_k >= -1 && fusion_k <= QS_MAX_TARGETS, "fusion width must be -1, 0 or 1..6");
    if (fusion_k == 0) {
        run_gates(s, c, nullptr);
    } else {
        int k = fusion_k < 0 ? autotune(c, s->dt, nullptr) : fusion_k;
        if (k == 0)
            run_gates(s, c, nullptr);
        else
            apply_plan(s, plan_fusion(c, k));
    }
    API_END
}

qs_status qs_plan_fusion(const qs_circuit* c, int k, qs_fused_circuit** out) {
    API_BEGIN
    QS_REQUIRE(out != nullptr, "null output");
    *out = nullptr;
    std::unique_ptr<qs_fused_circuit> f(new qs_fused_circuit());
    f->plan = plan_fusion(c, k);
    *out = f.release();
    API_END
}

qs_status qs_clear_plan_cache(void) {
    API_BEGIN
    clear_partition_cache();
    API_END
}

qs_status qs_fused_info(const qs_fused_circuit* f, int* n_blocks, int* n_source_gates) {
    API_BEGIN
    QS_REQUIRE(f != nullptr, "null plan");
    if (n_blocks) *n_blocks = int(f->plan.blocks.size());
    if (n_source_gates) *n_source_gates = f->plan.n_source_gates;
    API_END
}

qs_status qs_fused_block(const qs_fused_circuit* f, int b, int* width, int* targets, double* mat) {
    API_BEGIN
    QS_REQUIRE(f != nullptr, "null plan");
    QS_REQUIRE(b >= 0 && b < int(f->plan.blocks.size()), "block index out of range");
    const FusedBlock& fb = f->plan.blocks[b];
    const int w = int(fb.qubits.size());
    if (width) *width = w;
    if (targets)
        for (int j = 0; j < w; j++) targets[j] = fb.qubits[j];
    if (mat) {
        std::vector<cplx> M = fb.mat;
        if (fb.single_gate >= 0) {
            // a block holding one gate keeps that gate; report its matrix on the sorted qubits
            const qs_gate& g = f->plan.source[fb.single_gate];
            DenseOp d = dense_of_gate(g, f->plan.n, nullptr);
            const int D = 1 << w;
            M.assign(size_t(D) * D, 0.0);
            for (int i = 0; i < D; i++) M[size_t(i) * D + i] = 1.0;
            // embed: identity off the control block, the gate matrix on the target bits
            std::vector<int> lt, lc;
            auto local = [&](int q) { return int(std::find(fb.qubits.begin(), fb.qubits.end(), q) - fb.qubits.begin()); };
            for (int t : d.targets) lt.push_back(local(t));
            for (int q : d.controls) lc.push_back(local(q));
            const int dm = 1 << int(lt.size());
            uint64_t tmask = 0, cmask = 0, cval = 0;
            for (size_t j = 0; j < lt.size(); j++) tmask |= 1ull << lt[j];
            for (size_t j = 0; j < lc.size(); j++) {
                cmask |= 1ull << lc[j];
                if (d.cvals[j]) cval |= 1ull << lc[j];
            }
            std::vector<cplx> E(size_t(D) * D, 0.0);
            for (int col = 0; col < D; col++) {
                for (int r = 0; r < D; r++) {
                    if ((uint64_t(r) & cmask) != cval) {
                        if (r == col) E[size_t(r) * D + col] = 1.0;
                        continue;
                    }
                    if ((uint64_t(r) & ~tmask) != (uint64_t(col) & ~tmask)) continue;
                    int zr = 0, zc = 0;
                    for (size_t j = 0; j < lt.size(); j++) {
                        zr |= int((r >> lt[j]) & 1) << j;
                        zc |= int((col >> lt[j]) & 1) << j;
                    }
                    E[size_t(r) * D + col] = d.mat[size_t(zr) * dm + zc];
                }
            }
            M = E;
        }
        for (size_t e = 0; e < M.size(); e++) {
            mat[2 * e] = M[e].real();
            mat[2 * e + 1] = M[e].imag();
        }
    }
    API_END
}

qs_status qs_apply_fused_circuit(qs_state* s, const qs_fused_circuit* f) {
    API_BEGIN
    STATE_SETTINGS(s);
    check_state(s);
    QS_REQUIRE(f != nullptr, "null plan");
    apply_plan(s, f->plan);
    API_END
}

qs_status qs_destroy_fused(qs_fused_circuit* f) {
    API_BEGIN
    delete f;
    API_END
}

qs_status qs_fused_block_cost(const qs_fused_circuit* f, int b, qs_dtype dt, int* kernel, int* launches,
                              double* bytes) {
    API_BEGIN
    QS_REQUIRE(f != nullptr, "null plan");
    QS_REQUIRE(b >= 0 && b < int(f->plan.blocks.size()), "block index out of range");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    std::vector<Op> ops;
    for (size_t i = 0; i < f->plan.blocks.size(); i++) ops.push_back(block_op(f->plan, i));
    const std::vector<int> runs = diag_runs(ops);
    op_cost(ops[size_t(b)], f->plan.n, dt, kernel, launches, bytes);
    if (runs[size_t(b)] == 0) {  // applied in the pass of an earlier diagonal block
        if (launches) *launches = 0;
        if (bytes) *bytes = 0.0;
    } else if (runs[size_t(b)] > 1) {  // the first block of a tabulated diagonal run: one full pass
        if (kernel) *kernel = QS_KERNEL_DIAG;
        if (launches) *launches = 1;
        if (bytes) *bytes = 2.0 * double(amp_bytes(dt)) * std::ldexp(1.0, f->plan.n);
    }
    API_END
}

qs_status qs_fused_layout_passes(const qs_fused_circuit* f, qs_dtype dt, int* passes) {
    API_BEGIN
    QS_REQUIRE(f != nullptr && passes != nullptr, "null plan or output");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    *passes = 0;
    if (dt == QS_C128 && c128_math() == QS_MATH_DF) {
        std::vector<Op> ops;
        for (size_t i = 0; i < f->plan.blocks.size(); i++) ops.push_back(block_op(f->plan, i));
        const LayoutFold fold = layout_fold(ops, diag_runs(ops));
        *passes = 2 - int(fold.in) - int(fold.out);
    }
    API_END
}

qs_status qs_apply_fused_circuit_timed(qs_state* s, const qs_fused_circuit* f, float* block_ms) {
    API_BEGIN
    STATE_SETTINGS(s);
    check_state(s);
    QS_REQUIRE(f != nullptr && block_ms != nullptr, "null plan or output");
    apply_plan_impl(s, f->plan, block_ms);
    API_END
}

qs_status qs_dense_tile_rows(qs_dtype dt, int m, int* rows, int* tuned) {
    API_BEGIN
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "dtype must be QS_C64 or QS_C128");
    QS_REQUIRE(m >= 4 && m <= 6, "tile rows exist for 4..6 targets");
    QS_REQUIRE(rows != nullptr, "null output");
    const Arith ar = dt == QS_C64 ? Arith::F32 : (c128_math() == QS_MATH_DF ? Arith::DF : Arith::F64);
    *rows = dense_tile_rows(ar, m);
    if (tuned) *tuned = dense_tile_rows_tuned(ar, m) ? 1 : 0;
    API_END
}

qs_status qs_debug_set_tile_rows(qs_dtype dt, int m, int rows) {
    API_BEGIN
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "dtype must be QS_C64 or QS_C128");
    const Arith ar = dt == QS_C64 ? Arith::F32 : (c128_math() == QS_MATH_DF ? Arith::DF : Arith::F64);
    set_dense_tile_rows(ar, m, rows);
    API_END
}

qs_status qs_autotune_fusion(const qs_circuit* c, qs_dtype dt, int* best_k, double* pred_ms) {
    API_BEGIN
    QS_REQUIRE(c != nullptr && best_k != nullptr, "null circuit or output");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    QS_REQUIRE(c->n >= 1 && c->n <= QS_MAX_QUBITS, "qubit count out of range");
    *best_k = autotune(c, dt, pred_ms);
    API_END
}

qs_status qs_expectation(const qs_state* s, const qs_pauli_obs* obs, double out[2]) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(out != nullptr, "null output");
    reduce_expectation(const_cast<qs_state*>(s), obs, out);
    report_device_errors();
    API_END
}

qs_status qs_expectation_plan(int n, const qs_pauli_obs* obs, int* n_passes, uint64_t* tile_masks, int cap,
                              int* n_single) {
    API_BEGIN
    QS_REQUIRE(n >= 1 && n <= QS_MAX_QUBITS, "qubit count out of range (1..34)");
    QS_REQUIRE(n_passes != nullptr, "null output");
    QS_REQUIRE(cap >= 0 && (cap == 0 || tile_masks != nullptr), "null tile mask array");
    const std::vector<PauliGroup> groups = group_observable(obs, n);
    const ExpectPlan plan = plan_expectation(groups, n);
    *n_passes = int(plan.passes.size()) + (plan.diag ? 1 : 0);
    for (size_t p = 0; p < plan.tmask.size() && p < size_t(cap); p++) tile_masks[p] = plan.tmask[p];
    if (n_single) *n_single = int(plan.heavy.size());
    API_END
}

qs_status qs_expectation_noalloc(const void* dev_psi, int n, qs_dtype dt, void* stream, const qs_pauli_obs* obs,
                                 double out[2]) {
    API_BEGIN
    expectation_noalloc(dev_psi, n, dt, static_cast<cudaStream_t>(stream), obs, out);
    API_END
}

qs_status qs_inner_product(const qs_state* a, const qs_state* b, double out[2]) {
    API_BEGIN
    check_state(a);
    check_state(b);
    QS_REQUIRE(out != nullptr, "null output");
    QS_REQUIRE(a->n == b->n && a->dt == b->dt, "states differ in qubit count or dtype");
    reduce_inner(a, b, out);
    API_END
}

qs_status qs_transition_amplitude(const qs_state* bra, const qs_pauli_obs* H, const qs_state* ket, double out[2]) {
    API_BEGIN
    check_state(bra);
    check_state(ket);
    QS_REQUIRE(out != nullptr, "null output");
    QS_REQUIRE(bra->n == ket->n && bra->dt == ket->dt, "states differ in qubit count or dtype");
    reduce_transition(bra, H, ket, out);
    API_END
}

qs_status qs_marginal_probability(const qs_state* s, const int32_t* measured_value, double* out) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(measured_value != nullptr && out != nullptr, "null argument");
    reduce_marginal(s, measured_value, out);
    API_END
}

qs_status qs_sample(const qs_state* s, int count, const double* uniforms, uint64_t* out) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(count >= 0, "negative sample count");
    QS_REQUIRE(count == 0 || (uniforms != nullptr && out != nullptr), "null argument");
    sample_state(s, count, uniforms, out);
    API_END
}

qs_status qs_norm2(const qs_state* s, double* out) {
    API_BEGIN
    check_state(s);
    QS_REQUIRE(out != nullptr, "null output");
    reduce_norm2(const_cast<qs_state*>(s), out);
    report_device_errors();
    API_END
}

qs_status qs_apply_pauli_rotation(qs_state* s, uint64_t x_mask, uint64_t z_mask, double angle) {
    API_BEGIN
    STATE_SETTINGS(s);
    QS_REQUIRE(s != nullptr, "null state");
    const uint64_t all = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
    QS_REQUIRE(((x_mask | z_mask) & ~all) == 0, "Pauli mask names a qubit outside the state");
    Op op;
    op.kind = OpKind::PauliRot;
    op.xmask = x_mask;
    op.zmask = z_mask;
    op.angle = angle;
    DFScope df(s, use_df(s));
    launch_op_arith(op, s->data, s->n, arith_of(s), s->stream, stage_of(s));
    API_END
}

qs_status qs_apply_observable_rotation(qs_state* s, const qs_pauli_obs* H, double angle, int n_slices) {
    API_BEGIN
    STATE_SETTINGS(s);
    QS_REQUIRE(s != nullptr && H != nullptr, "null state or observable");
    QS_REQUIRE(n_slices >= 1, "n_slices must be positive");
    QS_REQUIRE(H->n_terms >= 0 && (H->n_terms == 0 || (H->coef && H->x_mask && H->z_mask)), "null observable arrays");
    const uint64_t all = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
    std::vector<Op> ops;
    for (int k = 0; k < H->n_terms; k++) {
        QS_REQUIRE(((H->x_mask[k] | H->z_mask[k]) & ~all) == 0, "Pauli mask names a qubit outside the state");
        Op op;
        op.kind = OpKind::PauliRot;
        op.xmask = H->x_mask[k];
        op.zmask = H->z_mask[k];
        op.angle = 2.0 * angle * H->coef[k] / n_slices;  // exp(i (angle / r) alpha_k P_k)
        ops.push_back(op);
    }
    DFScope df(s, use_df(s));
    for (int r = 0; r < n_slices; r++)
        for (const Op& op : ops) launch_op_arith(op, s->data, s->n, arith_of(s), s->stream, stage_of(s));
    API_END
}

qs_status qs_adjoint_grad(const qs_circuit* c, const double* theta, const qs_pauli_obs* H, qs_dtype dt, void* stream,
                          double* energy, double* grad) {
    API_BEGIN
    QS_REQUIRE(c != nullptr && H != nullptr, "null circuit or observable");
    QS_REQUIRE(energy != nullptr, "null energy output");
    QS_REQUIRE(c->n_params >= 0 && (c->n_params == 0 || grad != nullptr), "null gradient output");
    QS_REQUIRE(c->n >= 1 && c->n <= QS_MAX_QUBITS, "qubit count out of range");
    QS_REQUIRE(c->n_gates >= 0 && (c->n_gates == 0 || c->gates), "null gate array");
    QS_REQUIRE(dt == QS_C64 || dt == QS_C128, "unknown dtype");
    // parametric gates: uncontrolled rotations exp(i theta P / 2)
    for (int i = 0; i < c->n_gates; i++) {
        const qs_gate& g = c->gates[i];
        if (g.param_index < 0) continue;
        QS_REQUIRE(g.param_index < c->n_params, "param_index out of range");
        QS_REQUIRE(g.kind == QS_GATE_NAMED && (g.named == QS_NAMED_RX || g.named == QS_NAMED_RY ||
                                               g.named == QS_NAMED_RZ || g.named == QS_NAMED_PAULIROT),
                   "a parametric gate must be RX, RY, RZ or PAULIROT");
        if (g.mc != 0) throw Error{QS_ERR_UNSUPPORTED, "controlled parametric rotations are not differentiated"};
    }
    const std::vector<PauliGroup> groups = group_observable(H, c->n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    qs_state *psi = nullptr, *lam = nullptr;
    qs_status rc = qs_create_state(c->n, dt, stream, &psi);
    if (rc != QS_OK) throw Error{rc, std::string("adjoint: ") + qs_last_error()};
    rc = qs_create_state(c->n, dt, stream, &lam);
    if (rc != QS_OK) {
        qs_destroy_state(psi);
        throw Error{rc, std::string("adjoint: ") + qs_last_error()};
    }
    struct Guard {
        qs_state *a, *b;
        ~Guard() {
            qs_destroy_state(a);
            qs_destroy_state(b);
        }
    } guard{psi, lam};
    // both buffers stay in the double-float layout for the whole sweep when that arithmetic
    // is selected (they are scratch states, never seen outside this call)
    if (use_df(psi)) {
        psi->df = 1;
        lam->df = 1;
        launch_set_basis_arith(psi->data, c->n, Arith::DF, 0, st);
    }
    const Arith ar = arith_of(psi);
    // The reverse sweep as steps: single-qubit X/Y rotations use the fused reverse step
    // (gradient partials + un-apply in one pass); maximal runs of diagonal gates (CZ, phases,
    // RZ and Z-string rotations, diagonal gates) take one pass for the whole run; other gates
    // are un-applied on both buffers, and a parametric Pauli rotation with X or Y factors gets
    // its gradient from a transition amplitude first. Partial sums of the device-side
    // gradients land in per-block slots, reduced once after the sweep.
    auto fused_rot = [&](const qs_gate& g) {
        return g.param_index >= 0 && g.mc == 0 && (g.named == QS_NAMED_RX || g.named == QS_NAMED_RY);
    };
    struct Step {
        int kind = 0;               // 0 rotation, 1 diagonal run, 2 other gate, 3 rotations sharing a pass
        int gate = -1;              // kinds 0, 2
        std::vector<int> rots;      // kind 3: the rotations, latest first (slots slot0, slot0 + 1, ...)
        int slot0 = 0;              // first gradient slot
        std::shared_ptr<AdjDiagParams> diag;  // kind 1 (a few KB: held once, not copied with the step)
        size_t tab_byte = 0;        // kind 1: offset of its tables in the upload
        std::vector<int> params;    // kind 1: parameter index of each gradient term
    };
    std::vector<Step> steps;
    std::vector<cplx> tabs;         // every run's tables, in order
    int nslots = 0;
    // The steps depend only on the circuit and the angles: a host thread builds them while this
    // one plans and launches the forward pass and the energy (joined before the sweep, and on
    // every way out of this scope).
    std::exception_ptr step_err;
    std::thread step_builder([&]() {
        try {
            {
                std::vector<int> run;       // gate indices, reverse order
                int run_f = 0, run_g = 0, run_t = 0;  // its factor, gradient and table-entry bounds
                uint64_t run_sq = 0;        // qubits of its uncontrolled single-qubit diagonals (tables of 6)
                auto single_entries = [](uint64_t q) {
                    const int k = __builtin_popcountll(q);
                    return (k / 6) * 64 + (k % 6 ? 1 << (k % 6) : 0);
                };
                auto flush = [&]() {
                    run_f = run_g = run_t = 0;
                    run_sq = 0;
                    if (run.empty()) return;
                    Step stp;
                    stp.kind = 1;
                    stp.slot0 = nslots;
                    stp.diag = std::make_shared<AdjDiagParams>();
                    AdjDiagParams& A = *stp.diag;
                    A.n_amp = 1ull << c->n;
                    stp.tab_byte = tabs.size();
                    // single-qubit uncontrolled diagonals multiply into per-qubit pairs, then into tables
                    // over up to 4 qubits; every other diagonal keeps a factor of its own
                    std::map<int, std::pair<cplx, cplx>> one;
                    int ntab = 0;
                    auto add_factor = [&](const AdjDiagFactor& f, const std::vector<cplx>& t) {
                        QS_REQUIRE(A.nf < kAdjDiagMaxF, "diagonal run too long");
                        AdjDiagFactor g = f;
                        g.nrun = 0;
                        for (int j = 0; j < g.nq;) {
                            int k = j + 1;
                            while (k < g.nq && g.q[k] == g.q[k - 1] + 1) k++;
                            g.run[g.nrun++] = uint32_t(g.q[j]) | (uint32_t(k - j) << 8) | (uint32_t(j) << 16);
                            j = k;
                        }
                        if (!t.empty()) {
                            g.tab_off = ntab;
                            for (const cplx& v : t) tabs.push_back(v);
                            ntab += int(t.size());
                        }
                        A.f[A.nf++] = g;
                    };
                    for (int gi : run) {
                        const qs_gate& g = c->gates[gi];
                        Op op = dagger(op_of_gate(g, c->n, theta));
                        if (g.param_index >= 0) {
                            uint64_t zm = 0;
                            for (int j = 0; j < g.m; j++)
                                if (g.kind == QS_GATE_NAMED && g.named == QS_NAMED_RZ) zm |= 1ull << g.targets[j];
                                else if (g.pauli[j] == 3) zm |= 1ull << g.targets[j];
                            A.gz[A.ng++] = zm;
                            stp.params.push_back(g.param_index);
                        }
                        uint64_t cm = 0, cv = 0;
                        for (size_t j = 0; j < op.controls.size(); j++) {
                            cm |= 1ull << op.controls[j];
                            if (op.cvals[j]) cv |= 1ull << op.controls[j];
                        }
                        AdjDiagFactor f;
                        f.cond_mask = cm;
                        f.cond_val = cv;
                        if (op.kind == OpKind::Pauli) {
                            f.zmask = op.zmask;
                            add_factor(f, {});
                        } else if (op.kind == OpKind::Phase) {
                            if (op.phase == cplx(-1.0, 0.0)) {
                                f.sign_only = 1;
                                add_factor(f, {});
                            } else if (op.phase != cplx(1.0, 0.0)) {
                                add_factor(f, {op.phase});
                            }
                        } else if (op.targets.size() == 1 && cm == 0) {
                            auto it = one.find(op.targets[0]);
                            if (it == one.end()) one[op.targets[0]] = {op.data[0], op.data[1]};
                            else it->second = {it->second.first * op.data[0], it->second.second * op.data[1]};
                        } else {
                            f.nq = int(op.targets.size());
                            for (int j = 0; j < f.nq; j++) f.q[j] = op.targets[j];
                            add_factor(f, op.data);
                        }
                    }
                    // CZ gates (a -1 on the subspace where both of two qubits are 1, no other condition)
                    // with the same qubit distance d share one factor: the parity of x & (x >> d) over
                    // their lower qubits
                    {
                        std::map<int, uint64_t> pairs;
                        std::vector<AdjDiagFactor> keep;
                        for (int k = 0; k < A.nf; k++) {
                            const AdjDiagFactor& g = A.f[k];
                            if (g.sign_only && g.zmask == 0 && g.tab_off < 0 && __builtin_popcountll(g.cond_mask) == 2 &&
                                g.cond_val == g.cond_mask) {
                                const int a = __builtin_ctzll(g.cond_mask), b = 63 - __builtin_clzll(g.cond_mask);
                                uint64_t& m = pairs[b - a];
                                if (!((m >> a) & 1)) {
                                    m |= 1ull << a;
                                    continue;
                                }
                                m &= ~(1ull << a);  // the same CZ twice cancels
                                continue;
                            }
                            keep.push_back(g);
                        }
                        A.nf = 0;
                        for (const AdjDiagFactor& g : keep) A.f[A.nf++] = g;
                        for (const auto& pm : pairs) {
                            if (!pm.second) continue;
                            AdjDiagFactor g;
                            g.pair_shift = pm.first;
                            g.pair_mask = pm.second;
                            A.f[A.nf++] = g;
                        }
                    }
                    std::vector<std::pair<int, std::pair<cplx, cplx>>> ones(one.begin(), one.end());
                    for (size_t i0 = 0; i0 < ones.size(); i0 += 6) {
                        AdjDiagFactor f;
                        f.nq = int(std::min<size_t>(6, ones.size() - i0));
                        std::vector<cplx> t(size_t(1) << f.nq, cplx(1.0, 0.0));
                        for (int j = 0; j < f.nq; j++) {
                            f.q[j] = ones[i0 + j].first;
                            for (size_t li = 0; li < t.size(); li++)
                                t[li] *= ((li >> j) & 1) ? ones[i0 + j].second.second : ones[i0 + j].second.first;
                        }
                        add_factor(f, t);
                    }
                    A.ntab = ntab;
                    QS_REQUIRE(ntab <= kAdjDiagMaxTab, "diagonal run tables too large");
                    nslots += A.ng;
                    steps.push_back(std::move(stp));
                    run.clear();
                };
                for (int i = c->n_gates - 1; i >= 0; i--) {
                    const qs_gate& g = c->gates[i];
                    const Op op = op_of_gate(g, c->n, theta);
                    // a parametric rotation joins a diagonal run when its generator is a Z string, whatever
                    // its matrix at this angle: RX(0) is the identity, but its derivative (i/2) X is not
                    // diagonal and needs the rotation step
                    bool gen_diag = true;
                    if (g.param_index >= 0) {
                        if (g.named == QS_NAMED_RX || g.named == QS_NAMED_RY) gen_diag = false;
                        if (g.named == QS_NAMED_PAULIROT)
                            for (int j = 0; j < g.m; j++) gen_diag = gen_diag && (g.pauli[j] == 0 || g.pauli[j] == 3);
                    }
                    const bool diag = op.kind == OpKind::Diag || op.kind == OpKind::Phase ||
                                      (op.kind == OpKind::Pauli && op.xmask == 0);
                    const bool diag_param = g.param_index < 0 || (gen_diag && op.kind != OpKind::Dense && g.mc == 0);
                    if (diag && diag_param) {
                        // bound the run by the kernel's factor, gradient and table limits (worst case);
                        // uncontrolled single-qubit diagonals share tables of up to 6 qubits
                        const bool single = op.kind == OpKind::Diag && op.targets.size() == 1 && op.controls.empty();
                        const int tab_need = single ? 0 : op.kind == OpKind::Diag ? (1 << op.targets.size()) : 1;
                        const uint64_t sq = single ? run_sq | (1ull << op.targets[0]) : run_sq;
                        if (run_f + 1 > kAdjDiagMaxF || run_g + (g.param_index >= 0) > kAdjDiagMaxG ||
                            run_t + tab_need + single_entries(sq) > kAdjDiagMaxTab)
                            flush();
                        run.push_back(i);
                        run_f += 1;
                        run_g += g.param_index >= 0;
                        run_t += tab_need;
                        if (single) run_sq |= 1ull << op.targets[0];
                        continue;
                    }
                    flush();
                    Step stp;
                    stp.gate = i;
                    if (fused_rot(g)) {
                        stp.kind = 0;
                        stp.slot0 = nslots++;
                    } else {
                        stp.kind = 2;
                    }
                    steps.push_back(stp);
                }
                flush();
            }
            // up to adjoint_max_rotations consecutive rotation steps on distinct qubits share one pass
            // (their slots are adjacent)
            {
                const int maxr = std::min(adjoint_max_rotations(ar), c->n);
                std::vector<Step> merged;
                for (size_t i = 0; i < steps.size();) {
                    if (steps[i].kind != 0 || maxr < 2) {
                        merged.push_back(steps[i++]);
                        continue;
                    }
                    size_t j = i;
                    uint64_t used = 0;
                    while (j < steps.size() && int(j - i) < maxr && steps[j].kind == 0 &&
                           !((used >> c->gates[steps[j].gate].targets[0]) & 1)) {
                        used |= 1ull << c->gates[steps[j].gate].targets[0];
                        j++;
                    }
                    if (j - i >= 2) {
                        Step m = steps[i];
                        m.kind = 3;
                        for (size_t t = i; t < j; t++) m.rots.push_back(steps[t].gate);
                        merged.push_back(m);
                    } else {
                        merged.push_back(steps[i]);
                    }
                    i = j > i + 1 ? j : i + 1;
                }
                steps.swap(merged);
            }
        } catch (...) {
            step_err = std::current_exception();
        }
    });
    struct Joiner {
        std::thread& t;
        ~Joiner() {
            if (t.joinable()) t.join();
        }
    } joiner{step_builder};

    // forward: psi = U_G ... U_1 |0>, fused (the partition of a circuit structure is cached, so
    // repeated calls with new angles only rebuild the block matrices)
    // (tensor-core widths: 5 for double-float, 6 for complex64; the CUDA-core kernels' own)
    const int kf = ar == Arith::DF && tensor_c128_enabled()     ? 5
                   : ar == Arith::F32 && tensor_c64x_enabled() ? 6
                   : ar == Arith::F32                           ? 4
                                                                : 2;
    apply_plan(psi, plan_fusion(c, kf, theta));
    // lambda = H psi ; E = Re <psi|lambda>
    launch_apply_observable(groups, psi->data, lam->data, c->n, ar, st);
    double e2[2];
    reduce_inner(psi, lam, e2);
    *energy = e2[0];
    for (int p = 0; p < c->n_params; p++) grad[p] = 0.0;
    step_builder.join();
    if (step_err) std::rethrow_exception(step_err);
    const unsigned nb = adj_grid(c->n);
    double* d_part = nullptr;
    void* d_tab = nullptr;
    const size_t eb = kernel_entry_bytes(ar);
    if (nslots) QS_TRY_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d_part), sizeof(double) * (size_t(nslots) * nb + nslots), st));
    std::vector<int> slot_param(nslots, -1);
    try {
        if (!tabs.empty()) {
            std::vector<unsigned char> host(tabs.size() * eb);
            encode_entries(ar, tabs, host.data());
            QS_TRY_CUDA(dev_malloc_async(&d_tab, host.size(), st));
            QS_TRY_CUDA(cudaMemcpyAsync(d_tab, host.data(), host.size(), cudaMemcpyHostToDevice, st));
            QS_TRY_CUDA(cudaStreamSynchronize(st));  // the host copy dies on return
        }
        for (const Step& stp : steps) {
            if (stp.kind == 1) {
                launch_adjoint_diag(psi->data, lam->data, c->n, ar,
                                    static_cast<const unsigned char*>(d_tab) + stp.tab_byte * eb, *stp.diag,
                                    d_part ? d_part + size_t(stp.slot0) * nb : nullptr, nb, st);
                for (size_t g = 0; g < stp.params.size(); g++) slot_param[stp.slot0 + g] = stp.params[g];
                continue;
            }
            const qs_gate& g = c->gates[stp.gate];
            if (stp.kind == 3) {
                const int nr = int(stp.rots.size());
                int q[4], ax[4];
                double th[4];
                for (int r = 0; r < nr; r++) {
                    const qs_gate& gr = c->gates[stp.rots[r]];
                    q[r] = gr.targets[0];
                    ax[r] = gr.named == QS_NAMED_RX ? 1 : 2;
                    th[r] = theta ? theta[gr.param_index] : gr.params[0];
                    slot_param[stp.slot0 + r] = gr.param_index;
                }
                launch_adjoint_rotations(psi->data, lam->data, c->n, ar, nr, q, ax, th, d_part + size_t(stp.slot0) * nb, nb, st);
                continue;
            }
            if (stp.kind == 0) {
                const int axis = g.named == QS_NAMED_RX ? 1 : 2;
                const double th = theta ? theta[g.param_index] : g.params[0];
                launch_adjoint_rotation(psi->data, lam->data, c->n, ar, g.targets[0], axis, th,
                                        d_part + size_t(stp.slot0) * nb, nb, st);
                slot_param[stp.slot0] = g.param_index;
                continue;
            }
            Op op = op_of_gate(g, c->n, theta);
            if (g.param_index >= 0) {
                uint64_t xm = 0, zm = 0;
                for (int j = 0; j < g.m; j++) {
                    const int id = g.pauli[j], q = g.targets[j];
                    if (id == 1 || id == 2) xm |= 1ull << q;
                    if (id == 2 || id == 3) zm |= 1ull << q;
                }
                double t[2];
                reduce_pauli_transition(lam, psi, xm, zm, t);
                // d/dtheta exp(i theta P/2) = (i/2) P U  ->  dE/dtheta = -Im <lambda|P|psi>
                grad[g.param_index] += -t[1];
            }
            Op inv = dagger(op);
            launch_op_arith(inv, psi->data, c->n, ar, st, stage_of(psi));
            launch_op_arith(inv, lam->data, c->n, ar, st, stage_of(lam));
        }
        if (nslots) {
            double* d_sums = d_part + size_t(nslots) * nb;
            launch_slot_sums(d_part, nslots, nb, d_sums, st);
            std::vector<double> sums(nslots);
            QS_TRY_CUDA(cudaMemcpyAsync(sums.data(), d_sums, sizeof(double) * nslots, cudaMemcpyDeviceToHost, st));
            QS_TRY_CUDA(cudaStreamSynchronize(st));
            for (int sidx = 0; sidx < nslots; sidx++) grad[slot_param[sidx]] += -sums[sidx];
        }
    } catch (...) {
        if (d_part) dev_free_async(d_part, st);
        if (d_tab) dev_free_async(d_tab, st);
        throw;
    }
    if (d_tab) QS_TRY_CUDA(dev_free_async(d_tab, st));
    if (d_part) QS_TRY_CUDA(dev_free_async(d_part, st));
    QS_TRY_CUDA(cudaStreamSynchronize(st));
    report_device_errors();
    API_END
}

}  // extern "C"
