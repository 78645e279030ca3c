// Gate descriptors -> gate matrices and kernel forms (host C++).
//
// Named gates follow the paper's gate table (Sec. 4.3.4): Pauli matrices as printed in
// Sec. 4.3.2; rotations RX/RY/RZ = exp(+i theta P / 2), the table's sign; U1/U2/U3 from
// OpenQASM 2, to which the table defers; S = diag(1, i), T = diag(1, e^{i pi/4}) and the
// principal square roots of X and Y for the table's "pi/4 rotations". Each gate is then
// mapped to the cheapest update of Sec. 4.3.2: a Pauli gate or a SWAP is a permutation with
// phases (no multiplies), a diagonal gate whose entries are all 1 but one touches only the
// subspace where that entry sits (a phase on 2^(n-m) amplitudes), other diagonals scale
// every amplitude, and everything else is a dense gate-matrix update.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "qsim_internal.h"

namespace qs {

namespace {

const double kPi = 3.14159265358979323846;
const cplx kI(0.0, 1.0);

std::vector<cplx> mat2(cplx a, cplx b, cplx c, cplx d) { return {a, b, c, d}; }

// sigma_id as a 2x2 matrix (Sec. 4.3.2): I, X, Y, Z
cplx pauli_entry(int id, int row, int col) {
    switch (id) {
        case 0: return row == col ? 1.0 : 0.0;
        case 1: return row != col ? 1.0 : 0.0;
        case 2:
            if (row == col) return 0.0;
            return row == 0 ? -kI : kI;   // Y = [[0, -i], [i, 0]]
        case 3: return row == col ? (row == 0 ? 1.0 : -1.0) : 0.0;
    }
    return 0.0;
}

// Pauli string on m local qubits: bit j of the local index <-> ids[j].
std::vector<cplx> pauli_string(const int* ids, int m) {
    const int D = 1 << m;
    std::vector<cplx> P(size_t(D) * D);
    for (int z = 0; z < D; z++)
        for (int w = 0; w < D; w++) {
            cplx v = 1.0;
            for (int j = 0; j < m && v != 0.0; j++) v *= pauli_entry(ids[j], (z >> j) & 1, (w >> j) & 1);
            P[size_t(z) * D + w] = v;
        }
    return P;
}

// exp(i theta P / 2) = cos(theta/2) I + i sin(theta/2) P   (P^2 = I)
std::vector<cplx> rotation(const std::vector<cplx>& P, int D, double theta) {
    std::vector<cplx> R(P.size());
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    for (int z = 0; z < D; z++)
        for (int w = 0; w < D; w++) R[size_t(z) * D + w] = (z == w ? c : 0.0) + kI * s * P[size_t(z) * D + w];
    return R;
}

std::vector<cplx> u3(double th, double ph, double la) {
    const double c = std::cos(th / 2), s = std::sin(th / 2);
    return mat2(c, -std::exp(kI * la) * s, std::exp(kI * ph) * s, std::exp(kI * (ph + la)) * c);
}

int expected_targets(int named) {
    switch (named) {
        case QS_NAMED_CZ:
        case QS_NAMED_SWAP:
        case QS_NAMED_FREDKIN: return 2;
        case QS_NAMED_PAULIROT: return -1;
        default: return 1;
    }
}

double angle(const qs_gate& g, const double* theta) {
    if (theta && g.param_index >= 0) return theta[g.param_index];
    return g.params[0];
}

}  // namespace

void check_qubits(int n, const int* t, int m, const int* c, int mc) {
    QS_REQUIRE(n >= 1 && n <= QS_MAX_QUBITS, "qubit count out of range");
    QS_REQUIRE(m >= 1 && m <= QS_MAX_TARGETS, "target count out of range (1..6)");
    QS_REQUIRE(mc >= 0 && mc <= QS_MAX_CONTROLS, "control count out of range (0..8)");
    uint64_t seen = 0;
    for (int j = 0; j < m; j++) {
        QS_REQUIRE(t[j] >= 0 && t[j] < n, "target qubit index out of range");
        QS_REQUIRE(!((seen >> t[j]) & 1), "duplicate qubit in gate");
        seen |= 1ull << t[j];
    }
    for (int j = 0; j < mc; j++) {
        QS_REQUIRE(c[j] >= 0 && c[j] < n, "control qubit index out of range");
        QS_REQUIRE(!((seen >> c[j]) & 1), "control qubit coincides with a target or another control");
        seen |= 1ull << c[j];
    }
}

DenseOp dense_of_gate(const qs_gate& g, int n, const double* theta) {
    DenseOp op;
    QS_REQUIRE(g.m >= 1 && g.m <= QS_MAX_TARGETS, "target count out of range (1..6)");
    check_qubits(n, g.targets, g.m, g.controls, g.mc);
    op.targets.assign(g.targets, g.targets + g.m);
    op.controls.assign(g.controls, g.controls + g.mc);
    for (int j = 0; j < g.mc; j++) op.cvals.push_back(g.control_values[j] ? 1 : 0);
    const int D = 1 << g.m;
    switch (g.kind) {
        case QS_GATE_DENSE:
            QS_REQUIRE(g.mat != nullptr, "DENSE gate without matrix");
            op.mat.resize(size_t(D) * D);
            for (size_t i = 0; i < op.mat.size(); i++) op.mat[i] = cplx(g.mat[2 * i], g.mat[2 * i + 1]);
            return op;
        case QS_GATE_DIAG:
            QS_REQUIRE(g.mat != nullptr, "DIAG gate without entries");
            op.mat.assign(size_t(D) * D, 0.0);
            for (int i = 0; i < D; i++) op.mat[size_t(i) * D + i] = cplx(g.mat[2 * i], g.mat[2 * i + 1]);
            return op;
        case QS_GATE_PAULI:
            for (int j = 0; j < g.m; j++) QS_REQUIRE(g.pauli[j] >= 0 && g.pauli[j] <= 3, "Pauli id out of range");
            op.mat = pauli_string(g.pauli, g.m);
            return op;
        case QS_GATE_NAMED: break;
        default: throw Error{QS_ERR_INVALID_ARG, "unknown gate kind"};
    }
    const int et = expected_targets(g.named);
    QS_REQUIRE(et < 0 || et == g.m, "wrong number of targets for named gate");
    const double r2 = 1.0 / std::sqrt(2.0);
    const cplx h(0.5, 0.5), hc(0.5, -0.5);
    switch (g.named) {
        case QS_NAMED_X:
        case QS_NAMED_CNOT:
        case QS_NAMED_TOFFOLI: {
            int id = 1;
            op.mat = pauli_string(&id, 1);
            break;
        }
        case QS_NAMED_Y: { int id = 2; op.mat = pauli_string(&id, 1); break; }
        case QS_NAMED_Z: { int id = 3; op.mat = pauli_string(&id, 1); break; }
        case QS_NAMED_H: op.mat = mat2(r2, r2, r2, -r2); break;
        case QS_NAMED_S: op.mat = mat2(1.0, 0.0, 0.0, kI); break;
        case QS_NAMED_SDAG: op.mat = mat2(1.0, 0.0, 0.0, -kI); break;
        case QS_NAMED_T: op.mat = mat2(1.0, 0.0, 0.0, std::exp(kI * (kPi / 4))); break;
        case QS_NAMED_TDAG: op.mat = mat2(1.0, 0.0, 0.0, std::exp(-kI * (kPi / 4))); break;
        // principal square roots: sqrtX^2 = X, sqrtY^2 = Y
        case QS_NAMED_SQRTX: op.mat = mat2(h, hc, hc, h); break;
        case QS_NAMED_SQRTXDAG: op.mat = mat2(hc, h, h, hc); break;
        case QS_NAMED_SQRTY: op.mat = mat2(h, -h, h, h); break;
        case QS_NAMED_SQRTYDAG: op.mat = mat2(hc, hc, -hc, hc); break;
        case QS_NAMED_RX:
        case QS_NAMED_RY:
        case QS_NAMED_RZ: {
            int id = g.named == QS_NAMED_RX ? 1 : g.named == QS_NAMED_RY ? 2 : 3;
            op.mat = rotation(pauli_string(&id, 1), 2, angle(g, theta));
            break;
        }
        case QS_NAMED_U1: op.mat = mat2(1.0, 0.0, 0.0, std::exp(kI * g.params[0])); break;
        case QS_NAMED_U2: op.mat = u3(kPi / 2, g.params[0], g.params[1]); break;
        case QS_NAMED_U3: op.mat = u3(g.params[0], g.params[1], g.params[2]); break;
        case QS_NAMED_CZ: op.mat = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, -1.0}; break;
        case QS_NAMED_SWAP:
        case QS_NAMED_FREDKIN: op.mat = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1}; break;
        case QS_NAMED_PAULIROT:
            for (int j = 0; j < g.m; j++) QS_REQUIRE(g.pauli[j] >= 0 && g.pauli[j] <= 3, "Pauli id out of range");
            op.mat = rotation(pauli_string(g.pauli, g.m), D, angle(g, theta));
            break;
        default: throw Error{QS_ERR_INVALID_ARG, "unknown named gate"};
    }
    return op;
}

namespace {

// A diagonal gate whose entries are 1 except at local index `hot` becomes a phase on the
// subspace where the targets read `hot` (and the controls hold).
bool as_phase(const std::vector<cplx>& d, int* hot) {
    int h = -1;
    for (size_t i = 0; i < d.size(); i++) {
        if (d[i] != cplx(1.0, 0.0)) {
            if (h >= 0) return false;
            h = int(i);
        }
    }
    if (h < 0) h = 0;  // identity: any single entry works (phase 1)
    *hot = h;
    return true;
}

bool is_diagonal(const std::vector<cplx>& M, int D) {
    for (int z = 0; z < D; z++)
        for (int w = 0; w < D; w++)
            if (z != w && M[size_t(z) * D + w] != cplx(0.0, 0.0)) return false;
    return true;
}

}  // namespace

Op op_of_gate(const qs_gate& g, int n, const double* theta) {
    DenseOp d = dense_of_gate(g, n, theta);
    Op op;
    op.targets = d.targets;
    op.controls = d.controls;
    op.cvals = d.cvals;
    const int D = 1 << int(d.targets.size());

    auto make_pauli = [&](const int* ids, int m) {
        op.kind = OpKind::Pauli;
        op.targets.clear();
        for (int j = 0; j < m; j++) {
            const int q = d.targets[j];
            if (ids[j] == 1 || ids[j] == 2) op.xmask |= 1ull << q;
            if (ids[j] == 2 || ids[j] == 3) op.zmask |= 1ull << q;
        }
    };
    bool named = g.kind == QS_GATE_NAMED;
    if ((named && (g.named == QS_NAMED_X || g.named == QS_NAMED_CNOT || g.named == QS_NAMED_TOFFOLI))) {
        int id = 1;
        make_pauli(&id, 1);
        return op;
    }
    if (named && g.named == QS_NAMED_Y) {
        int id = 2;
        make_pauli(&id, 1);
        return op;
    }
    if (g.kind == QS_GATE_PAULI) {
        make_pauli(g.pauli, g.m);
        if (op.xmask == 0 && op.zmask == 0) {   // identity string
            op.kind = OpKind::Phase;
            op.targets.clear();
            op.phase = 1.0;
        }
        return op;
    }
    if (named && (g.named == QS_NAMED_SWAP || g.named == QS_NAMED_FREDKIN)) {
        op.kind = OpKind::Swap;
        return op;
    }
    if (named && g.named == QS_NAMED_PAULIROT) {
        // a string with an X or Y factor: one pass over amplitude pairs whatever its length
        // (Z strings stay diagonal gates below)
        uint64_t xm = 0, zm = 0;
        for (int j = 0; j < g.m; j++) {
            const int id = g.pauli[j], q = d.targets[j];
            if (id == 1 || id == 2) xm |= 1ull << q;
            if (id == 2 || id == 3) zm |= 1ull << q;
        }
        if (xm) {
            op.kind = OpKind::PauliRot;
            op.targets.clear();
            op.xmask = xm;
            op.zmask = zm;
            op.angle = angle(g, theta);
            return op;
        }
    }
    if (is_diagonal(d.mat, D)) {
        std::vector<cplx> diag(D);
        for (int i = 0; i < D; i++) diag[i] = d.mat[size_t(i) * D + i];
        int hot;
        if (as_phase(diag, &hot)) {
            // fix every target bit to the bits of `hot`: targets join the controls
            op.kind = OpKind::Phase;
            op.phase = diag[hot];
            for (size_t j = 0; j < d.targets.size(); j++) {
                op.controls.push_back(d.targets[j]);
                op.cvals.push_back((hot >> j) & 1);
            }
            op.targets.clear();
        } else {
            op.kind = OpKind::Diag;
            op.data = diag;
        }
        return op;
    }
    op.kind = OpKind::Dense;
    op.data = d.mat;
    return op;
}

namespace {
std::atomic<long long> g_alloc_held{0};
std::atomic<long long> g_alloc_fail_after{-1};
// true when this allocation is the one the test hook makes fail
bool injected_failure() {
    long long k = g_alloc_fail_after.load();
    while (k >= 0) {
        if (g_alloc_fail_after.compare_exchange_weak(k, k - 1)) return k == 0;
    }
    return false;
}
}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_alloc_held++;
    return e;
}
cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t st) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) g_alloc_held++;
    return e;
}
cudaError_t host_malloc_pinned_raw(void** p, size_t bytes) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_alloc_held++;
    return e;
}
cudaError_t dev_free(void* p) {
    if (!p) return cudaSuccess;
    g_alloc_held--;
    return cudaFree(p);
}
cudaError_t dev_free_async(void* p, cudaStream_t st) {
    if (!p) return cudaSuccess;
    g_alloc_held--;
    return cudaFreeAsync(p, st);
}
cudaError_t host_free_pinned(void* p) {
    if (!p) return cudaSuccess;
    g_alloc_held--;
    return cudaFreeHost(p);
}
void set_alloc_failure(long long after) { g_alloc_fail_after.store(after < 0 ? -1 : after); }
long long allocations_held() { return g_alloc_held.load(); }

int current_device() {
    int dev = 0;
    QS_TRY_CUDA(cudaGetDevice(&dev));
    QS_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index out of range");
    return dev;
}

namespace {
// 0: not set (the default, 8 rows, applies)
std::atomic<int> g_tile_rows[kMaxDevices][3][3];
}
int dense_tile_rows(Arith ar, int m) {
    if (m < 4 || m > 6) return 8;
    const int r = g_tile_rows[current_device()][int(ar)][m - 4].load();
    return r ? r : 8;
}
void set_dense_tile_rows(Arith ar, int m, int rows) {
    QS_REQUIRE(m >= 4 && m <= 6, "tile rows are set for 4..6 targets");
    QS_REQUIRE(rows == 0 || rows == 4 || rows == 8 || rows == 16, "tile rows must be 4, 8 or 16 (0: default)");
    g_tile_rows[current_device()][int(ar)][m - 4].store(rows);
}
bool dense_tile_rows_tuned(Arith ar, int m) {
    return m >= 4 && m <= 6 && g_tile_rows[current_device()][int(ar)][m - 4].load() != 0;
}

int device_sms() {
    static std::mutex mu;
    static int sms[kMaxDevices] = {};
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(mu);
    if (!sms[dev]) {
        int s = 0;
        QS_TRY_CUDA(cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev));
        sms[dev] = s > 0 ? s : 1;
    }
    return sms[dev];
}

IndexPlan make_index_plan(int n, const std::vector<int>& fixed, uint64_t setmask) {
    IndexPlan p;
    std::vector<int> f = fixed;
    std::sort(f.begin(), f.end());
    QS_REQUIRE(int(f.size()) <= kMaxFixed, "too many fixed qubits");
    QS_REQUIRE(int(f.size()) <= n, "more fixed qubits than qubits");
    p.nfix = int(f.size());
    for (int j = 0; j < p.nfix; j++) p.fixpos[j] = f[j];
    p.n_iter = 1ull << (n - p.nfix);
    p.setmask = setmask;
    return p;
}

}  // namespace qs
