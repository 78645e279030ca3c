// Gate fusion (Sec. 5.4, circuit optimisation): neighbouring gates are merged into one
// dense gate on the union of their qubits, so that a block of gates costs one pass over
// the state instead of one pass per gate; merging multiplies the arithmetic by
// 2^(|M1 u M2| - |M1|) and halves the memory traffic.
//
// Planner (the light strategy with a width budget k): every qubit belongs to at most one
// open block. A gate whose qubits (targets and controls) meet a set S of open blocks joins
// them when the union of their qubits has at most k elements; the blocks of S are pairwise
// disjoint and therefore commute, so merging them and appending the gate is exact. When the
// union is too wide, the blocks of S are emitted and the gate opens a new block. Open
// blocks that do not touch the gate commute with it and stay open. Merged matrices follow
// merge(g1, g2) = g2 * g1 (g1 applied first), built in FP64 by applying each gate to the
// columns of the block matrix.
#include <algorithm>
#include <cstring>

#include "qsim_internal.h"

namespace qs {

namespace {

struct OpenBlock {
    uint64_t mask = 0;
    std::vector<int> gates;  // indices into the circuit, in application order
    int order = 0;           // creation order (emission order among simultaneous closes)
};

// Apply dense op d (targets/controls given as positions inside `qubits`) to every column of
// the 2^w x 2^w row-major matrix M: M <- G M.
void apply_to_columns(std::vector<cplx>& M, int w, const DenseOp& d, const std::vector<int>& local_t,
                      const std::vector<int>& local_c) {
    const int D = 1 << w;
    const int m = int(local_t.size());
    const int dm = 1 << m;
    uint64_t tmask = 0, cmask = 0, cval = 0;
    for (int j = 0; j < m; j++) tmask |= 1ull << local_t[j];
    for (size_t j = 0; j < local_c.size(); j++) {
        cmask |= 1ull << local_c[j];
        if (d.cvals[j]) cval |= 1ull << local_c[j];
    }
    std::vector<uint64_t> off(dm);
    for (int a = 0; a < dm; a++) {
        uint64_t o = 0;
        for (int j = 0; j < m; j++)
            if ((a >> j) & 1) o |= 1ull << local_t[j];
        off[a] = o;
    }
    std::vector<cplx> in(dm), out(dm);
    for (int col = 0; col < D; col++) {
        for (int r0 = 0; r0 < D; r0++) {
            if (uint64_t(r0) & tmask) continue;
            if ((uint64_t(r0) & cmask) != cval) continue;
            for (int a = 0; a < dm; a++) in[a] = M[size_t(r0 + off[a]) * D + col];
            for (int z = 0; z < dm; z++) {
                cplx acc = 0.0;
                for (int a = 0; a < dm; a++) acc += d.mat[size_t(z) * dm + a] * in[a];
                out[z] = acc;
            }
            for (int z = 0; z < dm; z++) M[size_t(r0 + off[z]) * D + col] = out[z];
        }
    }
}

uint64_t gate_mask(const qs_gate& g) {
    uint64_t m = 0;
    for (int j = 0; j < g.m; j++) m |= 1ull << g.targets[j];
    for (int j = 0; j < g.mc; j++) m |= 1ull << g.controls[j];
    return m;
}

bool dense_is_diagonal(const DenseOp& d) {
    const int D = 1 << int(d.targets.size());
    for (int z = 0; z < D; z++)
        for (int w = 0; w < D; w++)
            if (z != w && d.mat[size_t(z) * D + w] != cplx(0.0, 0.0)) return false;
    return true;
}

void emit(const OpenBlock& b, const qs_circuit* c, FusionPlan& plan) {
    FusedBlock fb;
    for (int q = 0; q < 64; q++)
        if ((b.mask >> q) & 1) fb.qubits.push_back(q);
    fb.n_gates = int(b.gates.size());
    if (b.gates.size() == 1) {
        fb.single_gate = b.gates[0];
        plan.blocks.push_back(std::move(fb));
        return;
    }
    const int w = int(fb.qubits.size());
    const int D = 1 << w;
    fb.mat.assign(size_t(D) * D, 0.0);
    for (int i = 0; i < D; i++) fb.mat[size_t(i) * D + i] = 1.0;
    bool diag = true;
    for (int gi : b.gates) {
        const qs_gate& g = c->gates[gi];
        DenseOp d = dense_of_gate(g, c->n, nullptr);
        diag = diag && dense_is_diagonal(d);
        std::vector<int> lt, lc;
        auto local = [&](int q) { return int(std::find(fb.qubits.begin(), fb.qubits.end(), q) - fb.qubits.begin()); };
        for (int t : d.targets) lt.push_back(local(t));
        for (int q : d.controls) lc.push_back(local(q));
        apply_to_columns(fb.mat, w, d, lt, lc);
    }
    fb.diagonal = diag;
    plan.blocks.push_back(std::move(fb));
}

}  // namespace

FusionPlan plan_fusion(const qs_circuit* c, int k) {
    QS_REQUIRE(c != nullptr, "null circuit");
    QS_REQUIRE(c->n >= 1 && c->n <= QS_MAX_QUBITS, "qubit count out of range");
    QS_REQUIRE(c->n_gates >= 0 && (c->n_gates == 0 || c->gates != nullptr), "null gate array");
    QS_REQUIRE(k >= 1 && k <= QS_MAX_TARGETS, "fusion width must be in 1..6");
    FusionPlan plan;
    plan.n = c->n;
    plan.k = k;
    plan.n_source_gates = c->n_gates;
    std::vector<OpenBlock> open;          // slots; empty mask = free
    std::vector<int> owner(c->n, -1);     // qubit -> slot
    int counter = 0;
    auto close_slots = [&](std::vector<int> slots) {
        std::sort(slots.begin(), slots.end(), [&](int a, int b) { return open[a].order < open[b].order; });
        for (int s : slots) {
            emit(open[s], c, plan);
            for (int q = 0; q < c->n; q++)
                if (owner[q] == s) owner[q] = -1;
            open[s].mask = 0;
            open[s].gates.clear();
        }
    };
    for (int i = 0; i < c->n_gates; i++) {
        const qs_gate& g = c->gates[i];
        QS_REQUIRE(g.m >= 1 && g.m <= QS_MAX_TARGETS, "target count out of range (1..6)");
        check_qubits(c->n, g.targets, g.m, g.controls, g.mc);
        const uint64_t gm = gate_mask(g);
        std::vector<int> touched;
        uint64_t uni = gm;
        for (int q = 0; q < c->n; q++)
            if (((gm >> q) & 1) && owner[q] >= 0 &&
                std::find(touched.begin(), touched.end(), owner[q]) == touched.end()) {
                touched.push_back(owner[q]);
                uni |= open[owner[q]].mask;
            }
        int slot;
        if (__builtin_popcountll(uni) <= k) {
            // merge the touched blocks (disjoint, commuting) and append the gate
            OpenBlock nb;
            nb.mask = uni;
            std::sort(touched.begin(), touched.end(), [&](int a, int b) { return open[a].order < open[b].order; });
            nb.order = touched.empty() ? counter++ : open[touched[0]].order;
            for (int s : touched) {
                nb.gates.insert(nb.gates.end(), open[s].gates.begin(), open[s].gates.end());
                open[s].mask = 0;
                open[s].gates.clear();
            }
            nb.gates.push_back(i);
            slot = touched.empty() ? -1 : touched[0];
            if (slot < 0) {
                for (size_t s = 0; s < open.size(); s++)
                    if (open[s].mask == 0) { slot = int(s); break; }
                if (slot < 0) { open.emplace_back(); slot = int(open.size()) - 1; }
            }
            for (int q = 0; q < c->n; q++)
                if (((uni >> q) & 1)) owner[q] = slot;
            open[slot] = std::move(nb);
        } else {
            close_slots(touched);
            OpenBlock nb;
            nb.mask = gm;
            nb.order = counter++;
            nb.gates.push_back(i);
            slot = -1;
            for (size_t s = 0; s < open.size(); s++)
                if (open[s].mask == 0) { slot = int(s); break; }
            if (slot < 0) { open.emplace_back(); slot = int(open.size()) - 1; }
            open[slot] = std::move(nb);
            for (int q = 0; q < c->n; q++)
                if ((gm >> q) & 1) owner[q] = slot;
        }
    }
    std::vector<int> rest;
    for (size_t s = 0; s < open.size(); s++)
        if (open[s].mask) rest.push_back(int(s));
    close_slots(rest);
    // keep copies of the gates that stay unfused (their matrices are rebuilt at launch)
    for (auto& b : plan.blocks) {
        if (b.single_gate < 0) continue;
        qs_gate g = c->gates[b.single_gate];
        std::vector<double> mat;
        if (g.kind == QS_GATE_DENSE || g.kind == QS_GATE_DIAG) {
            const size_t D = size_t(1) << g.m;
            const size_t cnt = g.kind == QS_GATE_DENSE ? D * D : D;
            mat.assign(g.mat, g.mat + 2 * cnt);
        }
        plan.source_mats.push_back(std::move(mat));
        plan.source.push_back(g);
        b.single_gate = int(plan.source.size()) - 1;
    }
    for (size_t i = 0; i < plan.source.size(); i++)
        if (!plan.source_mats[i].empty()) plan.source[i].mat = plan.source_mats[i].data();
    return plan;
}

}  // namespace qs
