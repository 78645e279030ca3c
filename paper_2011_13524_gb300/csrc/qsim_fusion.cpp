// Gate fusion (Sec. 5.4, circuit optimisation): neighbouring gates are merged into one
// dense gate on the union of their qubits, so that a block of gates costs one pass over
// the state instead of one pass per gate; merging multiplies the arithmetic by
// 2^(|M1 u M2| - |M1|) and halves the memory traffic.
//
// Partitions of the gate list into blocks of at most k qubits are formed by two methods (the
// second with three lookahead depths) and the one with the fewest blocks is kept (ties: the
// first).
//
// 1. Open-block greedy (the light strategy with a width budget k): every qubit belongs to at
//    most one open block. A gate whose qubits (targets and controls) meet a set S of open
//    blocks joins them when the union of their qubits has at most k elements; the blocks of S
//    are pairwise disjoint and therefore commute, so merging them and appending the gate is
//    exact. When the union is too wide, the blocks of S are emitted and the gate opens a new
//    block. Open blocks that do not touch the gate commute with it and stay open.
// 2. Frontier growth: a block starts from the earliest gate not yet emitted and takes every
//    later gate whose qubits lie inside the block's qubit set Q and whose earlier gates on
//    those qubits are all emitted or already in the block. While |Q| < k the block widens by
//    the ready gate whose new qubit set lets the most gates join. A block built this way is
//    closed under "comes earlier on a shared qubit", so emitting it before the gates that remain
//    only moves it past gates on other qubits, with which it commutes: the product is exact.
//
// Merged matrices follow merge(g1, g2) = g2 * g1 (g1 applied first), built in FP64 by
// applying each gate, in circuit order, to the columns of the block matrix.
#include <algorithm>
#include <cstring>
#include <exception>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>

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

// Qubits of a gate on which it commutes with Z, X or Y (block-diagonal in that single-qubit
// basis). Two gates whose shared qubits all carry a common such basis commute: both are then
// block-diagonal in the joint eigenbasis of the shared qubits and act on disjoint qubits
// otherwise. Controls commute with Z; named gates take their table's structure; a dense
// matrix is tested entry by entry.
struct GateTags {
    uint64_t zc = 0, xc = 0, yc = 0;
};

GateTags gate_tags(const qs_gate& g, int n) {
    GateTags t;
    for (int j = 0; j < g.mc; j++) t.zc |= 1ull << g.controls[j];
    uint64_t tm = 0;
    for (int j = 0; j < g.m; j++) tm |= 1ull << g.targets[j];
    auto pauli_tag = [&](int id, int q) {
        const uint64_t b = 1ull << q;
        if (id == 0) { t.zc |= b; t.xc |= b; t.yc |= b; }
        else if (id == 1) t.xc |= b;
        else if (id == 2) t.yc |= b;
        else t.zc |= b;
    };
    if (g.kind == QS_GATE_DIAG) {
        t.zc |= tm;
        return t;
    }
    if (g.kind == QS_GATE_PAULI) {
        for (int j = 0; j < g.m; j++) pauli_tag(g.pauli[j], g.targets[j]);
        return t;
    }
    if (g.kind == QS_GATE_NAMED) {
        switch (g.named) {
            case QS_NAMED_Z: case QS_NAMED_S: case QS_NAMED_SDAG: case QS_NAMED_T: case QS_NAMED_TDAG:
            case QS_NAMED_RZ: case QS_NAMED_U1: case QS_NAMED_CZ:
                t.zc |= tm;
                return t;
            case QS_NAMED_X: case QS_NAMED_SQRTX: case QS_NAMED_SQRTXDAG: case QS_NAMED_RX:
            case QS_NAMED_CNOT: case QS_NAMED_TOFFOLI:
                t.xc |= tm;
                return t;
            case QS_NAMED_Y: case QS_NAMED_SQRTY: case QS_NAMED_SQRTYDAG: case QS_NAMED_RY:
                t.yc |= tm;
                return t;
            case QS_NAMED_PAULIROT:
                for (int j = 0; j < g.m; j++) pauli_tag(g.pauli[j], g.targets[j]);
                return t;
            default:
                return t;  // H, U2, U3, SWAP, FREDKIN: no common basis claimed
        }
    }
    // dense matrix: test each target bit
    const DenseOp d = dense_of_gate(g, n, nullptr);
    const int m = int(d.targets.size()), D = 1 << m;
    double scale = 0.0;
    for (const cplx& v : d.mat) scale = std::max(scale, std::abs(v));
    const double tol = 1e-14 * std::max(scale, 1.0);
    for (int j = 0; j < m; j++) {
        const int b = 1 << j;
        bool z = true, x = true, y = true;
        for (int r = 0; r < D && (z || x || y); r++)
            for (int c = 0; c < D; c++) {
                const cplx v = d.mat[size_t(r) * D + c];
                if (((r ^ c) & b) && std::abs(v) > tol) z = false;
                // X K X = K: K[r][c] = K[r^b][c^b]; Y K Y = K: the same up to the sign (-1)^(bit r + bit c)
                const cplx w = d.mat[size_t(r ^ b) * D + (c ^ b)];
                if (std::abs(v - w) > tol) x = false;
                const double sg = (((r & b) != 0) != ((c & b) != 0)) ? -1.0 : 1.0;
                if (std::abs(v - sg * w) > tol) y = false;
            }
        const uint64_t q = 1ull << d.targets[j];
        if (z) t.zc |= q;
        if (x) t.xc |= q;
        if (y) t.yc |= q;
    }
    return t;
}

bool dense_is_diagonal(const DenseOp& d) {
    const int D = 1 << int(d.targets.size());
    for (int z = 0; z < D; z++)
        for (int w = 0; w < D; w++)
            if (z != w && d.mat[size_t(z) * D + w] != cplx(0.0, 0.0)) return false;
    return true;
}

FusedBlock emit(const OpenBlock& b, const qs_circuit* c, const double* theta) {
    FusedBlock fb;
    for (int q = 0; q < 64; q++)
        if ((b.mask >> q) & 1) fb.qubits.push_back(q);
    fb.n_gates = int(b.gates.size());
    if (b.gates.size() == 1) {
        fb.single_gate = b.gates[0];
        return fb;
    }
    const int w = int(fb.qubits.size());
    const int D = 1 << w;
    fb.mat.assign(size_t(D) * D, 0.0);
    for (int i = 0; i < D; i++) fb.mat[size_t(i) * D + i] = 1.0;
    bool diag = true;
    for (int gi : b.gates) {
        const qs_gate& g = c->gates[gi];
        DenseOp d = dense_of_gate(g, c->n, theta);
        diag = diag && dense_is_diagonal(d);
        std::vector<int> lt, lc;
        auto local = [&](int q) { return int(std::find(fb.qubits.begin(), fb.qubits.end(), q) - fb.qubits.begin()); };
        for (int t : d.targets) lt.push_back(local(t));
        for (int q : d.controls) lc.push_back(local(q));
        apply_to_columns(fb.mat, w, d, lt, lc);
    }
    fb.diagonal = diag;
    return fb;
}

// Partition 1: open-block greedy. Returns the blocks in emission order.
std::vector<OpenBlock> partition_greedy(const qs_circuit* c, const std::vector<uint64_t>& masks, int k) {
    std::vector<OpenBlock> out;
    std::vector<OpenBlock> open;          // slots; empty mask = free
    std::vector<int> owner(c->n, -1);     // qubit -> slot
    int counter = 0;
    auto free_slot = [&]() {
        for (size_t s = 0; s < open.size(); s++)
            if (open[s].mask == 0) return int(s);
        open.emplace_back();
        return int(open.size()) - 1;
    };
    auto close_slots = [&](std::vector<int> slots) {
        std::sort(slots.begin(), slots.end(), [&](int a, int b) { return open[a].order < open[b].order; });
        for (int s : slots) {
            out.push_back(open[s]);
            for (int q = 0; q < c->n; q++)
                if (owner[q] == s) owner[q] = -1;
            open[s].mask = 0;
            open[s].gates.clear();
        }
    };
    for (int i = 0; i < c->n_gates; i++) {
        const uint64_t gm = masks[i];
        std::vector<int> touched;
        uint64_t uni = gm;
        for (int q = 0; q < c->n; q++)
            if (((gm >> q) & 1) && owner[q] >= 0 &&
                std::find(touched.begin(), touched.end(), owner[q]) == touched.end()) {
                touched.push_back(owner[q]);
                uni |= open[owner[q]].mask;
            }
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
            const int slot = touched.empty() ? free_slot() : touched[0];
            for (int q = 0; q < c->n; q++)
                if ((uni >> q) & 1) owner[q] = slot;
            open[slot] = std::move(nb);
        } else {
            close_slots(touched);
            OpenBlock nb;
            nb.mask = gm;
            nb.order = counter++;
            nb.gates.push_back(i);
            const int slot = free_slot();
            open[slot] = std::move(nb);
            for (int q = 0; q < c->n; q++)
                if ((gm >> q) & 1) owner[q] = slot;
        }
    }
    std::vector<int> rest;
    for (size_t s = 0; s < open.size(); s++)
        if (open[s].mask) rest.push_back(int(s));
    close_slots(rest);
    return out;
}

// Partition 2: frontier growth. `rem` lists the gates not yet emitted, in circuit order. A scan
// over it keeps, for the gates it passes that stay outside the block, the qubits they touch
// (`blocked`) and, per qubit, whether all of them commute with Z, X or Y there (bz, bx, by). A
// later gate may join the block when on each of its blocked qubits it shares one of those bases:
// it then commutes with every gate it moves ahead of. Membership: gate g is in the block when
// in[g] == blk, or, during a trial widening, when trial[g] == tid.
struct Frontier {
    const std::vector<uint64_t>& masks;
    const std::vector<GateTags>& tags;
    const std::vector<int>& rem;
    uint64_t all;
    std::vector<int>& in;
    std::vector<int>& trial;
    int blk = 0;
    int tid = 0;
    long long visits = 0;  // gates visited by close_over and widening so far: a deterministic work count
    struct Scan {
        uint64_t blocked = 0, bz = ~0ull, bx = ~0ull, by = ~0ull;
        bool ready(uint64_t m, const GateTags& t) const {
            const uint64_t ok = (t.zc & bz) | (t.xc & bx) | (t.yc & by);
            return (m & blocked & ~ok) == 0;
        }
        void pass(uint64_t m, const GateTags& t) {
            blocked |= m;
            bz &= ~(m & ~t.zc);
            bx &= ~(m & ~t.xc);
            by &= ~(m & ~t.yc);
        }
        // no gate on these qubits can be ready any more
        bool closed(uint64_t q) const { return (blocked & q) == q && ((bz | bx | by) & q) == 0; }
    };
    bool member(int g, bool use_trial) const { return in[g] == blk || (use_trial && trial[g] == tid); }
    // Adds to the block (or to the trial) every gate that can join with qubit set q.
    int close_over(uint64_t q, bool use_trial) {
        Scan sc;
        int added = 0;
        for (int g : rem) {
            visits++;
            if (member(g, use_trial)) continue;
            const uint64_t m = masks[g];
            if ((m & ~q) == 0 && sc.ready(m, tags[g])) {
                if (use_trial) trial[g] = tid;
                else in[g] = blk;
                added++;
            } else {
                sc.pass(m, tags[g]);
                if (sc.closed(q)) break;
            }
        }
        return added;
    }
    // Distinct qubit sets q | m of the ready gates that widen q without exceeding k qubits; with
    // id >= 0 the gates of trial id count as members too.
    std::vector<uint64_t> widening(uint64_t q, int k, int id = -1) {
        std::vector<uint64_t> cand;
        Scan sc;
        for (int g : rem) {
            visits++;
            if (in[g] == blk || (id >= 0 && trial[g] == id)) continue;
            const uint64_t m = masks[g];
            if ((m & ~q) && __builtin_popcountll(q | m) <= k && sc.ready(m, tags[g]) &&
                std::find(cand.begin(), cand.end(), q | m) == cand.end())
                cand.push_back(q | m);
            sc.pass(m, tags[g]);
            if (sc.closed(all)) break;
        }
        return cand;
    }
};

// Lookahead over widenings, for a fixed block membership B. The gates a qubit set X can hold,
// closure(X), grow with X, and one ordered scan finds them (a gate joins when it lies in X and no
// earlier non-member on its qubits blocks it). So the gates a chain of widenings q -> u -> u2 ...
// adds in total are |closure(last) \ B|, and the search needs, per distinct X, only that count
// and X's widenings (given B and closure(X)); both are memoized until B changes.
struct Lookahead {
    Frontier& f;
    int k;
    std::unordered_map<uint64_t, int> cnt;
    std::unordered_map<uint64_t, std::vector<uint64_t>> wid;
    void reset() {
        cnt.clear();
        wid.clear();
    }
    int count(uint64_t X) {
        auto it = cnt.find(X);
        if (it != cnt.end()) return it->second;
        f.tid++;
        const int v = f.close_over(X, true);
        cnt.emplace(X, v);
        return v;
    }
    std::vector<uint64_t> widenings(uint64_t X) {
        auto it = wid.find(X);
        if (it != wid.end()) return it->second;
        f.tid++;
        f.close_over(X, true);
        std::vector<uint64_t> w = f.widening(X, k, f.tid);
        wid.emplace(X, w);
        return w;
    }
    // the most gates that `levels` more widenings of X add beyond closure(X)
    int more(uint64_t X, int levels) {
        const int cx = count(X);
        int best = 0;
        for (uint64_t u2 : widenings(X)) {
            int got = count(u2) - cx;
            if (levels > 1 && __builtin_popcountll(u2) < k) got += more(u2, levels - 1);
            best = std::max(best, got);
        }
        return best;
    }
};

// depth: 1 picks each widening by the gates it absorbs; d > 1 by the best total after d - 1
// more widenings (each trial runs on top of the previous one's membership).
// A search that would visit more than max_visits gates is abandoned (empty result).
std::vector<OpenBlock> partition_frontier(const qs_circuit* c, const std::vector<uint64_t>& masks,
                                          const std::vector<GateTags>& tags, int k, int depth = 1,
                                          long long max_visits = -1) {
    std::vector<OpenBlock> out;
    std::vector<int> rem(c->n_gates);
    for (int i = 0; i < c->n_gates; i++) rem[i] = i;
    std::vector<int> in(c->n_gates, -1), trial(c->n_gates, -1);
    const uint64_t all = c->n >= 64 ? ~0ull : ((1ull << c->n) - 1);
    Frontier f{masks, tags, rem, all, in, trial};
    Lookahead la{f, k, {}, {}};
    while (!rem.empty()) {
        if (max_visits >= 0 && f.visits > max_visits) return {};
        uint64_t q = masks[rem[0]];
        in[rem[0]] = f.blk;
        f.close_over(q, false);
        while (__builtin_popcountll(q) < k) {
            const std::vector<uint64_t> cand = f.widening(q, k);
            if (cand.empty()) break;
            la.reset();  // the block's membership changed
            int best = -1;
            uint64_t best_q = 0;
            for (uint64_t u : cand) {
                int got = la.count(u);
                if (depth > 1 && __builtin_popcountll(u) < k) got += la.more(u, depth - 1);
                // more gates first, then the narrower set
                if (got > best || (got == best && __builtin_popcountll(u) < __builtin_popcountll(best_q))) {
                    best = got;
                    best_q = u;
                }
            }
            q = best_q;
            f.close_over(q, false);
        }
        OpenBlock b;
        std::vector<int> keep;
        for (int g : rem) {
            if (in[g] == f.blk) {
                b.gates.push_back(g);
                b.mask |= masks[g];
            } else {
                keep.push_back(g);
            }
        }
        out.push_back(std::move(b));
        rem.swap(keep);
        f.blk++;
    }
    return out;
}

}  // namespace

// The partition depends only on the qubit sets of the gates and on k, not on angles or matrix
// entries: a circuit run again with new parameters (an optimisation loop, the adjoint's forward
// pass) reuses it. A few recent partitions are kept.
namespace {
struct PartitionKey {
    int n = 0, k = 0;
    std::vector<uint64_t> masks;  // per gate: qubits, then the Z, X, Y commuting-basis masks
    bool operator==(const PartitionKey& o) const { return n == o.n && k == o.k && masks == o.masks; }
};
std::mutex g_part_mu;
std::list<std::pair<PartitionKey, std::vector<OpenBlock>>> g_part_cache;
constexpr size_t kPartCacheSize = 16;

std::vector<OpenBlock> partition(const qs_circuit* c, const std::vector<uint64_t>& masks,
                                 const std::vector<GateTags>& tags, int k) {
    PartitionKey key{c->n, k, masks};
    for (const GateTags& t : tags) {
        key.masks.push_back(t.zc);
        key.masks.push_back(t.xc);
        key.masks.push_back(t.yc);
    }
    {
        std::lock_guard<std::mutex> lk(g_part_mu);
        for (auto it = g_part_cache.begin(); it != g_part_cache.end(); ++it)
            if (it->first == key) {
                g_part_cache.splice(g_part_cache.begin(), g_part_cache, it);
                return it->second;
            }
    }
    // four partitions, independent of each other, on host threads: greedy, frontier growth, and
    // frontier growth with a wider lookahead (depth 2 always, depth 3 within a budget of visited
    // gates, about 0.1 s); the one with the fewest blocks is kept (ties: the earlier one)
    std::vector<OpenBlock> cand[4];
    std::exception_ptr err[4];
    auto run = [&](int i) {
        try {
            if (i == 0)
                cand[0] = partition_greedy(c, masks, k);
            else if (i == 1)
                cand[1] = partition_frontier(c, masks, tags, k);
            else
                cand[i] = partition_frontier(c, masks, tags, k, i, i == 2 ? -1 : 15000000);
        } catch (...) {
            err[i] = std::current_exception();
        }
    };
    if (c->n_gates >= 64 && std::thread::hardware_concurrency() > 1) {
        std::vector<std::thread> pool;
        for (int i = 1; i < 4; i++) pool.emplace_back(run, i);
        run(0);
        for (auto& th : pool) th.join();
    } else {
        for (int i = 0; i < 4; i++) run(i);
    }
    for (auto& e : err)
        if (e) std::rethrow_exception(e);
    std::vector<OpenBlock> best = cand[1].size() < cand[0].size() ? std::move(cand[1]) : std::move(cand[0]);
    for (int i = 2; i < 4; i++)
        if (!cand[i].empty() && cand[i].size() < best.size()) best = std::move(cand[i]);
    std::lock_guard<std::mutex> lk(g_part_mu);
    g_part_cache.emplace_front(std::move(key), best);
    if (g_part_cache.size() > kPartCacheSize) g_part_cache.pop_back();
    return best;
}
}  // namespace

void clear_partition_cache() {
    std::lock_guard<std::mutex> lk(g_part_mu);
    g_part_cache.clear();
}

FusionPlan plan_fusion(const qs_circuit* c, int k, const double* theta) {
    QS_REQUIRE(c != nullptr, "null circuit");
    QS_REQUIRE(c->n >= 1 && c->n <= QS_MAX_QUBITS, "qubit count out of range");
    QS_REQUIRE(c->n_gates >= 0 && (c->n_gates == 0 || c->gates != nullptr), "null gate array");
    QS_REQUIRE(k >= 1 && k <= QS_MAX_TARGETS, "fusion width must be in 1..6");
    std::vector<uint64_t> masks(c->n_gates);
    std::vector<GateTags> tags(c->n_gates);
    for (int i = 0; i < c->n_gates; i++) {
        const qs_gate& g = c->gates[i];
        QS_REQUIRE(g.m >= 1 && g.m <= QS_MAX_TARGETS, "target count out of range (1..6)");
        check_qubits(c->n, g.targets, g.m, g.controls, g.mc);
        masks[i] = gate_mask(g);
        tags[i] = gate_tags(g, c->n);
    }
    FusionPlan plan;
    plan.n = c->n;
    plan.k = k;
    plan.n_source_gates = c->n_gates;
    // block matrices: independent of each other, built by several host threads for long plans
    const std::vector<OpenBlock> parts = partition(c, masks, tags, k);
    plan.blocks.resize(parts.size());
    size_t work = 0;
    for (const OpenBlock& blk : parts) work += blk.gates.size() << (2 * __builtin_popcountll(blk.mask));
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nth = work < (1u << 16) ? 1u : std::min<unsigned>(std::min(hw, 8u), unsigned(parts.size()));
    if (nth <= 1) {
        for (size_t i = 0; i < parts.size(); i++) plan.blocks[i] = emit(parts[i], c, theta);
    } else {
        std::vector<std::thread> pool;
        std::vector<std::exception_ptr> errs(nth);
        for (unsigned w = 0; w < nth; w++)
            pool.emplace_back([&, w]() {
                try {
                    for (size_t i = w; i < parts.size(); i += nth) plan.blocks[i] = emit(parts[i], c, theta);
                } catch (...) {
                    errs[w] = std::current_exception();
                }
            });
        for (auto& th : pool) th.join();
        for (auto& e : errs)
            if (e) std::rethrow_exception(e);
    }
    // keep copies of the gates that stay unfused (their matrices are rebuilt at launch)
    for (auto& b : plan.blocks) {
        if (b.single_gate < 0) continue;
        qs_gate g = c->gates[b.single_gate];
        if (theta && g.param_index >= 0) g.params[0] = theta[g.param_index];  // the angle this plan was made for
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
