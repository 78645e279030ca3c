"""CPU-only checks of the C ABI library: it builds, loads, exports every function the header
declares, validates arguments without a GPU, and its host-side fusion planner produces block
matrices whose product equals the unfused circuit (checked with the oracle)."""
import ctypes
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W
import paper_2011_13524_gb300 as qs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsim_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:qs_status|const char\*)\s+(qs_\w+)\(", text, re.M)))


def test_header_declares_and_library_exports_every_function():
    names = declared_functions()
    assert len(names) >= 20
    L = qs.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(qs.exported_symbols())


def test_version_and_error_message():
    assert b"sm_103a" in qs.lib().qs_version()
    rc = qs.lib().qs_set_c128_math(7)
    assert rc == qs.QS_ERR_INVALID_ARG
    assert b"mode" in qs.lib().qs_last_error()
    old = qs.get_c128_math()
    qs.set_c128_math(qs.QS_MATH_FP64)
    assert qs.get_c128_math() == qs.QS_MATH_FP64
    qs.set_c128_math(old)
    rc = qs.lib().qs_set_tensor_cores(1)  # no such path
    assert rc == qs.QS_ERR_INVALID_ARG


def test_library_defaults():
    """A fresh process: complex128 gates run in double-float arithmetic with the tensor-core
    blocks of both dtypes on (the configuration the benchmark times), read through the ABI."""
    code = ("import paper_2011_13524_gb300 as qs; "
            "print(qs.get_c128_math(), qs.get_tensor_cores())")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, check=True)
    math_mode, mask = map(int, out.stdout.split())
    assert math_mode == qs.QS_MATH_DF
    assert mask == qs.QS_TENSOR_C128 | qs.QS_TENSOR_C64X


def test_invalid_arguments_without_gpu():
    L = qs.lib()
    h = ctypes.c_void_p()
    assert L.qs_create_state(0, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert L.qs_create_state(40, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert L.qs_create_state(4, 9, None, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert L.qs_wrap_state(None, 4, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert L.qs_wrap_state(ctypes.c_void_p(8), 4, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert L.qs_destroy_state(None) == qs.QS_OK
    assert L.qs_apply_gate(None, None) == qs.QS_ERR_INVALID_ARG
    # planner validation (host only)
    bad = W.Circuit(3, [W.Gate("CNOT", (1,), controls=(1,), control_values=(1,))])
    c, keep = qs.make_circuit(bad)
    assert L.qs_plan_fusion(ctypes.byref(c), 3, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    assert b"control" in L.qs_last_error()
    ok = W.Circuit(3, [W.Gate("H", (0,))])
    c, keep = qs.make_circuit(ok)
    assert L.qs_plan_fusion(ctypes.byref(c), 7, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG
    out_of_range = W.Circuit(3, [W.Gate("H", (3,))])
    c, keep = qs.make_circuit(out_of_range)
    assert L.qs_plan_fusion(ctypes.byref(c), 2, ctypes.byref(h)) == qs.QS_ERR_INVALID_ARG


def run_plan_with_oracle(plan, n):
    psi = oracle.zero_state(n)
    for b in range(plan.n_blocks):
        t, M = plan.block(b)
        oracle.apply_matrix(psi, n, t, M)
    return psi


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_fusion_plan_product_equals_circuit(k):
    """Merging is exact algebra (Sec. 5.4): applying the planned blocks (with the oracle)
    reproduces the unfused circuit."""
    n = 8
    for circ in [W.u3cz_circuit(n, 4, 3), W.Circuit(n, W.random_gate_suite(n, 17)),
                 W.hea_circuit(n, 2, 5), W.rzrxrz_cnot_circuit(n, 2, 9)]:
        ref = oracle.run_circuit(circ)
        plan = qs.FusedCircuit(circ, k)
        assert plan.n_source_gates == len(circ.gates)
        widest = max(len(g.targets) + len(g.controls) for g in circ.gates)
        assert all(w <= max(k, widest) for w in plan.widths())   # a wider gate stays alone
        got = run_plan_with_oracle(plan, n)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_fusion_reduces_block_count():
    c = W.u3cz_circuit(30, 20, 1)
    counts = {k: qs.FusedCircuit(c, k).n_blocks for k in (1, 2, 3, 4, 5, 6)}
    assert counts[1] < len(c.gates)
    assert counts[2] < counts[1] and counts[4] < counts[2] and counts[6] <= counts[5]
    # frontier growth reorders gates on disjoint qubits: on the brickwork a 4-qubit block
    # covers two layers of a 4-qubit window (~11 gates), a 6-qubit block a light-cone triangle
    assert counts[4] <= 80 and counts[6] <= 42, counts


def test_fusion_benchmark_plans():
    """The plans of the benchmark workloads (host only): the depth-20 U3+CZ circuit at n = 30 in
    at most 74 / 53 / 36 blocks at k = 4 / 5 / 6, and 50 launches at k = 5 (its trailing diagonal
    blocks share one pass); the 20-layer ansatz at n = 20 in at most 35 blocks at k = 5. Planning
    twice from an empty partition cache gives the same plan."""
    c = W.u3cz_circuit(30, 20, 20201127)
    bound = {4: 74, 5: 53, 6: 36}
    for k, b in bound.items():
        assert qs.FusedCircuit(c, k).n_blocks <= b, k
    plan = qs.FusedCircuit(c, 5)
    assert sum(plan.block_cost(i, qs.QS_C128)[1] for i in range(plan.n_blocks)) <= 50
    first = [tuple(plan.block(i)[0]) for i in range(plan.n_blocks)]
    qs.clear_plan_cache()
    again = qs.FusedCircuit(c, 5)
    assert [tuple(again.block(i)[0]) for i in range(again.n_blocks)] == first
    assert qs.FusedCircuit(W.hea_circuit(20, 20, 20201127), 5).n_blocks <= 35


def commuting_mix_circuit(n, seed):
    """Gates that commute in several bases: diagonal layers (CZ, RZ, S, T, U1, controlled phases,
    DIAG), X-basis layers (RX, CNOT targets, sqrtX, X-string PAULIROT), Y rotations, PAULI and
    PAULIROT strings of mixed factors, dense matrices that equal such gates, and a few general
    gates (H, U3, SWAP) in between."""
    rng = W.SplitMix64(seed)
    gates = []
    def q():
        return int(rng.next_u64() % n)
    def two():
        a = q()
        b = (a + 1 + int(rng.next_u64() % (n - 1))) % n
        return a, b
    for layer in range(6):
        for _ in range(n):
            r = int(rng.next_u64() % 12)
            a, b = two()
            th = 2 * math.pi * rng.uniform()
            if r == 0:
                gates.append(W.Gate("CZ", (a, b)))
            elif r == 1:
                gates.append(W.Gate("RZ", (a,), params=(th,)))
            elif r == 2:
                gates.append(W.Gate("RX", (a,), params=(th,)))
            elif r == 3:
                gates.append(W.Gate("CNOT", (a,), controls=(b,), control_values=(1,)))
            elif r == 4:
                gates.append(W.Gate("RY", (a,), params=(th,)))
            elif r == 5:
                gates.append(W.Gate(["S", "T", "sqrtX", "sqrtY", "Z", "X"][int(rng.next_u64() % 6)], (a,)))
            elif r == 6:
                gates.append(W.Gate("U1", (a,), params=(th,), controls=(b,), control_values=(int(rng.next_u64() % 2),)))
            elif r == 7:
                gates.append(W.Gate("PAULIROT", (a, b), pauli=(1 + int(rng.next_u64() % 3), 1 + int(rng.next_u64() % 3)),
                                    params=(th,)))
            elif r == 8:
                gates.append(W.Gate("DIAG", (a, b), matrix=np.exp(1j * np.array([rng.uniform() for _ in range(4)]))))
            elif r == 9:
                gates.append(W.Gate("DENSE", (a,), matrix=oracle.rotation(oracle.PAULI[1 + int(rng.next_u64() % 3)], th)))
            elif r == 10:
                gates.append(W.Gate("PAULI", (a, b), pauli=(int(rng.next_u64() % 4), 1 + int(rng.next_u64() % 3))))
            else:
                gates.append([W.Gate("H", (a,)), W.Gate("U3", (a,), params=(th, 0.3, -0.2)), W.Gate("SWAP", (a, b))][layer % 3])
    return W.Circuit(n, gates)


@pytest.mark.parametrize("k", [2, 3, 4, 6])
def test_fusion_commuting_reorders_exact(k):
    """Blocks formed across commuting gates (shared qubits with a common Z, X or Y basis) give the
    circuit's product: mixed commuting circuits and the hardware-efficient ansatz at n = 9."""
    n = 9
    for circ in [commuting_mix_circuit(n, 101 + k), commuting_mix_circuit(n, 202 + k), W.hea_circuit(n, 5, 7)]:
        ref = oracle.run_circuit(circ)
        plan = qs.FusedCircuit(circ, k)
        got = run_plan_with_oracle(plan, n)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_fusion_commutation_respects_non_commuting_gates():
    """Hadamards (no common basis with Z or X gates) interleaved with diagonal and X-type gates
    on overlapping qubits: every block order the planner picks must keep them in place."""
    n = 7
    rng = W.SplitMix64(77)
    gates = []
    for _ in range(120):
        a = int(rng.next_u64() % n)
        b = (a + 1 + int(rng.next_u64() % (n - 1))) % n
        r = int(rng.next_u64() % 5)
        if r == 0:
            gates.append(W.Gate("H", (a,)))
        elif r == 1:
            gates.append(W.Gate("CZ", (a, b)))
        elif r == 2:
            gates.append(W.Gate("RZ", (a,), params=(rng.uniform() * 6,)))
        elif r == 3:
            gates.append(W.Gate("RX", (a,), params=(rng.uniform() * 6,)))
        else:
            gates.append(W.Gate("CNOT", (a,), controls=(b,), control_values=(1,)))
    circ = W.Circuit(n, gates)
    ref = oracle.run_circuit(circ)
    for k in (2, 3, 4, 5):
        got = run_plan_with_oracle(qs.FusedCircuit(circ, k), n)
        assert np.max(np.abs(got - ref)) < 1e-12, k


def test_fusion_commutation_shrinks_commuting_circuits():
    """The ansatz's RZ layers commute with the CZ ladders: far fewer blocks than the
    disjoint-qubit rule alone gives (k = 4: 94 for n = 20, 20 layers). In an IQP-like circuit
    everything between the two Hadamard layers commutes: one block per neighbouring pair."""
    c = W.hea_circuit(20, 20, 1)
    assert qs.FusedCircuit(c, 4).n_blocks <= 64
    assert qs.FusedCircuit(W.iqp_circuit(30, 20, 1), 2).n_blocks <= 29
    n = 9
    iqp = W.iqp_circuit(n, 8, 5)
    ref = oracle.run_circuit(iqp)
    for k in (2, 4, 6):
        assert np.max(np.abs(run_plan_with_oracle(qs.FusedCircuit(iqp, k), n) - ref)) < 1e-12


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_fusion_reordered_blocks_exact(k):
    """Blocks taken out of circuit order (frontier growth) still give the circuit's product:
    deeper circuits and mixed controlled / multi-target gates at n = 10."""
    n = 10
    for circ in [W.u3cz_circuit(n, 10, 21), W.Circuit(n, W.random_gate_suite(n, 23) * 2),
                 W.hea_circuit(n, 4, 6), W.rzrxrz_cnot_circuit(n, 5, 7)]:
        ref = oracle.run_circuit(circ)
        plan = qs.FusedCircuit(circ, k)
        got = run_plan_with_oracle(plan, n)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_expectation_plan_packs_flip_groups_into_tiles():
    """The host plan of qs_expectation: each tiled read holds qubits 0..2 plus 9 others, every
    flip mask lies inside the tile of some read, and a 30-qubit transverse-field Ising chain
    (31 flip-mask groups) needs 3 reads instead of 31."""
    n = 30
    obs = W.tfim_observable(n, 1.0)
    masks, single = qs.expectation_plan(n, obs)
    assert len(masks) == 3 and single == 0
    for m in masks:
        assert m & 7 == 7 and bin(m).count("1") == 12 and m < (1 << n)
    for f in set(int(x) for x in obs.x_mask):
        assert any(f & ~m == 0 for m in masks), f
    # small states: the tile is the whole state; a read takes at most 24 flip-mask groups
    r = W.random_pauli_observable(9, 30, 1)
    groups = len(set(int(x) for x in r.x_mask))
    masks, single = qs.expectation_plan(9, r)
    assert masks == [(1 << 9) - 1] * ((groups + 23) // 24) and single == 0
    # a diagonal observable: one read whatever its size
    z = W.PauliObservable(24, np.ones(40), np.zeros(40, dtype=np.uint64),
                          np.arange(1, 41, dtype=np.uint64) * 12345)
    masks, single = qs.expectation_plan(24, z)
    assert len(masks) == 1 and single == 0
    # a flip mask with 10 X positions above qubit 2 fits no tile: a single-group read
    wide = sum(1 << q for q in range(3, 13))
    w = W.PauliObservable(20, np.array([1.0, 0.5]), np.array([wide, 1], dtype=np.uint64),
                          np.array([0, 0], dtype=np.uint64))
    masks, single = qs.expectation_plan(20, w)
    assert single == 1 and len(masks) == 1 and masks[0] & 1
    # Heisenberg chain (XX, YY share a flip mask; ZZ diagonal) on 24 qubits: 3 reads
    terms = []
    for i in range(23):
        m = (1 << i) | (1 << (i + 1))
        terms += [(1.0, m, 0), (1.0, m, m), (1.0, 0, m)]
    h = W.PauliObservable(24, np.array([t[0] for t in terms]), np.array([t[1] for t in terms], dtype=np.uint64),
                          np.array([t[2] for t in terms], dtype=np.uint64))
    masks, single = qs.expectation_plan(24, h)
    assert single == 0 and len(masks) <= 3
    with pytest.raises(qs.QsError):
        qs.expectation_plan(35, obs)


def test_diagonal_runs_share_one_pass_in_block_costs():
    """Consecutive uncontrolled diagonal and phase blocks of a plan run as one pass: the block
    costs (host only) report one launch and one full pass for the first block of each run, none
    for the others. A run's product is held as two tables: each block in turn joins the first
    if the union of its qubits stays within 12, else the second if within 8; a run ends at the
    first block that fits neither."""
    n = 16
    gates = []
    for layer in range(4):
        for q in range(n):
            gates.append(W.Gate("RZ", (q,), params=(0.1 * (q + layer),)))
        for q in range(layer % 2, n - 1, 2):
            gates.append(W.Gate("CZ", (q, q + 1)))
    plan = qs.FusedCircuit(W.Circuit(n, gates), 4)
    costs = [plan.block_cost(b, qs.QS_C128) for b in range(plan.n_blocks)]
    full = 2 * 16 * 2 ** n
    launches = [l for _, l, _ in costs]
    assert sum(launches) < plan.n_blocks
    # a run starts at each block with a launch; its blocks up to the next launch share it
    runs, cur = [], None
    for b, (kind, l, by) in enumerate(costs):
        assert kind in ("diag", "phase")
        if l:
            cur = [b]
            runs.append(cur)
            assert 0 < by <= full
        else:
            assert by == 0 and cur is not None
            cur.append(b)
    def split_add(sp, q):
        for i, lim in ((0, 12), (1, 8)):
            if len(sp[i] | q) <= lim:
                sp[i] |= q
                return True
        return False

    for i, r in enumerate(runs):
        sp = [set(), set()]
        for b in r:
            assert split_add(sp, set(plan.block(b)[0]))
        if i + 1 < len(runs):  # the next run's first block fits neither table
            assert not split_add(sp, set(plan.block(runs[i + 1][0])[0]))
        if len(r) > 1:
            assert costs[r[0]][2] == full


def test_layout_passes_folded_into_first_and_last_blocks():
    """A double-float complex128 run of a plan adds separate layout-change passes only where its
    first block is not an uncontrolled 4- or 5-target tensor-core block (entry) and its last
    launch is not a run of diagonal blocks (exit); complex64 and FP64 runs add none (host only)."""
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    try:
        qs.set_c128_math(qs.QS_MATH_DF)
        qs.set_tensor_cores(qs.QS_TENSOR_C128)
        p4 = qs.FusedCircuit(W.u3cz_circuit(14, 6, 35), 4)    # dense_oz ... diag, phase
        p5 = qs.FusedCircuit(W.u3cz_circuit(14, 6, 36), 5)    # dense_oz5 ... dense_oz5
        p3 = qs.FusedCircuit(W.u3cz_circuit(14, 6, 35), 3)    # 3-target blocks ... phase
        assert p4.block_cost(0, qs.QS_C128)[0] == "dense_oz"
        assert p4.layout_passes(qs.QS_C128) == 0
        assert p5.layout_passes(qs.QS_C128) == 1
        assert p3.layout_passes(qs.QS_C128) == 2
        assert p4.layout_passes(qs.QS_C64) == 0
        # the benchmark circuit (n = 30, depth 20) at k = 5: both changes folded
        assert qs.FusedCircuit(W.u3cz_circuit(30, 20, 20201127), 5).layout_passes(qs.QS_C128) == 0
        qs.set_tensor_cores(0)  # CUDA-core first block: the entry change is a pass of its own
        assert p4.layout_passes(qs.QS_C128) == 1
        qs.set_c128_math(qs.QS_MATH_FP64)
        assert p4.layout_passes(qs.QS_C128) == 0
    finally:
        qs.set_c128_math(old_m)
        qs.set_tensor_cores(old_t)


def test_diagonal_run_table_limits():
    """A diagonal run's two tables at their limits (host only): three 4-qubit diagonals fill the
    first table (12 qubits), two more fill the second (8), and the next one, on 4 new qubits, fits
    neither and starts a second run; a diagonal whose qubits all lie in one table joins the run
    (one whose qubits straddle both tables would not)."""
    n = 28
    rng = W.SplitMix64(2828)

    def diag(qubits):
        d = np.exp(1j * 2 * np.pi * np.array([rng.uniform() for _ in range(1 << len(qubits))]))
        return W.Gate("DIAG", tuple(qubits), matrix=d)

    gates = [diag(range(4 * b, 4 * b + 4)) for b in range(5)]   # qubits 0..19
    gates.append(diag((0, 5, 10, 11)))                           # inside the first table
    gates.append(diag(range(20, 24)))                            # fits neither table
    gates.append(diag(range(24, 28)))
    plan = qs.FusedCircuit(W.Circuit(n, gates), 4)
    blocks = [tuple(sorted(plan.block(b)[0])) for b in range(plan.n_blocks)]
    launches = [plan.block_cost(b, qs.QS_C128)[1] for b in range(plan.n_blocks)]
    assert len(blocks) == len(gates), blocks
    first_run = [i for i, b in enumerate(blocks) if max(b) < 20]
    assert len(first_run) == 6 and launches[first_run[0]] == 1
    assert all(launches[i] == 0 for i in first_run[1:])
    later = [i for i in range(len(blocks)) if i not in first_run]
    assert sorted(launches[i] for i in later) == [0, 1], (blocks, launches)
    # qubits in both tables: the block fits neither table alone and starts a new run
    gates2 = gates[:5] + [diag((0, 5, 10, 15))]
    plan2 = qs.FusedCircuit(W.Circuit(n, gates2), 4)
    launches2 = [plan2.block_cost(b, qs.QS_C128)[1] for b in range(plan2.n_blocks)]
    assert plan2.n_blocks == 6 and launches2 == [1, 0, 0, 0, 0, 1], launches2
