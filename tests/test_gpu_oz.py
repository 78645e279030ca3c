"""GPU parity of the tensor-core path for 4-target dense blocks of double-float complex128 runs
(QS_MATH_DF with QS_TENSOR_C128: bf16 slices, exact FP32 sums on tcgen05) against the FP64
oracle, at the complex128 bound (1e-12 max-abs amplitude error)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_13524_gb300 as qs
    qs.lib()
    return qs


@pytest.fixture
def oz(qs):
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    qs.set_c128_math(qs.QS_MATH_DF)
    qs.set_tensor_cores(qs.QS_TENSOR_C128)
    yield qs
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def run_one(qs, n, gate, psi0):
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(W.Circuit(n, [gate]), 0)
    return st.get_vector()


@pytest.mark.parametrize("n", [4, 5, 8, 11, 12, 13, 15])
def test_oz_single_gate_placements(oz, n):
    """One 4-target dense gate (random, non-unitary) on low, high, mixed and unsorted targets;
    n = 4 is a single group, n = 11 exactly one 128-group tile, n = 12, 13, 15 several tiles."""
    qs = oz
    rng = W.SplitMix64(100 + n)
    psi0 = W.random_state(n, n)
    placements = [(0, 1, 2, 3), (n - 1, n - 2, n - 3, n - 4), (0, 2, n - 1, 1), (3, 0, n - 2, 1)]
    for t in placements:
        if len(set(t)) < 4:
            continue
        K = W.random_complex_matrix(16, rng)
        g = W.Gate("DENSE", t, matrix=K)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        got = run_one(qs, n, g, psi0)
        assert maxabs(got, ref) < 1e-12 * max(1.0, float(np.max(np.abs(ref)))), t


@pytest.mark.parametrize("n", [6, 9, 14])
def test_oz_controlled_gate(oz, n):
    qs = oz
    rng = W.SplitMix64(7 + n)
    psi0 = W.random_state(n, 3 * n)
    for t, c, cv in [((1, 2, 3, 4), (0,), (1,)), ((0, n - 1, 2, 3), (1,), (0,))]:
        g = W.Gate("DENSE", t, controls=c, control_values=cv, matrix=W.random_unitary(16, rng))
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        assert maxabs(run_one(qs, n, g, psi0), ref) < 1e-12


def test_oz_scaled_and_zero_groups(oz):
    """Groups of very different magnitude, all-zero groups (basis-like states) and a
    non-unitary matrix with large entries: errors stay relative to each group's scale."""
    qs = oz
    n = 12
    rng = W.SplitMix64(5)
    psi0 = W.random_state(n, 9)
    psi0[: 1 << 8] *= 1e-6          # groups with tiny amplitudes
    psi0[1 << 10: 1 << 11] = 0.0     # whole zero groups for targets above bit 3
    K = W.random_complex_matrix(16, rng) * 7.5
    g = W.Gate("DENSE", (4, 5, 6, 7), matrix=K)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    got = run_one(qs, n, g, psi0)
    err = np.abs(got - ref)
    assert float(np.max(err)) < 1e-12 * 8
    small = slice(0, 1 << 8)
    # in tiny groups the error scales down with the group (relative to 1e-6 amplitudes)
    assert float(np.max(err[small])) < 1e-17


@pytest.mark.parametrize("n", [12, 16, 20])
def test_oz_fused_circuits(oz, n):
    qs = oz
    c = W.u3cz_circuit(n, 20 if n < 20 else 10, 40 + n)
    ref = oracle.run_circuit(c)
    st = qs.State(n, qs.QS_C128)
    st.run(c, 4)
    got = st.get_vector()
    assert maxabs(got, ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-12


def test_oz_matches_cuda_core_path(oz):
    """Same plan through the tensor-core kernel and the double-float CUDA-core kernel."""
    qs = oz
    n = 18
    c = W.Circuit(n, W.random_gate_suite(n, 12))
    plan = qs.FusedCircuit(c, 4)
    a = qs.State(n, qs.QS_C128)
    a.apply_plan(plan)
    mask = qs.get_tensor_cores()
    qs.set_tensor_cores(0)
    b = qs.State(n, qs.QS_C128)
    b.apply_plan(plan)
    qs.set_tensor_cores(mask)
    assert maxabs(a.get_vector(), b.get_vector()) < 1e-12


def test_oz_full_size_sampled(oz):
    import torch
    from test_gpu_parity import product_then_cz, sampled_amplitudes
    qs = oz
    n = 30
    circ, u3, cz = product_then_cz(n, 20, 778)
    st = qs.State(n, qs.QS_C128)
    plan = qs.FusedCircuit(circ, 4)
    st.apply_plan(plan)
    st.synchronize()
    rng = W.SplitMix64(8)
    xs = [rng.next_u64() & ((1 << n) - 1) for _ in range(2000)] + [0, (1 << n) - 1]
    ref = sampled_amplitudes(n, u3, cz, xs)
    idx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    got = st.tensor[idx].cpu().numpy()
    assert maxabs(got, ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-11
    st.close()
    del st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [5, 6, 11, 12, 13, 16])
def test_oz5_single_gate_placements(oz, n):
    """One 5-target dense gate (random, non-unitary) on low, high, mixed and unsorted targets:
    n = 5 is a single group, n = 12 exactly one 128-group tile, 13 and 16 several tiles; both
    output halves and all four threads of a group are exercised."""
    qs = oz
    rng = W.SplitMix64(200 + n)
    psi0 = W.random_state(n, 3 * n + 1)
    placements = [(0, 1, 2, 3, 4), tuple(range(n - 1, n - 6, -1)), (0, 2, n - 1, 1, n - 2), (4, 0, n - 3, 1, 2)]
    for t in placements:
        if len(set(t)) < 5 or max(t) >= n:
            continue
        K = W.random_complex_matrix(32, rng)
        g = W.Gate("DENSE", t, matrix=K)
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        got = run_one(qs, n, g, psi0)
        assert maxabs(got, ref) < 1e-12 * max(1.0, float(np.max(np.abs(ref)))), t


def test_oz5_controlled_and_scaled(oz):
    """A controlled 5-target unitary, and a large non-unitary matrix on a state with tiny and
    zero groups (errors relative to each group's scale)."""
    qs = oz
    n = 13
    rng = W.SplitMix64(77)
    psi0 = W.random_state(n, 12)
    g = W.Gate("DENSE", (1, 2, 3, 5, 9), controls=(0,), control_values=(1,), matrix=W.random_unitary(32, rng))
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    assert maxabs(run_one(qs, n, g, psi0), ref) < 1e-12
    # unsorted targets including qubits 0, 1 and 2 (the paired 32-byte accesses), control value 0
    g = W.Gate("DENSE", (9, 2, 0, 6, 1), controls=(4,), control_values=(0,), matrix=W.random_unitary(32, rng))
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    assert maxabs(run_one(qs, n, g, psi0), ref) < 1e-12
    psi1 = psi0.copy()
    psi1[: 1 << 9] *= 1e-6
    psi1[1 << 11: 1 << 12] = 0.0
    K = W.random_complex_matrix(32, rng) * 6.0
    g = W.Gate("DENSE", (4, 5, 6, 7, 8), matrix=K)   # every group below 2^9 is entirely tiny
    ref = psi1.copy()
    oracle.apply_gate(ref, n, g)
    got = run_one(qs, n, g, psi1)
    err = np.abs(got - ref)
    assert float(np.max(err)) < 1e-12 * 8
    assert float(np.max(err[: 1 << 9])) < 1e-17


@pytest.mark.parametrize("n", [12, 16, 20])
def test_oz5_fused_circuits(oz, n):
    qs = oz
    c = W.u3cz_circuit(n, 20 if n < 20 else 10, 60 + n)
    ref = oracle.run_circuit(c)
    st = qs.State(n, qs.QS_C128)
    st.run(c, 5)
    assert maxabs(st.get_vector(), ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-12


def test_oz5_matches_cuda_core_path(oz):
    qs = oz
    n = 17
    c = W.Circuit(n, W.random_gate_suite(n, 31))
    plan = qs.FusedCircuit(c, 5)
    a = qs.State(n, qs.QS_C128)
    a.apply_plan(plan)
    mask = qs.get_tensor_cores()
    qs.set_tensor_cores(0)
    b = qs.State(n, qs.QS_C128)
    b.apply_plan(plan)
    qs.set_tensor_cores(mask)
    assert maxabs(a.get_vector(), b.get_vector()) < 1e-12


def test_oz5_full_size_sampled(oz):
    import torch
    from test_gpu_parity import product_then_cz, sampled_amplitudes
    qs = oz
    n = 30
    circ, u3, cz = product_then_cz(n, 20, 779)
    st = qs.State(n, qs.QS_C128)
    st.apply_plan(qs.FusedCircuit(circ, 5))
    st.synchronize()
    rng = W.SplitMix64(9)
    xs = [rng.next_u64() & ((1 << n) - 1) for _ in range(2000)] + [0, (1 << n) - 1]
    ref = sampled_amplitudes(n, u3, cz, xs)
    idx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    got = st.tensor[idx].cpu().numpy()
    assert maxabs(got, ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-11
    st.close()
    del st
    torch.cuda.empty_cache()


def test_oz_paired_access_alignment(oz):
    """Blocks whose lowest target is qubit 0 move amplitude pairs with 256-bit accesses when the
    state is 32-byte aligned; a state wrapped 16 bytes into a buffer takes the single-amplitude
    path. Both give the oracle's result (4- and 5-target blocks, complex128 double-float; and
    complex64 5-target blocks, whose pairs need only the 16 bytes every state has)."""
    import torch
    qs = oz
    n = 13
    rng = W.SplitMix64(57)
    psi0 = W.random_state(n, 13)
    gates = [W.Gate("DENSE", (0, 1, 2, 3), matrix=W.random_unitary(16, rng)),
             W.Gate("DENSE", (0, 4, 5, 9, 12), matrix=W.random_unitary(32, rng)),
             W.Gate("DENSE", (0, 1, 2, 3, 4), controls=(7,), control_values=(1,), matrix=W.random_unitary(32, rng))]
    ref = psi0.copy()
    for g in gates:
        oracle.apply_gate(ref, n, g)
    for offset in (0, 1):  # amplitudes: 0 -> 32-byte aligned, 1 -> 16 bytes off
        buf = torch.zeros((1 << n) + 2, dtype=torch.complex128, device="cuda")
        view = buf[offset:offset + (1 << n)]
        st = qs.State(n, qs.QS_C128, tensor=view)
        st.load(psi0)
        st.run(W.Circuit(n, gates), 0)
        assert maxabs(st.get_vector(), ref) < 1e-12, offset
        assert buf[:offset].abs().max().item() == 0 if offset else True
        assert buf[offset + (1 << n):].abs().max().item() == 0
    c64_gates = gates[1:]
    ref64 = psi0.copy()
    for g in c64_gates:
        oracle.apply_gate(ref64, n, g)
    qs.set_tensor_cores(qs.QS_TENSOR_C128 | qs.QS_TENSOR_C64X)
    for offset in (0, 2):  # complex64 states are 16-byte aligned (a wrapped pointer must be)
        buf = torch.zeros((1 << n) + 2, dtype=torch.complex64, device="cuda")
        st = qs.State(n, qs.QS_C64, tensor=buf[offset:offset + (1 << n)])
        st.load(psi0)
        st.run(W.Circuit(n, c64_gates), 0)
        assert maxabs(st.get_vector(), ref64) < 1e-5, offset


def _diag_only_circuit(n, seed):
    rng = W.SplitMix64(seed)
    gates = []
    for q in range(n):
        gates.append(W.Gate("RZ", (q,), params=(2 * np.pi * rng.uniform(),)))
    for q in range(0, n - 1, 2):
        gates.append(W.Gate("CZ", (q, q + 1)))
    return W.Circuit(n, gates)


@pytest.mark.parametrize("case", ["u3cz_k4", "u3cz_k5", "cuda_core_first", "diag_only"])
def test_oz_plan_folds_layout_changes(oz, case):
    """A double-float plan run changes the layout in its first and last passes where they read
    every amplitude once: an uncontrolled tensor-core block first (it splits the IEEE doubles as
    it loads them), a diagonal run last (it writes RN(hi + lo)). Each combination (both folded;
    the first only; the last only, after a CUDA-core first block; a plan of one diagonal run)
    matches the oracle at the complex128 bound from a state whose amplitudes span 1e-12 .. 1,
    with exact zeros."""
    qs = oz
    n = 14
    if case == "u3cz_k4":
        c, k, first, last = W.u3cz_circuit(n, 6, 35), 4, "dense_oz", ("diag", "phase")
    elif case == "u3cz_k5":
        c, k, first, last = W.u3cz_circuit(n, 6, 36), 5, "dense_oz5", ("dense_oz5",)
    elif case == "cuda_core_first":
        qs.set_tensor_cores(0)
        c, k, first, last = W.u3cz_circuit(n, 6, 35), 4, "dense_smem", ("diag", "phase")
    else:
        c, k, first, last = _diag_only_circuit(12, 5), 4, "diag", ("diag", "phase")
        n = 12
    plan = qs.FusedCircuit(c, k)
    kinds = [plan.block_cost(b, qs.QS_C128)[0] for b in range(plan.n_blocks)]
    assert kinds[0] == first and kinds[-1] in last, kinds
    psi0 = W.random_state(n, 40 + n) * 10.0 ** -np.linspace(0, 12, 1 << n)
    psi0[::29] = 0.0
    ref = psi0.copy()
    for g in c.gates:
        oracle.apply_gate(ref, n, g)
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.apply_plan(plan)
    got = st.get_vector()
    assert maxabs(got, ref) < 1e-12 * float(np.max(np.abs(ref))), case
    # the state is IEEE complex128 again: a second run continues from it
    st.apply_plan(plan)
    for g in c.gates:
        oracle.apply_gate(ref, n, g)
    assert maxabs(st.get_vector(), ref) < 2e-12 * float(np.max(np.abs(ref))), case
    st.close()
