"""Tensor-core path for complex64 dense blocks of 5-6 targets (tcgen05.mma kind::tf32 with the
3xTF32 split) against the FP64 oracle and against the FP32 CUDA-core kernels: every target
placement class (low, high, mixed qubits), controls, 5-target blocks padded to 6, ragged tiles
(fewer than 32 groups, or a partial last tile), and fused circuits at widths 5 and 6."""
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


def run(qs, n, gates, psi0, tensor):
    old = qs.get_tensor_cores()
    qs.set_tensor_cores(tensor)
    try:
        st = qs.State(n, qs.QS_C64)
        st.load(psi0)
        for g in gates:
            st.apply_gate(g)
        st.synchronize()
        return st.get_vector().astype(np.complex128)
    finally:
        qs.set_tensor_cores(old)


PLACEMENTS = {
    "low": (0, 1, 2, 3, 4, 5),
    "high": None,           # the six highest qubits
    "mixed": (7, 0, 11, 3, 9, 5),
    "reversed": (5, 4, 3, 2, 1, 0),
}


@pytest.mark.parametrize("n", [6, 10, 11, 13, 17])
@pytest.mark.parametrize("place", list(PLACEMENTS))
def test_tc_six_targets(qs, n, place):
    t = PLACEMENTS[place] or tuple(range(n - 6, n))
    if max(t) >= n:
        pytest.skip("placement needs more qubits")
    rng = W.SplitMix64(n * 31 + len(place))
    g = W.Gate("DENSE", t, matrix=W.random_unitary(64, rng))
    psi0 = W.random_state(n, n + 1)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g], psi0, True)
    cuda_cores = run(qs, n, [g], psi0, False)
    assert np.max(np.abs(got - ref)) < 2e-6
    assert np.max(np.abs(got - cuda_cores)) < 2e-6


@pytest.mark.parametrize("n", [7, 12, 15])
def test_tc_five_targets_padded_and_controls(qs, n):
    rng = W.SplitMix64(n)
    psi0 = W.random_state(n, 3 * n)
    qs_ = list(range(n))
    picks = [qs_.pop(rng.randint(0, len(qs_) - 1)) for _ in range(min(n, 8))]
    gates = [W.Gate("DENSE", tuple(picks[:5]), matrix=W.random_unitary(32, rng))]
    if n >= 8:
        gates.append(W.Gate("DENSE", tuple(picks[:6]), controls=(picks[6], picks[7]), control_values=(1, 0),
                            matrix=W.random_unitary(64, rng)))
        gates.append(W.Gate("DENSE", tuple(picks[1:6]), controls=(picks[7],), control_values=(1,),
                            matrix=W.random_unitary(32, rng)))
    ref = psi0.copy()
    for g in gates:
        oracle.apply_gate(ref, n, g)
    got = run(qs, n, gates, psi0, True)
    assert np.max(np.abs(got - ref)) < 4e-6


def test_tc_non_unitary_scaling(qs):
    """K need not be unitary: a scaled Gaussian matrix keeps relative FP32-class accuracy."""
    n = 12
    rng = W.SplitMix64(5)
    K = W.random_complex_matrix(64, rng) * 0.05
    g = W.Gate("DENSE", (2, 9, 4, 11, 0, 6), matrix=K)
    psi0 = W.random_state(n, 9)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g], psi0, True)
    assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)) * 10)


@pytest.mark.parametrize("k", [5, 6])
def test_tc_fused_circuits(qs, k):
    for n, c in [(14, W.u3cz_circuit(14, 8, 3)), (16, W.rzrxrz_cnot_circuit(16, 3, 5)),
                 (12, W.Circuit(12, W.random_gate_suite(12, 77)))]:
        ref = oracle.run_circuit(c)
        st = qs.State(n, qs.QS_C64)
        st.run(c, k)
        st.synchronize()
        assert np.max(np.abs(st.get_vector() - ref)) < 1e-5


def test_tc_full_size_fused_equals_cuda_cores(qs):
    """n = 28 complex64, depth-6 circuit fused at width 6: tensor cores vs CUDA cores, and the norm."""
    import torch
    n = 28
    c = W.u3cz_circuit(n, 6, 42)
    old = qs.get_tensor_cores()
    try:
        qs.set_tensor_cores(True)
        a = qs.State(n, qs.QS_C64)
        a.run(c, 6)
        qs.set_tensor_cores(False)
        b = qs.State(n, qs.QS_C64)
        b.run(c, 6)
        a.synchronize()
        b.synchronize()
        assert (a.tensor - b.tensor).abs().max().item() < 5e-6
        # the tensor cores round their FP32 accumulator toward zero at every MMA: the norm shrinks
        # by at most ~4e-6 per 6-qubit block (measured 2.0e-6); this circuit has < 25 such blocks
        assert abs(a.norm2() - 1.0) < 1e-4
        assert abs(b.norm2() - 1.0) < 1e-5
    finally:
        qs.set_tensor_cores(old)
    del a, b
    torch.cuda.empty_cache()


def test_tc_bias_bound(qs):
    """60 applications of one unitary 6-qubit block: the tensor-core result stays within the
    complex64 bound of the oracle, and the norm shrinks by at most 4e-6 per block."""
    n = 14
    rng = W.SplitMix64(3)
    U = W.random_unitary(64, rng)
    g = W.Gate("DENSE", (0, 3, 5, 7, 9, 12), matrix=U)
    psi0 = W.random_state(n, 1)
    ref = psi0.copy()
    for _ in range(60):
        oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g] * 60, psi0, True)
    assert np.max(np.abs(got - ref)) < 1e-5
    shrink = 1.0 - np.vdot(got, got).real
    assert 0.0 <= shrink < 60 * 4e-6
