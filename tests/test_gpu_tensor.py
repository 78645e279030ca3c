"""Edge cases of the complex64 tensor-core blocks (bf16 slices, exact FP32 sums; QS_TENSOR_C64X)
that the placement sweeps leave out: a 6-target block on a 6-qubit state (one group, a tile of
one row), targets given in descending order, a non-unitary scaled matrix, and one unitary block
applied 60 times in a row (the sums round to nearest once per output, so the norm shows no
drift), each against the FP64 oracle and the FP32 CUDA-core kernels."""
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


def run(qs, n, gates, psi0, mask):
    old = qs.get_tensor_cores()
    qs.set_tensor_cores(mask)
    try:
        st = qs.State(n, qs.QS_C64)
        st.load(psi0)
        for g in gates:
            st.apply_gate(g)
        st.synchronize()
        return st.get_vector().astype(np.complex128)
    finally:
        qs.set_tensor_cores(old)


@pytest.mark.parametrize("n,t", [(6, (0, 1, 2, 3, 4, 5)), (6, (5, 4, 3, 2, 1, 0)), (11, (10, 8, 6, 4, 2, 0)),
                                 (13, (12, 11, 10, 9, 8, 7))])
def test_tc6_single_group_and_descending_targets(qs, n, t):
    rng = W.SplitMix64(n * 31 + t[0])
    g = W.Gate("DENSE", t, matrix=W.random_unitary(64, rng))
    psi0 = W.random_state(n, n + 1)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g], psi0, qs.QS_TENSOR_C64X)
    cuda_cores = run(qs, n, [g], psi0, 0)
    assert np.max(np.abs(got - ref)) < 1e-6
    assert np.max(np.abs(got - cuda_cores)) < 1e-6


def test_tc6_non_unitary_scaling(qs):
    """K need not be unitary: a scaled Gaussian matrix keeps FP32-class accuracy relative to the
    largest output."""
    n = 12
    rng = W.SplitMix64(5)
    K = W.random_complex_matrix(64, rng) * 0.05
    g = W.Gate("DENSE", (2, 9, 4, 11, 0, 6), matrix=K)
    psi0 = W.random_state(n, 9)
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g], psi0, qs.QS_TENSOR_C64X)
    assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)) * 10)


def test_tc6_repeated_block_no_drift(qs):
    """60 applications of one unitary 6-qubit block: within the complex64 bound of the oracle, and
    the norm stays 1 to FP32 rounding (no systematic shrink)."""
    n = 14
    rng = W.SplitMix64(3)
    U = W.random_unitary(64, rng)
    g = W.Gate("DENSE", (0, 3, 5, 7, 9, 12), matrix=U)
    psi0 = W.random_state(n, 1)
    ref = psi0.copy()
    for _ in range(60):
        oracle.apply_gate(ref, n, g)
    got = run(qs, n, [g] * 60, psi0, qs.QS_TENSOR_C64X)
    assert np.max(np.abs(got - ref)) < 1e-5
    assert abs(1.0 - np.vdot(got, got).real) < 1e-5
