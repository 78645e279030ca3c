"""Tensor-core path for complex64 dense blocks of 5 and 6 targets with bf16 slices and exact FP32
sums (QS_TENSOR_C64X, on by default) against the FP64 oracle and the FP32 CUDA-core kernels:
target placements (low, high, mixed, unsorted), controls, ragged tiles, fused circuits at widths
5 and 6, and full-size runs whose norm shows no drift (one rounding to nearest per output)."""
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


@pytest.mark.parametrize("n", [5, 6, 11, 12, 13, 17])
def test_bz5_single_gate_placements(qs, n):
    rng = W.SplitMix64(400 + n)
    psi0 = W.random_state(n, 5 * n)
    for t in [(0, 1, 2, 3, 4), tuple(range(n - 1, n - 6, -1)), (0, 2, n - 1, 1, n - 2), (4, 0, n - 3, 1, 2)]:
        if len(set(t)) < 5 or max(t) >= n:
            continue
        g = W.Gate("DENSE", t, matrix=W.random_unitary(32, rng))
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        got = run(qs, n, [g], psi0, qs.QS_TENSOR_C64X)
        cuda_cores = run(qs, n, [g], psi0, 0)
        assert np.max(np.abs(got - ref)) < 1e-6, t
        assert np.max(np.abs(got - cuda_cores)) < 1e-6, t


def test_bz5_controlled_and_non_unitary(qs):
    n = 12
    rng = W.SplitMix64(91)
    psi0 = W.random_state(n, 4)
    gates = [W.Gate("DENSE", (2, 3, 5, 8, 11), controls=(0,), control_values=(1,), matrix=W.random_unitary(32, rng)),
             W.Gate("DENSE", (1, 4, 6, 7, 9), controls=(10, 0), control_values=(0, 1), matrix=W.random_unitary(32, rng)),
             W.Gate("DENSE", (0, 3, 6, 9, 10), matrix=W.random_complex_matrix(32, rng) * 3.0)]
    for g in gates:
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        got = run(qs, n, [g], psi0, qs.QS_TENSOR_C64X)
        assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, float(np.max(np.abs(ref))))


@pytest.mark.parametrize("n", [12, 16, 20])
def test_bz5_fused_circuits(qs, n):
    c = W.u3cz_circuit(n, 20 if n < 20 else 10, 70 + n)
    ref = oracle.run_circuit(c)
    old = qs.get_tensor_cores()
    try:
        qs.set_tensor_cores(qs.QS_TENSOR_C64X)
        st = qs.State(n, qs.QS_C64)
        st.run(c, 5)
        st.synchronize()
        assert np.max(np.abs(st.get_vector() - ref)) < 1e-5
    finally:
        qs.set_tensor_cores(old)


def test_bz5_full_size_no_drift(qs):
    """n = 28 complex64, depth-20 circuit fused at width 5: tensor cores (exact sums, one FP32
    rounding per output) against the CUDA cores, and the norm stays within FP32 rounding."""
    import torch
    n = 28
    c = W.u3cz_circuit(n, 20, 43)
    old = qs.get_tensor_cores()
    try:
        qs.set_tensor_cores(qs.QS_TENSOR_C64X)
        a = qs.State(n, qs.QS_C64)
        a.run(c, 5)
        qs.set_tensor_cores(0)
        b = qs.State(n, qs.QS_C64)
        b.run(c, 5)
        a.synchronize()
        b.synchronize()
        assert (a.tensor - b.tensor).abs().max().item() < 5e-6
        assert abs(a.norm2() - 1.0) < 1e-5
        assert abs(b.norm2() - 1.0) < 1e-5
    finally:
        qs.set_tensor_cores(old)
    del a, b
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [6, 7, 12, 13, 17])
def test_bz6_single_gate_placements(qs, n):
    rng = W.SplitMix64(600 + n)
    psi0 = W.random_state(n, 7 * n)
    for t in [(0, 1, 2, 3, 4, 5), tuple(range(n - 1, n - 7, -1)), (7, 0, n - 1, 3, n - 2, 5), (5, 4, 3, 2, 1, 0)]:
        if len(set(t)) < 6 or max(t) >= n:
            continue
        g = W.Gate("DENSE", t, matrix=W.random_unitary(64, rng))
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        got = run(qs, n, [g], psi0, qs.QS_TENSOR_C64X)
        cuda_cores = run(qs, n, [g], psi0, 0)
        assert np.max(np.abs(got - ref)) < 1e-6, t
        assert np.max(np.abs(got - cuda_cores)) < 1e-6, t


def test_bz6_controlled(qs):
    n = 11
    rng = W.SplitMix64(92)
    psi0 = W.random_state(n, 6)
    g = W.Gate("DENSE", (1, 2, 4, 6, 8, 9), controls=(0, 10), control_values=(1, 0), matrix=W.random_unitary(64, rng))
    ref = psi0.copy()
    oracle.apply_gate(ref, n, g)
    assert np.max(np.abs(run(qs, n, [g], psi0, qs.QS_TENSOR_C64X) - ref)) < 1e-6


@pytest.mark.parametrize("n", [12, 18])
def test_bz6_fused_circuits(qs, n):
    c = W.u3cz_circuit(n, 16, 90 + n)
    ref = oracle.run_circuit(c)
    old = qs.get_tensor_cores()
    try:
        qs.set_tensor_cores(qs.QS_TENSOR_C64X)
        st = qs.State(n, qs.QS_C64)
        st.run(c, 6)
        st.synchronize()
        assert np.max(np.abs(st.get_vector() - ref)) < 1e-5
    finally:
        qs.set_tensor_cores(old)


def test_bz6_full_size_no_drift(qs):
    import torch
    n = 28
    c = W.u3cz_circuit(n, 20, 44)
    old = qs.get_tensor_cores()
    try:
        qs.set_tensor_cores(qs.QS_TENSOR_C64X)
        a = qs.State(n, qs.QS_C64)
        a.run(c, 6)
        qs.set_tensor_cores(0)
        b = qs.State(n, qs.QS_C64)
        b.run(c, 6)
        a.synchronize()
        b.synchronize()
        assert (a.tensor - b.tensor).abs().max().item() < 5e-6
        assert abs(a.norm2() - 1.0) < 1e-5
    finally:
        qs.set_tensor_cores(old)
    del a, b
    torch.cuda.empty_cache()
