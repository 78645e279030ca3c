"""GPU parity of the Pauli rotation pass (exp(i angle P / 2) for strings of any length, Sec. 4.3.2)
and of the Trotterized observable rotation (Sec. 4.5) against the oracle."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {1: 1e-5, 2: 1e-12}


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_13524_gb300 as qs
    qs.lib()
    return qs


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(b, dtype=np.complex128))))


def random_masks(n, rng, dense=False):
    xm = zm = 0
    while xm == 0 and zm == 0:
        for q in range(n):
            pid = int(rng.next_u64() % 4)
            if dense and pid == 0:
                pid = 1 + int(rng.next_u64() % 3)
            if pid in (1, 2):
                xm |= 1 << q
            if pid in (2, 3):
                zm |= 1 << q
    return xm, zm


@pytest.mark.parametrize("n", [1, 3, 7, 12, 17])
def test_pauli_rotation_random_strings(qs, n):
    """Strings of every length up to n (well beyond the 6-target gate limit), Y factors, Z-only
    strings; complex128 in FP64 and double-float arithmetic, complex64."""
    rng = W.SplitMix64(60 + n)
    old = qs.get_c128_math()
    try:
        for trial in range(4):
            xm, zm = random_masks(n, rng, dense=trial % 2 == 0)
            if trial == 3:
                xm = 0  # a Z string: the diagonal branch
                zm = zm or 1
            angle = 4 * math.pi * rng.uniform() - 2 * math.pi
            psi0 = W.random_state(n, 11 * n + trial)
            ref = oracle.apply_pauli_rotation(psi0.copy(), n, xm, zm, angle)
            for dtype, math_mode in ((2, qs.QS_MATH_FP64), (2, qs.QS_MATH_DF), (1, qs.QS_MATH_FP64)):
                qs.set_c128_math(math_mode)
                st = qs.State(n, dtype)
                st.load(psi0)
                st.apply_pauli_rotation(xm, zm, angle)
                got = st.get_vector()
                st.close()
                assert maxabs(got, ref) < TOL[dtype], (trial, dtype, math_mode)
    finally:
        qs.set_c128_math(old)


def test_paulirot_gate_uses_the_pass(qs):
    """PAULIROT gates with X/Y factors on 4 and 6 targets (and a control) through qs_apply_gate."""
    n = 9
    rng = W.SplitMix64(5)
    psi0 = W.random_state(n, 7)
    gates = [W.Gate("PAULIROT", (0, 3, 5, 8), pauli=(1, 2, 3, 1), params=(0.7,)),
             W.Gate("PAULIROT", (1, 2, 4, 6, 7, 8), pauli=(2, 2, 1, 3, 1, 2), params=(-2.1,)),
             W.Gate("PAULIROT", (2, 6), pauli=(1, 3), params=(1.3,), controls=(4,), control_values=(1,))]
    for g in gates:
        ref = psi0.copy()
        oracle.apply_gate(ref, n, g)
        for dtype in (2, 1):
            st = qs.State(n, dtype)
            st.load(psi0)
            st.apply_gate(g)
            assert maxabs(st.get_vector(), ref) < TOL[dtype], (g.targets, dtype)
            st.close()
    del rng


def test_observable_rotation_vs_oracle(qs):
    """Transverse-field Ising chain and a random observable with Y terms and an identity term:
    the Trotter product with several slices, complex128 (double-float) and complex64."""
    n = 10
    old = qs.get_c128_math()
    try:
        for obs in (W.tfim_observable(n, 1.0), W.random_pauli_observable(n, 7, 2718)):
            psi0 = W.random_state(n, 19)
            ref = oracle.observable_rotation(psi0, n, obs, 0.37, 3)
            for dtype, math_mode in ((2, qs.QS_MATH_DF), (2, qs.QS_MATH_FP64), (1, qs.QS_MATH_FP64)):
                qs.set_c128_math(math_mode)
                st = qs.State(n, dtype)
                st.load(psi0)
                st.apply_observable_rotation(obs, 0.37, 3)
                err = maxabs(st.get_vector(), ref)
                assert err < TOL[dtype], (dtype, math_mode, err)
                st.close()
    finally:
        qs.set_c128_math(old)


def test_pauli_rotation_invalid_mask(qs):
    st = qs.State(5, 2)
    with pytest.raises(qs.QsError):
        st.apply_pauli_rotation(1 << 5, 0, 0.3)
    with pytest.raises(qs.QsError):
        st.apply_observable_rotation(W.tfim_observable(5, 1.0), 0.1, 0)
    st.close()


def test_pauli_rotation_full_size(qs):
    """n = 30 complex128: exp(i angle P / 2)|0...0> = cos|0> + i sin i^nY |xmask>, closed form;
    the state elsewhere stays zero and the norm stays 1."""
    import torch
    n = 30
    rng = W.SplitMix64(30)
    xm, zm = random_masks(n, rng, dense=True)
    angle = 1.234
    st = qs.State(n, 2)
    st.apply_pauli_rotation(xm, zm, angle)
    st.synchronize()
    ny = bin(xm & zm).count("1")
    a0 = st.tensor[0].item()
    a1 = st.tensor[xm].item()
    assert abs(a0 - math.cos(angle / 2)) < 1e-13
    assert abs(a1 - 1j * math.sin(angle / 2) * (1j ** ny)) < 1e-13
    assert abs(st.norm2() - 1.0) < 1e-12
    st.tensor[0] = 0
    st.tensor[xm] = 0
    assert float(st.tensor.abs().max().item()) == 0.0
    st.close()
    del st
    torch.cuda.empty_cache()
