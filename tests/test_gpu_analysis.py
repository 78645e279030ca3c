"""GPU parity of the analysis calls (Sec. 4.2.2, Sec. 4.5): transition amplitude of an
observable, marginal probabilities, and Z-basis sampling with caller-drawn uniforms, against
the oracle."""
import math

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


@pytest.mark.parametrize("n", [1, 4, 9, 13])
def test_transition_amplitude(qs, n):
    obs = W.random_pauli_observable(n, 9, 300 + n)
    bra0, ket0 = W.random_state(n, 2 * n), W.random_state(n, 2 * n + 1) * 0.7
    ref = oracle.transition_amplitude(bra0, ket0, n, obs)
    for dtype, tol in ((2, 1e-12), (1, 1e-5)):
        bra, ket = qs.State(n, dtype), qs.State(n, dtype)
        bra.load(bra0)
        ket.load(ket0)
        got = bra.transition_amplitude(obs, ket)
        assert abs(got - ref) < tol, (dtype, got, ref)
        # bra = ket: the expectation value
        e = ket.expectation(obs)
        assert abs(ket.transition_amplitude(obs, ket) - complex(e[0], e[1])) < tol
        bra.close()
        ket.close()


@pytest.mark.parametrize("n", [1, 5, 12, 16])
def test_marginal_probability(qs, n):
    rng = W.SplitMix64(500 + n)
    psi0 = W.random_state(n, 3 * n) * 1.1
    for dtype, tol in ((2, 1e-13), (1, 1e-6)):
        st = qs.State(n, dtype)
        st.load(psi0)
        pats = [[2] * n, [0] * n, [1] * n] + [[int(rng.next_u64() % 3) for _ in range(n)] for _ in range(6)]
        for mv in pats:
            ref = oracle.marginal_probability(psi0, n, mv)
            assert abs(st.marginal_probability(mv) - ref) < tol, (dtype, mv)
        with pytest.raises(qs.QsError):
            st.marginal_probability([3] + [2] * (n - 1))
        st.close()


def check_samples(psi, uniforms, got):
    """Same index as the oracle's inverse-CDF search, except within rounding of a bin edge,
    where the returned index must still bracket the target."""
    ref = oracle.sample(psi, uniforms)
    cdf = np.cumsum(np.abs(np.asarray(psi, dtype=np.complex128)) ** 2)
    total = cdf[-1]
    mism = 0
    for u, g, r in zip(uniforms, got, ref):
        if g == r:
            continue
        mism += 1
        t = u * total
        lo = cdf[g - 1] if g > 0 else 0.0
        assert lo - 1e-12 * total <= t <= cdf[g] + 1e-12 * total, (u, g, r)
    assert mism <= max(1, len(uniforms) // 1000)


@pytest.mark.parametrize("n", [1, 6, 11, 15])
def test_sampling(qs, n):
    rng = W.SplitMix64(900 + n)
    psi0 = W.random_state(n, 5 * n) * 0.9
    u = np.array([rng.uniform() for _ in range(3000)])
    for dtype in (2, 1):
        st = qs.State(n, dtype)
        st.load(psi0)
        got = st.sample(u)
        vec = st.get_vector().astype(np.complex128)
        check_samples(vec, u, got)
        st.close()


def test_sampling_edge_cases(qs):
    st = qs.State(6, 2)
    st.set_basis(37)
    assert set(st.sample([0.0, 0.5, 0.999999]).tolist()) == {37}
    assert st.sample([]).size == 0
    with pytest.raises(qs.QsError):
        st.sample([1.0])
    with pytest.raises(qs.QsError):
        st.sample([-0.1])
    st.close()


def test_sampling_full_size(qs):
    """n = 30 complex128, H on qubits 0..2 of |0...0>: eight equally likely outcomes 0..7, so a
    uniform u draws floor(8 u) (away from the bin edges)."""
    import torch
    n = 30
    st = qs.State(n, 2)
    for q in range(3):
        st.apply_gate(W.Gate("H", (q,)))
    rng = W.SplitMix64(31)
    u = np.array([rng.uniform() for _ in range(500)])
    u = u[np.abs(8 * u - np.round(8 * u)) > 1e-9]
    got = st.sample(u)
    assert np.array_equal(got.astype(np.int64), np.floor(8 * u).astype(np.int64))
    assert abs(st.marginal_probability([1, 2, 0] + [0] * (n - 3)) - 0.25) < 1e-13
    st.close()
    del st
    torch.cuda.empty_cache()
