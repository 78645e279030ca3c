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


@pytest.mark.parametrize("n", [2, 11, 12, 15, 17])
@pytest.mark.parametrize("dtype", [2, 1])
def test_transition_amplitude_tiled_kinds(qs, n, dtype):
    """Every observable kind of the tiled passes (Ising, Heisenberg with Y pairs, one flip group
    with many Z patterns, random strings, some too wide for a tile) against the oracle on the
    states the GPU holds."""
    from test_gpu_expect import observables
    bra0, ket0 = W.random_state(n, 40 + n), W.random_state(n, 80 + n) * 0.8
    bra, ket = qs.State(n, dtype), qs.State(n, dtype)
    bra.load(bra0)
    ket.load(ket0)
    vb, vk = bra.get_vector().astype(np.complex128), ket.get_vector().astype(np.complex128)
    nb, nk = float(np.linalg.norm(vb)), float(np.linalg.norm(vk))
    for name, obs in observables(n, 2000 + n).items():
        ref = oracle.transition_amplitude(vb, vk, n, obs)
        got = bra.transition_amplitude(obs, ket)
        scale = float(np.sum(np.abs(obs.coef))) * nb * nk
        assert abs(got - ref) <= 1e-13 * max(1.0, scale), (name, got, ref)
    bra.close()
    ket.close()


def single_qubit_state(theta, phi):
    return np.array([math.cos(theta / 2), complex(math.cos(phi), math.sin(phi)) * math.sin(theta / 2)])


PAULI = {(0, 0): np.eye(2), (1, 0): np.array([[0, 1], [1, 0]]), (1, 1): np.array([[0, -1j], [1j, 0]]),
         (0, 1): np.diag([1.0, -1.0])}


def test_transition_amplitude_full_size(qs):
    """n = 30 complex128: two product states from U3 gates, an observable with nearest-neighbour
    ZZ, XX and YY, single X, Y and Z and a wide Y string; <bra|P|ket> factorises over qubits."""
    import torch
    n = 30
    rng = W.SplitMix64(404)
    ang = [[(math.pi * rng.uniform(), 2 * math.pi * rng.uniform()) for _ in range(n)] for _ in range(2)]
    states = []
    for a in ang:
        st = qs.State(n, 2)
        st.run(W.Circuit(n, [W.Gate("U3", (q,), params=(a[q][0], a[q][1], 0.0)) for q in range(n)]), 0)
        states.append(st)
    terms = []
    for i in range(n - 1):
        m = (1 << i) | (1 << (i + 1))
        terms += [(rng.uniform_range(-1, 1), 0, m), (rng.uniform_range(-1, 1), m, 0), (rng.uniform_range(-1, 1), m, m)]
    for q in range(n):
        terms += [(rng.uniform_range(-1, 1), 1 << q, 0), (rng.uniform_range(-1, 1), 1 << q, 1 << q),
                  (rng.uniform_range(-1, 1), 0, 1 << q)]
    wide = sum(1 << q for q in range(3, 30, 2))
    terms.append((0.9, wide, wide))
    obs = W.PauliObservable(n, np.array([t[0] for t in terms]), np.array([t[1] for t in terms], dtype=np.uint64),
                            np.array([t[2] for t in terms], dtype=np.uint64))
    b1 = [single_qubit_state(*ang[0][q]) for q in range(n)]
    k1 = [single_qubit_state(*ang[1][q]) for q in range(n)]
    ref = 0j
    for c, xm, zm in zip(obs.coef, obs.x_mask, obs.z_mask):
        v = complex(c)
        for q in range(n):
            v *= np.vdot(b1[q], PAULI[((int(xm) >> q) & 1, (int(zm) >> q) & 1)] @ k1[q])
        ref += v
    got = states[0].transition_amplitude(obs, states[1])
    assert abs(got - ref) < 1e-11, (got, ref)
    for st in states:
        st.close()
    del states
    torch.cuda.empty_cache()
