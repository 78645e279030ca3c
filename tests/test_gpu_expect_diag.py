"""GPU parity of the streaming pass for diagonal observables (every term a Z string, at most 12
distinct Z qubits; Sec. 4.5 with every flip mask zero) against the oracle: chains, single Z on
the lowest and highest qubit, strings over low and high qubits at once, an identity term;
n from 1 (a partial chunk) to 20, complex128 and complex64, and n = 30 against the closed form of
a product state."""
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


def z_obs(n, terms):
    return W.PauliObservable(n, np.array([t[0] for t in terms], dtype=np.float64),
                             np.zeros(len(terms), dtype=np.uint64),
                             np.array([t[1] for t in terms], dtype=np.uint64))


def diagonal_observables(n, seed):
    rng = W.SplitMix64(seed)
    top = n - 1
    qubits = sorted(set([0, min(1, top), min(5, top), n // 2, max(0, n - 2), top]))
    u = sum(1 << q for q in qubits)
    out = {
        "z0z1": z_obs(n, [(1.0, 3 if n > 1 else 1)]),
        "z_top": z_obs(n, [(-0.7, 1 << top), (0.25, 0)]),
        "chain": z_obs(n, [(rng.uniform_range(-1, 1), (1 << i) | (1 << (i + 1))) for i in range(min(n, 12) - 1)]
                       + [(0.5, 1)]),
        "spread": z_obs(n, [(rng.uniform_range(-1, 1), rng.next_u64() & u) for _ in range(40)]),
    }
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 10, 11, 12, 14, 20])
@pytest.mark.parametrize("dtype", [2, 1])
def test_diagonal_expectation_vs_oracle(qs, n, dtype):
    psi0 = W.random_state(n, 31 * n + dtype) * 0.9
    st = qs.State(n, dtype)
    st.load(psi0)
    vec = st.get_vector().astype(np.complex128)
    for name, obs in diagonal_observables(n, 500 + n).items():
        masks, single = qs.expectation_plan(n, obs)
        union = 0
        for z in obs.z_mask:
            union |= int(z)
        assert masks == [union] and single == 0, (name, masks)  # the one streaming read
        ref, _ = oracle.expectation(vec, obs)
        scale = float(np.sum(np.abs(obs.coef))) * float(np.vdot(vec, vec).real)
        got, gim = st.expectation(obs)
        assert abs(got - ref) <= 1e-13 * max(1.0, scale) + 1e-14, (name, got, ref)
        assert gim == 0.0
    st.close()


def test_diagonal_expectation_scaled_state(qs):
    """Amplitudes over many orders of magnitude and exact zeros."""
    n = 16
    psi0 = W.random_state(n, 9)
    psi0[: 1 << 11] *= 1e-9
    psi0[1 << 13: 1 << 14] = 0.0
    psi0[-100:] *= 500.0
    for dtype in (2, 1):
        st = qs.State(n, dtype)
        st.load(psi0)
        vec = st.get_vector().astype(np.complex128)
        for obs in diagonal_observables(n, 11).values():
            ref, _ = oracle.expectation(vec, obs)
            scale = float(np.sum(np.abs(obs.coef))) * float(np.vdot(vec, vec).real)
            assert abs(st.expectation(obs)[0] - ref) <= 1e-13 * scale
        st.close()


@pytest.mark.parametrize("dtype", [2, 1])
def test_diagonal_expectation_full_size(qs, dtype):
    """n = 30: U3 product state; <Z0 Z1> + ZZ on the top pair + single Z terms, against the
    product of each qubit's cos(theta)."""
    n = 30
    rng = W.SplitMix64(404)
    thetas = [math.pi * rng.uniform() for _ in range(n)]
    c = W.Circuit(n, [W.Gate("U3", (q,), params=(thetas[q], 2 * math.pi * rng.uniform(), 0.0)) for q in range(n)])
    terms = [(1.0, 3), (-0.5, (1 << 28) | (1 << 29)), (0.3, 1 << 5), (0.2, 1 << 17), (0.1, 0)]
    obs = z_obs(n, terms)
    want = 0.0
    for a, z in terms:
        v = a
        for q in range(n):
            if (z >> q) & 1:
                v *= math.cos(thetas[q])
        want += v
    st = qs.State(n, dtype)
    st.run(c, 0)
    got = st.expectation(obs)[0]
    assert abs(got - want) < (1e-12 if dtype == 2 else 1e-5), (got, want)
    st.close()
