"""GPU parity of the tiled Pauli-expectation passes (Sec. 4.5) against the oracle.

Observables whose flip-mask groups share tiles (transverse-field Ising, Heisenberg chains with Y
pairs), groups with many terms whose Z patterns vary over the item bits (the Walsh-Hadamard
route), random strings (some too wide for a tile, which take single-group launches), identity
terms; complex128 and complex64; n from 1 (a partial tile) to 30 (closed forms of a product
state)."""
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


def obs_from(n, terms):
    coef = np.array([t[0] for t in terms], dtype=np.float64)
    xm = np.array([t[1] for t in terms], dtype=np.uint64)
    zm = np.array([t[2] for t in terms], dtype=np.uint64)
    return W.PauliObservable(n, coef, xm, zm)


def heisenberg(n, rng):
    """sum_i a_i X_i X_{i+1} + b_i Y_i Y_{i+1} + c_i Z_i Z_{i+1} with random weights."""
    terms = []
    for i in range(n - 1):
        m = (1 << i) | (1 << (i + 1))
        terms += [(rng.uniform_range(-1, 1), m, 0), (rng.uniform_range(-1, 1), m, m), (rng.uniform_range(-1, 1), 0, m)]
    if n == 1:
        terms.append((0.5, 1, 1))
    return obs_from(n, terms)


def one_group_many_z(n, rng):
    """70 terms sharing one flip mask with random Z patterns (Re and Im components, several
    item masks per thread), single Y terms on every qubit and an identity term."""
    f = (1 << (n - 1)) | (2 if n > 2 else 0) if n > 1 else 1
    terms = [(rng.uniform_range(-1, 1), f, rng.next_u64() & ((1 << n) - 1)) for _ in range(70)]
    terms += [(rng.uniform_range(-1, 1), 1 << q, 1 << q) for q in range(n)]
    terms.append((0.3, 0, 0))
    return obs_from(n, terms)


def many_z_strings(n, rng):
    """Diagonal group only: 60 random Z strings (the transform over 16 items)."""
    return obs_from(n, [(rng.uniform_range(-1, 1), 0, rng.next_u64() & ((1 << n) - 1)) for _ in range(60)])


def observables(n, seed):
    rng = W.SplitMix64(seed)
    return {"tfim": W.tfim_observable(n, 0.8), "heisenberg": heisenberg(n, rng),
            "random": W.random_pauli_observable(n, 14, seed), "one_group": one_group_many_z(n, rng),
            "z_strings": many_z_strings(n, rng)}


@pytest.mark.parametrize("n", [1, 2, 5, 11, 12, 13, 16, 19])
@pytest.mark.parametrize("dtype", [2, 1])
def test_tiled_expectation_vs_oracle(qs, n, dtype):
    """Every observable kind against the oracle on the state the GPU holds (the complex64 state
    rounded to float, so both sides sum the same amplitudes): FP64-class accuracy for both dtypes."""
    psi0 = W.random_state(n, 7 * n + dtype) * 1.2
    st = qs.State(n, dtype)
    st.load(psi0)
    vec = st.get_vector().astype(np.complex128)
    for name, obs in observables(n, 1000 + n).items():
        ref, _ = oracle.expectation(vec, obs)
        scale = float(np.sum(np.abs(obs.coef))) * float(np.vdot(vec, vec).real)
        got, gim = st.expectation(obs)
        assert abs(got - ref) <= 1e-13 * max(1.0, scale) + 1e-14, (name, got, ref)
        assert gim == 0.0
    st.close()


def test_tiled_expectation_scaled_state(qs):
    """Amplitudes spread over many orders of magnitude (tiles of very different norm) and exact
    zeros: the grid sums follow each thread's own scale."""
    n = 15
    psi0 = W.random_state(n, 3)
    psi0[: 1 << 10] *= 1e-7
    psi0[1 << 12: 1 << 13] = 0.0
    psi0[-64:] *= 300.0
    for dtype in (2, 1):
        st = qs.State(n, dtype)
        st.load(psi0)
        vec = st.get_vector().astype(np.complex128)
        for obs in observables(n, 77).values():
            ref, _ = oracle.expectation(vec, obs)
            scale = float(np.sum(np.abs(obs.coef))) * float(np.vdot(vec, vec).real)
            assert abs(st.expectation(obs)[0] - ref) <= 1e-13 * scale
        st.close()


def product_state_expectation(thetas, phis, obs):
    """<P> on the product state prod_q U3(theta_q, phi_q, 0)|0>: each qubit's Bloch vector is
    (sin t cos p, sin t sin p, cos t), and a Pauli string's value is the product of its factors."""
    bloch = [(math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)) for t, p in zip(thetas, phis)]
    total = 0.0
    for c, xm, zm in zip(obs.coef, obs.x_mask, obs.z_mask):
        v = float(c)
        for q in range(len(thetas)):
            x, z = (int(xm) >> q) & 1, (int(zm) >> q) & 1
            if x and z:
                v *= bloch[q][1]
            elif x:
                v *= bloch[q][0]
            elif z:
                v *= bloch[q][2]
        total += v
    return total


@pytest.mark.parametrize("dtype", [2, 1])
def test_tiled_expectation_full_size(qs, dtype):
    """n = 30: a product state from U3 gates, an observable with nearest-neighbour ZZ, XX and
    YY, single X, Y and Z, long-range XZ and Y...Y strings (tile and single-group reads),
    against the closed form."""
    import torch
    n = 30
    rng = W.SplitMix64(303)
    thetas = [math.pi * rng.uniform() for _ in range(n)]
    phis = [2 * math.pi * rng.uniform() for _ in range(n)]
    c = W.Circuit(n, [W.Gate("U3", (q,), params=(thetas[q], phis[q], 0.0)) for q in range(n)])
    terms = []
    for i in range(n - 1):
        m = (1 << i) | (1 << (i + 1))
        terms += [(rng.uniform_range(-1, 1), 0, m), (rng.uniform_range(-1, 1), m, 0), (rng.uniform_range(-1, 1), m, m)]
    for q in range(n):
        terms += [(rng.uniform_range(-1, 1), 1 << q, 0), (rng.uniform_range(-1, 1), 1 << q, 1 << q),
                  (rng.uniform_range(-1, 1), 0, 1 << q)]
    for i in range(n - 7):
        terms.append((rng.uniform_range(-1, 1), 1 << i, 1 << (i + 7)))
    wide = sum(1 << q for q in range(3, 30, 2))     # 14 Y factors above qubit 2: a single-group read
    terms.append((0.9, wide, wide))
    terms.append((0.25, 0, 0))
    obs = obs_from(n, terms)
    ref = product_state_expectation(thetas, phis, obs)
    st = qs.State(n, dtype)
    st.run(c, 0)
    got, _ = st.expectation(obs)
    assert abs(got - ref) < (1e-11 if dtype == 2 else 2e-5), (got, ref)
    st.close()
    del st
    torch.cuda.empty_cache()
