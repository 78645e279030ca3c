"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (max-abs amplitude error): 1e-12 for complex128, 1e-5 for complex64, the bounds
the workload states; fidelity 1 - |<ref|psi>|^2 is reported beside them. Sizes span several
thread blocks and ragged tails (n = 1 .. 22); full-size (n = 30) runs are checked on sampled
amplitudes that a closed form gives one by one. Every test runs under both complex128
arithmetics (IEEE FP64, and double-float with tensor-core blocks, the library default).
"""
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


@pytest.fixture(scope="module", autouse=True, params=["fp64", "double-float"])
def c128_arith(qs, request):
    """Every test of this file runs with both complex128 arithmetics as the process-wide setting:
    IEEE FP64 kernels and double-float with tensor-core blocks (the default); complex64 tests run
    the same kernels twice. Tests that pick an arithmetic themselves restore this one."""
    old = qs.get_c128_math()
    qs.set_c128_math(qs.QS_MATH_FP64 if request.param == "fp64" else qs.QS_MATH_DF)
    yield request.param
    qs.set_c128_math(old)


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(b, dtype=np.complex128))))


def fidelity_gap(ref, psi):
    ref = np.asarray(ref, dtype=np.complex128)
    psi = np.asarray(psi, dtype=np.complex128)
    return 1.0 - abs(np.vdot(ref, psi)) ** 2 / (np.vdot(ref, ref).real * np.vdot(psi, psi).real)


def run_gpu(qs, circuit, dtype, fusion_k=0, psi0=None, owned=False):
    st = qs.State(circuit.n, dtype, owned=owned)
    if psi0 is not None:
        st.load(psi0)
    if fusion_k:
        st.run(circuit, fusion_k)
    else:
        for g in circuit.gates:
            st.apply_gate(g)
    out = st.get_vector()
    st.close()
    return out


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_every_gate_kind(qs, n, dtype):
    for seed in range(3):
        gates = W.random_gate_suite(n, 1000 * n + seed)
        psi0 = W.random_state(n, seed + 7)
        for g in gates:
            ref = psi0.copy()
            oracle.apply_gate(ref, n, g)
            got = run_gpu(qs, W.Circuit(n, [g]), dtype, psi0=psi0)
            assert maxabs(got, ref) < TOL[dtype], (g.name, g.targets, g.controls)


@pytest.mark.parametrize("dtype", [2, 1])
def test_dense_every_placement(qs, dtype):
    """1- and 2-qubit dense gates on every target (ordered pair) of n = 7, non-unitary K."""
    n = 7
    rng = W.SplitMix64(99)
    psi0 = W.random_state(n, 3)
    for t in range(n):
        g = W.Gate("DENSE", (t,), matrix=W.random_complex_matrix(2, rng) * 0.5)
        ref = psi0.copy(); oracle.apply_gate(ref, n, g)
        assert maxabs(run_gpu(qs, W.Circuit(n, [g]), dtype, psi0=psi0), ref) < TOL[dtype]
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            g = W.Gate("DENSE", (a, b), matrix=W.random_complex_matrix(4, rng) * 0.3)
            ref = psi0.copy(); oracle.apply_gate(ref, n, g)
            assert maxabs(run_gpu(qs, W.Circuit(n, [g]), dtype, psi0=psi0), ref) < TOL[dtype]


@pytest.mark.parametrize("m", [3, 4, 5, 6])
@pytest.mark.parametrize("dtype", [2, 1])
def test_wide_dense_with_controls(qs, m, dtype):
    n = 12
    rng = W.SplitMix64(7 + m)
    psi0 = W.random_state(n, 11)
    for trial in range(4):
        qs_ = list(range(n))
        picks = [qs_.pop(rng.randint(0, len(qs_) - 1)) for _ in range(m + 2)]
        ctrl = tuple(picks[m:]) if trial % 2 else ()
        cv = (1, 0) if trial % 2 else ()
        g = W.Gate("DENSE", tuple(picks[:m]), controls=ctrl, control_values=cv,
                   matrix=W.random_unitary(1 << m, rng))
        ref = psi0.copy(); oracle.apply_gate(ref, n, g)
        assert maxabs(run_gpu(qs, W.Circuit(n, [g]), dtype, psi0=psi0), ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [2, 1])
def test_config_n12_depth10(qs, dtype):
    """n = 12, |0..0>, depth-10 U3 + CZ brickwork: the final state and <Z0 Z1>."""
    c = W.u3cz_circuit(12, 10, 2021)
    ref = oracle.run_circuit(c)
    got = run_gpu(qs, c, dtype)
    assert maxabs(got, ref) < TOL[dtype]
    assert fidelity_gap(ref, got) < (1e-12 if dtype == 2 else 1e-6)
    zz = W.PauliObservable(12, np.array([1.0]), np.array([0], dtype=np.uint64), np.array([3], dtype=np.uint64))
    st = qs.State(12, dtype)
    st.run(c)
    e, ei = st.expectation(zz)
    assert abs(e - oracle.expectation(ref, zz)[0]) < (1e-12 if dtype == 2 else 1e-5)
    assert abs(ei) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype", [2, 1])
def test_fused_circuits(qs, k, dtype):
    n = 14
    for c in [W.u3cz_circuit(n, 6, 5), W.Circuit(n, W.random_gate_suite(n, 23)), W.rzrxrz_cnot_circuit(n, 3, 4)]:
        ref = oracle.run_circuit(c)
        got = run_gpu(qs, c, dtype, fusion_k=k)
        assert maxabs(got, ref) < TOL[dtype]


@pytest.mark.parametrize("n", [13, 17, 20, 22])
def test_circuit_family_vs_oracle(qs, n):
    c = W.u3cz_circuit(n, 8 if n > 20 else 20, n)
    ref = oracle.run_circuit(c)
    for k in (0, 2, 4):
        got = run_gpu(qs, c, 2, fusion_k=k)
        assert maxabs(got, ref) < 1e-12
    got = run_gpu(qs, c, 1, fusion_k=4)
    assert maxabs(got, ref) < 1e-5


@pytest.mark.parametrize("dtype", [2, 1])
def test_expectation_norm_inner(qs, dtype):
    for n in [1, 4, 9, 15]:
        psi = W.random_state(n, n) * 1.3
        obs = W.random_pauli_observable(n, 9, 100 + n)
        st = qs.State(n, dtype)
        st.load(psi)
        tol = 1e-12 if dtype == 2 else 2e-5
        re, im = st.expectation(obs)
        ore, oim = oracle.expectation(psi, obs)
        assert abs(re - ore) < tol and abs(im - oim) < tol
        assert abs(st.norm2() - oracle.norm2(psi, n)) < tol
        other = qs.State(n, dtype)
        phi = W.random_state(n, n + 50)
        other.load(phi)
        assert abs(st.inner(other) - oracle.inner(psi, phi, n)) < tol
    n = 16
    obs = W.tfim_observable(n, 1.0)
    c = W.u3cz_circuit(n, 4, 8)
    ref = oracle.run_circuit(c)
    st = qs.State(n, dtype)
    st.run(c, 2)
    assert abs(st.expectation(obs)[0] - oracle.expectation(ref, obs)[0]) < (1e-11 if dtype == 2 else 1e-4)


def test_identity_and_empty(qs):
    n = 3
    st = qs.State(n, 2)
    ident = W.PauliObservable(n, np.array([0.25]), np.array([0], dtype=np.uint64), np.array([0], dtype=np.uint64))
    assert abs(st.expectation(ident)[0] - 0.25) < 1e-15
    empty = W.PauliObservable(n, np.zeros(0), np.zeros(0, dtype=np.uint64), np.zeros(0, dtype=np.uint64))
    assert st.expectation(empty) == (0.0, 0.0)
    st.run(W.Circuit(n, []), 0)
    st.run(W.Circuit(n, []), 4)
    v = st.get_vector()
    assert v[0] == 1 and np.count_nonzero(v) == 1
    st.set_basis(5)
    assert st.get_vector()[5] == 1


def test_invalid_gate_reports_error(qs):
    st = qs.State(4, 2)
    with pytest.raises(qs.QsError) as e:
        st.apply_gate(W.Gate("H", (4,)))
    assert e.value.code == qs.QS_ERR_INVALID_ARG
    with pytest.raises(qs.QsError):
        st.apply_gate(W.Gate("CNOT", (1,), controls=(1,), control_values=(1,)))
    # the state is still usable afterwards
    st.apply_gate(W.Gate("X", (0,)))
    assert st.get_vector()[1] == 1


def test_library_owned_state(qs):
    c = W.u3cz_circuit(10, 5, 77)
    ref = oracle.run_circuit(c)
    assert maxabs(run_gpu(qs, c, 2, fusion_k=3, owned=True), ref) < 1e-12


@pytest.mark.parametrize("dtype", [2, 1])
def test_adjoint_gradient_vs_parameter_shift(qs, dtype):
    n = 6
    c = W.hea_circuit(n, 3, 12)
    obs = W.tfim_observable(n, 1.0)
    e, g = qs.adjoint_grad(c, obs, dtype=dtype)
    assert abs(e - oracle.energy(c, obs)) < (1e-12 if dtype == 2 else 1e-5)
    ps = oracle.grad_parameter_shift(c, obs, range(c.n_params))
    assert np.max(np.abs(g - ps)) < (1e-11 if dtype == 2 else 1e-4)
    # explicit theta
    theta = c.parameters() + 0.1
    e2, g2 = qs.adjoint_grad(c, obs, theta=theta, dtype=dtype)
    cb = c.bind(theta)
    assert abs(e2 - oracle.energy(cb, obs)) < (1e-12 if dtype == 2 else 1e-5)
    ps2 = oracle.grad_parameter_shift(cb, obs, range(0, c.n_params, 5))
    assert np.max(np.abs(g2[::5] - ps2)) < (1e-11 if dtype == 2 else 1e-4)


def test_adjoint_autograd_function(qs):
    import torch
    n = 4
    c = W.hea_circuit(n, 2, 3)
    obs = W.random_pauli_observable(n, 4, 9)
    theta = torch.tensor(c.parameters(), dtype=torch.float64, requires_grad=True)
    E = qs.AdjointEnergy.apply(theta, c, obs)
    E.backward()
    ps = oracle.grad_parameter_shift(c, obs, range(c.n_params))
    assert np.max(np.abs(theta.grad.numpy() - ps)) < 1e-11


# ---------------------------------------------------------------- full size, sampled outputs
def product_then_cz(n, depth, seed):
    """depth U3 layers on every qubit, then all CZ brickwork layers: amplitude x equals
    prod_q phi_q[x_q] * (-1)^{# CZ pairs with both bits set}, each phi_q a 1-qubit oracle run."""
    full = W.u3cz_circuit(n, depth, seed)
    u3 = [g for g in full.gates if g.name == "U3"]
    cz = [g for g in full.gates if g.name == "CZ"]
    return W.Circuit(n, u3 + cz), u3, cz


def sampled_amplitudes(n, u3, cz, xs):
    phis = []
    for q in range(n):
        phi = oracle.zero_state(1)
        for g in u3:
            if g.targets[0] == q:
                oracle.apply_gate(phi, 1, W.Gate("U3", (0,), params=g.params))
        phis.append(phi)
    out = []
    for x in xs:
        a = 1.0 + 0j
        for q in range(n):
            a *= phis[q][(x >> q) & 1]
        sgn = 1
        for g in cz:
            i, j = g.targets
            if (x >> i) & 1 and (x >> j) & 1:
                sgn = -sgn
        out.append(a * sgn)
    return np.array(out)


@pytest.mark.parametrize("fusion_k", [0, 4])
def test_full_size_n30_sampled(qs, fusion_k):
    import torch
    n = 30
    circ, u3, cz = product_then_cz(n, 20, 4242)
    st = qs.State(n, 2)
    st.run(circ, fusion_k)
    st.synchronize()
    rng = W.SplitMix64(5)
    xs = [rng.next_u64() & ((1 << n) - 1) for _ in range(2000)] + [0, (1 << n) - 1]
    ref = sampled_amplitudes(n, u3, cz, xs)
    idx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    got = st.tensor[idx].cpu().numpy()
    assert maxabs(got, ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-11
    st.close()
    del st
    torch.cuda.empty_cache()


def test_full_size_n30_fused_equals_unfused(qs):
    """Property at any size: the fused run equals the per-gate run, norm stays 1."""
    import torch
    n = 30
    c = W.u3cz_circuit(n, 3, 99)
    a = qs.State(n, 2)
    a.run(c, 0)
    b = qs.State(n, 2)
    b.run(c, 4)
    diff = (a.tensor - b.tensor).abs().max().item()
    assert diff < 1e-12
    assert abs(a.norm2() - 1.0) < 1e-11
    a.close(); b.close()
    del a, b
    torch.cuda.empty_cache()


def test_adjoint_mixed_rotations_and_pauli_rotation(qs):
    """Parametric RX, RY, RZ (fused reverse step) and a two-qubit PAULIROT (transition path),
    with a shared parameter, against parameter shift."""
    n = 5
    gates = [W.Gate("H", (0,)), W.Gate("RX", (1,), params=(0.4,), param_index=0),
             W.Gate("CNOT", (2,), controls=(1,), control_values=(1,)),
             W.Gate("PAULIROT", (0, 3), pauli=(1, 2), params=(-0.9,), param_index=1),
             W.Gate("RY", (4,), params=(1.3,), param_index=2), W.Gate("U3", (2,), params=(0.1, 0.5, -0.3)),
             W.Gate("RZ", (3,), params=(0.4,), param_index=0), W.Gate("CZ", (0, 4)),
             W.Gate("RZ", (2,), params=(2.2,), param_index=3)]
    c = W.Circuit(n, gates, n_params=4)
    obs = W.random_pauli_observable(n, 6, 77)
    for dtype, tol in ((2, 1e-11), (1, 1e-4)):
        e, g = qs.adjoint_grad(c, obs, dtype=dtype)
        ps = oracle.grad_parameter_shift(c, obs, range(4))
        assert abs(e - oracle.energy(c, obs)) < tol
        assert np.max(np.abs(g - ps)) < tol


def test_adjoint_diagonal_runs(qs):
    """Runs of diagonal gates in the reverse sweep (one pass per run): CZ ladders, a controlled
    phase, S and T, a 2-qubit DIAG gate with a control, RZ twice on one qubit inside a run, a
    parametric Z-string PAULIROT and a Z-string PAULI gate, between dense layers; complex128 and
    complex64 against parameter shift, and the energy against the oracle."""
    n = 7
    rng = W.SplitMix64(91)
    gates = [W.Gate("H", (q,)) for q in range(n)]
    gates += [W.Gate("RZ", (q,), params=(0.3 + 0.1 * q,), param_index=q) for q in range(n)]
    gates += [W.Gate("CZ", (q, q + 1)) for q in range(n - 1)]
    gates += [W.Gate("RZ", (2,), params=(-0.7,), param_index=7), W.Gate("S", (4,)), W.Gate("T", (1,)),
              W.Gate("U1", (5,), params=(0.9,), controls=(0,), control_values=(1,)),
              W.Gate("DIAG", (3, 6), controls=(2,), control_values=(0,),
                     matrix=np.exp(1j * np.array([0.1, -0.4, 0.8, 1.9]))),
              W.Gate("PAULIROT", (1, 4, 6), pauli=(3, 3, 3), params=(0.55,), param_index=8),
              W.Gate("PAULI", (0, 5), pauli=(3, 3)),
              W.Gate("RZ", (2,), params=(0.25,), param_index=9)]
    gates += [W.Gate("RY", (q,), params=(0.2 * q - 0.5,), param_index=10 + q) for q in range(n)]
    gates += [W.Gate("CZ", (q, q + 2)) for q in range(n - 2)]
    gates += [W.Gate("RZ", (q,), params=(1.1 - 0.3 * q,), param_index=10 + n + q) for q in range(n)]
    gates += [W.Gate("RX", (q,), params=(0.5,), param_index=2) for q in (0, 3)]  # shares RZ(2)'s angle
    c = W.Circuit(n, gates, n_params=10 + 2 * n)
    obs = W.random_pauli_observable(n, 8, 5150)
    # parameter 2 enters three gates: the two-point shift rule is exact only for one occurrence,
    # so that component is checked against central differences
    single = [p for p in range(c.n_params) if p != 2]
    ps = oracle.grad_parameter_shift(c, obs, single)
    fd2 = oracle.grad_finite_difference(c, obs, [2], h=1e-5)[0]
    e_ref = oracle.energy(c, obs)
    old = qs.get_c128_math()
    try:
        for dtype, math_mode, tol, fd_tol in ((2, qs.QS_MATH_DF, 1e-11, 1e-8), (2, qs.QS_MATH_FP64, 1e-11, 1e-8),
                                              (1, qs.QS_MATH_FP64, 1e-4, 1e-4)):
            qs.set_c128_math(math_mode)
            e, g = qs.adjoint_grad(c, obs, dtype=dtype)
            assert abs(e - e_ref) < tol, (dtype, math_mode)
            assert np.max(np.abs(g[single] - ps)) < tol, (dtype, math_mode, np.max(np.abs(g[single] - ps)))
            assert abs(g[2] - fd2) < fd_tol, (dtype, math_mode, g[2], fd2)
    finally:
        qs.set_c128_math(old)


def test_adjoint_cz_parities_and_wide_diagonal_runs(qs):
    """A diagonal run whose CZ gates are grouped by qubit distance (distances 1, 3 and 5, one CZ
    repeated so that it cancels) and whose uncontrolled single-qubit diagonals (RZ, T, S on every
    qubit) fill more than one table of 6 qubits, between RY layers: gradients against parameter
    shift and the energy against the oracle, in double-float, FP64 and complex64."""
    n = 9
    gates = [W.Gate("H", (q,)) for q in range(n)]
    gates += [W.Gate("RY", (q,), params=(0.3 + 0.07 * q,), param_index=q) for q in range(n)]
    gates += [W.Gate("CZ", (0, 1)), W.Gate("CZ", (2, 3)), W.Gate("CZ", (0, 1)), W.Gate("CZ", (1, 4)),
              W.Gate("CZ", (0, 5)), W.Gate("CZ", (3, 8)), W.Gate("CZ", (4, 5)), W.Gate("CZ", (6, 7))]
    gates += [W.Gate("RZ", (q,), params=(0.9 - 0.11 * q,), param_index=n + q) for q in range(n)]
    gates += [W.Gate("T", (q,)) for q in range(0, n, 2)] + [W.Gate("S", (q,)) for q in range(1, n, 2)]
    gates += [W.Gate("CZ", (q, q + 3)) for q in range(n - 3)]
    gates += [W.Gate("RY", (q,), params=(-0.4 + 0.05 * q,), param_index=2 * n + q) for q in range(n)]
    c = W.Circuit(n, gates, n_params=3 * n)
    obs = W.random_pauli_observable(n, 10, 777)
    ps = oracle.grad_parameter_shift(c, obs, list(range(c.n_params)))
    e_ref = oracle.energy(c, obs)
    old = qs.get_c128_math()
    try:
        for dtype, math_mode, tol in ((2, qs.QS_MATH_DF, 1e-11), (2, qs.QS_MATH_FP64, 1e-11), (1, qs.QS_MATH_FP64, 1e-4)):
            qs.set_c128_math(math_mode)
            e, g = qs.adjoint_grad(c, obs, dtype=dtype)
            assert abs(e - e_ref) < tol, (dtype, math_mode)
            assert np.max(np.abs(g - ps)) < tol, (dtype, math_mode, np.max(np.abs(g - ps)))
    finally:
        qs.set_c128_math(old)


def test_adjoint_zero_angles(qs):
    """Every parametric rotation at angle 0, where its matrix is the identity but its derivative
    is not: RX, RY and an XY Pauli rotation keep their rotation steps, RZ and a ZZ Pauli rotation
    their diagonal run, and single rotations, pairs sharing a pass and a CZ between them all give
    the parameter-shift gradient, in double-float, FP64 and complex64."""
    n = 6
    gates = [W.Gate("H", (q,)) for q in range(n)]
    gates += [W.Gate("RY", (q,), params=(0.3 + 0.1 * q,)) for q in range(n)]
    gates += [W.Gate("RX", (0,), params=(0.0,), param_index=0), W.Gate("RY", (1,), params=(0.0,), param_index=1),
              W.Gate("RZ", (2,), params=(0.0,), param_index=2),
              W.Gate("PAULIROT", (3, 4), pauli=(1, 2), params=(0.0,), param_index=3),
              W.Gate("PAULIROT", (4, 5), pauli=(3, 3), params=(0.0,), param_index=4),
              W.Gate("CZ", (0, 5)), W.Gate("RX", (5,), params=(0.0,), param_index=5)]
    gates += [W.Gate("RX" if q % 2 else "RY", (q,), params=(0.0,), param_index=6 + q) for q in range(n)]
    c = W.Circuit(n, gates, n_params=6 + n)
    obs = W.random_pauli_observable(n, 40, 70)
    ps = oracle.grad_parameter_shift(c, obs, range(c.n_params))
    assert np.min(np.abs(ps)) > 0.01  # no gradient of this case vanishes
    e_ref = oracle.energy(c, obs)
    old = qs.get_c128_math()
    try:
        for dtype, math_mode, tol in ((2, qs.QS_MATH_DF, 1e-11), (2, qs.QS_MATH_FP64, 1e-11), (1, qs.QS_MATH_FP64, 1e-4)):
            qs.set_c128_math(math_mode)
            e, g = qs.adjoint_grad(c, obs, dtype=dtype)
            assert abs(e - e_ref) < tol, (dtype, math_mode)
            assert np.max(np.abs(g - ps)) < tol, (dtype, math_mode, g, ps)
    finally:
        qs.set_c128_math(old)


def test_adjoint_hea_n12_vs_parameter_shift(qs):
    """The hardware-efficient ansatz of the differentiation configuration at n = 12 (RY and RZ
    layers, CZ ladders): the RZ layer and the ladder form one diagonal run per layer."""
    c = W.hea_circuit(12, 6, 4)
    obs = W.tfim_observable(12, 1.0)
    e, g = qs.adjoint_grad(c, obs)
    assert abs(e - oracle.energy(c, obs)) < 1e-12
    idx = list(range(0, c.n_params, 7))
    ps = oracle.grad_parameter_shift(c, obs, idx)
    assert np.max(np.abs(g[idx] - ps)) < 1e-11


@pytest.mark.parametrize("n", [12, 20])
def test_comparison_circuit_vs_oracle(qs, n):
    """The comparison circuit of Sec. 7 (RZ RX RZ rotation layers, CNOT ring with target i and
    control (i + 1) mod n, 10 repetitions and a final layer): complex128 at the autotuned width
    and complex64 against the oracle."""
    c = W.rzrxrz_cnot_circuit(n, 10, 700 + n)
    ref = oracle.run_circuit(c)
    for dtype in (2, 1):
        st = qs.State(n, dtype)
        st.run(c, -1)
        got = st.get_vector()
        st.close()
        assert maxabs(got, ref) < TOL[dtype], dtype
        assert fidelity_gap(ref, got) < (1e-12 if dtype == 2 else 1e-6)


def test_commuting_circuits_vs_oracle(qs):
    """Circuits whose fusion plans move blocks across commuting gates (an IQP-like circuit and
    the hardware-efficient ansatz), autotuned width, complex128 and complex64, against the oracle."""
    for c in (W.iqp_circuit(16, 12, 3), W.hea_circuit(16, 8, 4).bind(W.hea_circuit(16, 8, 4).parameters())):
        ref = oracle.run_circuit(c)
        for dtype in (2, 1):
            st = qs.State(c.n, dtype)
            st.run(c, -1)
            assert maxabs(st.get_vector(), ref) < TOL[dtype], dtype
            st.close()


@pytest.mark.parametrize("n", [24, 26])
def test_circuit_family_vs_oracle_large(qs, n):
    """The depth-20 U3+CZ family at n = 24 and 26 against the FP64 oracle (the largest sizes the
    oracle cross-check covers), complex128 at the autotuned width with the library's default
    arithmetic (double-float, tensor-core blocks) and on the double-float CUDA cores, whole
    vectors compared."""
    c = W.u3cz_circuit(n, 20, 300 + n)
    ref = oracle.run_circuit(c)
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    try:
        qs.set_c128_math(qs.QS_MATH_DF)
        for tmask in (qs.QS_TENSOR_C128, 0):
            qs.set_tensor_cores(tmask)
            st = qs.State(n, qs.QS_C128)
            st.run(c, -1)
            got = st.get_vector()
            st.close()
            assert maxabs(got, ref) < 1e-12, tmask
            assert fidelity_gap(ref, got) < 1e-12
    finally:
        qs.set_c128_math(old_m)
        qs.set_tensor_cores(old_t)


def test_precision_n24_vs_oracle(qs):
    """The precision configuration against the FP64 oracle at n = 24: complex64 (FP32 gates,
    FP64-built fused matrices, FP64 norm and expectation sums) and complex128 on the GPU;
    max-abs amplitude error, 1 - fidelity and the transverse-field Ising energy error (h = 1)."""
    n = 24
    c = W.u3cz_circuit(n, 20, 2424)
    ref = oracle.run_circuit(c)
    tf = W.tfim_observable(n, 1.0)
    e_ref = oracle.expectation(ref, tf)[0]
    for dtype, amp_tol, fid_tol, e_tol in ((2, 1e-12, 1e-12, 1e-11), (1, 1e-5, 1e-6, 1e-5)):
        st = qs.State(n, dtype)
        st.run(c, -1)
        got = st.get_vector().astype(np.complex128)
        assert maxabs(got, ref) < amp_tol, dtype
        assert fidelity_gap(ref, got) < fid_tol, dtype
        assert abs(st.expectation(tf)[0] - e_ref) < e_tol, dtype
        assert abs(st.norm2() - 1.0) < (1e-12 if dtype == 2 else 1e-5)
        st.close()


@pytest.mark.parametrize("dtype,math_mode", [(2, "df"), (2, "fp64"), (1, "fp64")])
def test_consecutive_diagonal_blocks_one_pass(qs, dtype, math_mode):
    """A circuit of diagonal gates only (RZ, CZ, T, S, controlled phases) fused at width 4: the
    plan's consecutive diagonal blocks run as one pass with their product in two tables (on at
    most 12 and at most 8 qubits; here a run uses both); the state matches the oracle and the
    block costs count one launch per pass."""
    n = 14
    rng = W.SplitMix64(1414)
    gates = []
    for layer in range(6):
        for q in range(n):
            gates.append(W.Gate("RZ", (q,), params=(4 * rng.uniform(),)))
        for q in range(layer % 2, n - 1, 2):
            gates.append(W.Gate("CZ", (q, q + 1)))
        gates.append(W.Gate("T", (int(rng.next_u64() % n),)))
        gates.append(W.Gate("S", (int(rng.next_u64() % n),)))
    c = W.Circuit(n, gates)
    psi0 = W.random_state(n, 99)
    ref = psi0.copy()
    for g in gates:
        oracle.apply_gate(ref, n, g)
    old = qs.get_c128_math()
    try:
        qs.set_c128_math(qs.QS_MATH_DF if math_mode == "df" else qs.QS_MATH_FP64)
        plan = qs.FusedCircuit(c, 4)
        costs = [plan.block_cost(b, dtype) for b in range(plan.n_blocks)]
        assert all(k in ("diag", "phase") for k, _, _ in costs)
        launches = sum(l for _, l, _ in costs)
        assert launches < plan.n_blocks  # several blocks share a pass
        second = set()  # qubits of the second table in the first run (greedy split)
        first = set()
        for b in range(plan.n_blocks):
            if b > 0 and costs[b][1]:
                break
            q = set(plan.block(b)[0])
            if len(first | q) <= 12:
                first |= q
            else:
                second |= q
        assert len(first) == 12 and 0 < len(second) <= 8
        full = 2 * (16 if dtype == 2 else 8) * 2 ** n
        assert all(by <= full and (l == 0) == (by == 0) for _, l, by in costs)
        st = qs.State(n, dtype)
        st.load(psi0)
        st.apply_plan(plan)
        assert maxabs(st.get_vector(), ref) < TOL[dtype]
        st.load(psi0)
        ms = st.apply_plan_timed(plan)
        assert len(ms) == plan.n_blocks
        assert maxabs(st.get_vector(), ref) < TOL[dtype]
    finally:
        qs.set_c128_math(old)


@pytest.mark.parametrize("dtype,math_mode", [(2, "df"), (2, "fp64"), (1, "fp64")])
def test_diagonal_run_quarter_turn_table(qs, dtype, math_mode):
    """A diagonal run whose second table holds only 1, i, -1, -i (two CZ and an S after three
    general 4-qubit diagonals filling the first table): the quarter turns are applied exactly by
    swaps and signs before the first table's entry; as the last pass of a double-float run it
    also writes IEEE doubles. The state matches the oracle."""
    n = 16
    rng = W.SplitMix64(1616)
    gates = []
    for b in range(3):
        d = np.exp(1j * 2 * np.pi * np.array([rng.uniform() for _ in range(16)]))
        gates.append(W.Gate("DIAG", tuple(range(4 * b, 4 * b + 4)), matrix=d))
    gates += [W.Gate("CZ", (12, 13)), W.Gate("CZ", (13, 14)), W.Gate("S", (14,))]
    c = W.Circuit(n, gates)
    psi0 = W.random_state(n, 161)
    ref = psi0.copy()
    for g in gates:
        oracle.apply_gate(ref, n, g)
    old = qs.get_c128_math()
    try:
        qs.set_c128_math(qs.QS_MATH_DF if math_mode == "df" else qs.QS_MATH_FP64)
        plan = qs.FusedCircuit(c, 4)
        costs = [plan.block_cost(b, dtype) for b in range(plan.n_blocks)]
        assert [l for _, l, _ in costs] == [1] + [0] * (plan.n_blocks - 1), costs
        assert set(plan.block(plan.n_blocks - 1)[0]) == {12, 13, 14}
        if dtype == 2 and math_mode == "df":
            assert plan.layout_passes(dtype) == 1  # entry only: the run writes IEEE doubles
        st = qs.State(n, dtype)
        st.load(psi0)
        st.apply_plan(plan)
        assert maxabs(st.get_vector(), ref) < TOL[dtype]
        st.close()
    finally:
        qs.set_c128_math(old)
