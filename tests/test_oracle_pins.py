"""Pins the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against an independent route fixed by the paper or by
mathematics: full 2^n x 2^n operators built with Kronecker products or entry by
entry from Eq. (update_decomp), matrix exponentials from scipy, closed-form states
(GHZ, QFT of a basis state), algebraic identities of the named gates and of Pauli
matrices, the paper's printed four-qubit observable, and finite differences for
gradients. A dropped term, a wrong sign, a wrong bit order or a transposed gate
matrix in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W

RNG_SEED = 1234
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kron_chain(ops_by_qubit, n):
    """Full operator sum-free tensor product: ops_by_qubit[q] acts on qubit q (identity if
    missing). Qubit n-1 is the left-most Kronecker factor (little-endian index, Sec. 4.2.1)."""
    full = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        full = np.kron(full, ops_by_qubit.get(q, np.eye(2)))
    return full


def entrywise_operator(n, targets, K, controls=(), cvals=()):
    """Full operator from Eq. (update_decomp): <x|K|y> = K~[r(x), r(y)] if x, y agree off the
    targets (and the controls hold), identity otherwise."""
    N = 1 << n
    tmask = sum(1 << t for t in targets)
    cmask = sum(1 << c for c in controls)
    cval = sum((1 << c) for c, v in zip(controls, cvals) if v)
    F = np.zeros((N, N), dtype=np.complex128)

    def r(x):
        return sum(((x >> t) & 1) << j for j, t in enumerate(targets))

    for x in range(N):
        for y in range(N):
            if (x & ~tmask) != (y & ~tmask):
                continue
            if (x & cmask) == cval:
                F[x, y] = K[r(x), r(y)]
            elif x == y:
                F[x, y] = 1.0
    return F


def rand_vec(n, rng):
    v = np.array([complex(rng.normal(), rng.normal()) for _ in range(1 << n)])
    return v


# ------------------------------------------------------------------ conventions
def test_little_endian_index():
    """Sec. 4.2.1 listing: basis index 2 of two qubits is |10>, i.e. qubit 1 set."""
    psi = oracle.zero_state(2)
    oracle.apply_gate(psi, 2, W.Gate("X", (1,)))
    assert np.allclose(psi, [0, 0, 1, 0])
    psi = oracle.zero_state(2)
    oracle.apply_gate(psi, 2, W.Gate("X", (0,)))
    assert np.allclose(psi, [0, 1, 0, 0])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_one_qubit_gate_vs_kron(n):
    rng = W.SplitMix64(RNG_SEED + n)
    for t in range(n):
        K = W.random_complex_matrix(2, rng)          # K need not be unitary (Sec. 4.3.2)
        v = rand_vec(n, rng)
        ref = kron_chain({t: K}, n) @ v
        psi = v.copy()
        oracle.apply_matrix(psi, n, (t,), K)
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_two_qubit_local_order_vs_kron():
    """Reading of the local index: bit j <-> targets[j], so K = B (x) A on targets (a, b)
    equals A on a and B on b."""
    rng = W.SplitMix64(7)
    n = 5
    for a, b in [(0, 1), (1, 0), (4, 2), (0, 4), (3, 1)]:
        A = W.random_complex_matrix(2, rng)
        B = W.random_complex_matrix(2, rng)
        v = rand_vec(n, rng)
        psi = v.copy()
        oracle.apply_matrix(psi, n, (a, b), np.kron(B, A))
        ref = kron_chain({a: A, b: B}, n) @ v
        assert np.max(np.abs(psi - ref)) < 1e-12


@pytest.mark.parametrize("m", [1, 2, 3])
def test_dense_vs_entrywise_operator(m):
    rng = W.SplitMix64(100 + m)
    n = 5
    for trial in range(6):
        qs = list(range(n))
        tg = []
        for _ in range(m):
            tg.append(qs.pop(rng.randint(0, len(qs) - 1)))
        ctrl, cv = (), ()
        if trial % 2 == 1 and len(qs) >= 2:
            ctrl = (qs.pop(rng.randint(0, len(qs) - 1)), qs.pop(rng.randint(0, len(qs) - 1)))
            cv = (rng.randint(0, 1), rng.randint(0, 1))
        K = W.random_complex_matrix(1 << m, rng)
        v = rand_vec(n, rng)
        psi = v.copy()
        oracle.apply_matrix(psi, n, tuple(tg), K, ctrl, cv)
        ref = entrywise_operator(n, tg, K, ctrl, cv) @ v
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_diagonal_vs_entrywise():
    rng = W.SplitMix64(5)
    n = 5
    for tg, ctrl, cv in [((2,), (), ()), ((0, 3), (), ()), ((4, 1, 2), (0,), (1,)), ((1,), (3, 4), (0, 1))]:
        d = np.array([complex(rng.normal(), rng.normal()) for _ in range(1 << len(tg))])
        v = rand_vec(n, rng)
        psi = v.copy()
        oracle.apply_diagonal(psi, n, tg, d, ctrl, cv)
        ref = entrywise_operator(n, tg, np.diag(d), ctrl, cv) @ v
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_controlled_gates_vs_projector_sum():
    """CNOT(c -> t) = |0><0|_c (x) I + |1><1|_c (x) X; control value 0 swaps the projectors."""
    rng = W.SplitMix64(9)
    n = 4
    P0 = np.diag([1.0, 0.0]).astype(np.complex128)
    P1 = np.diag([0.0, 1.0]).astype(np.complex128)
    X = oracle.PAULI[1]
    for c, t, val in [(0, 1, 1), (3, 0, 1), (2, 3, 0)]:
        Pa, Pb = (P0, P1) if val == 1 else (P1, P0)
        full = kron_chain({c: Pa}, n) + kron_chain({c: Pb, t: X}, n)
        v = rand_vec(n, rng)
        psi = v.copy()
        oracle.apply_gate(psi, n, W.Gate("CNOT", (t,), controls=(c,), control_values=(val,)))
        assert np.max(np.abs(psi - full @ v)) < 1e-12


def test_printed_dense_matrix_is_cnot():
    """The 4x4 DenseMatrix of the C++ appendix example on targets {0, 1}: under the local-bit
    reading it flips qubit 0 when qubit 1 is set, i.e. CNOT with control 1 and target 0."""
    M = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
    rng = W.SplitMix64(11)
    v = rand_vec(3, rng)
    a = v.copy()
    oracle.apply_matrix(a, 3, (0, 1), M)
    b = v.copy()
    oracle.apply_gate(b, 3, W.Gate("CNOT", (0,), controls=(1,), control_values=(1,)))
    assert np.max(np.abs(a - b)) < 1e-15


def test_swap_toffoli_fredkin_are_permutations():
    n = 4
    for x in range(1 << n):
        def run(g):
            psi = np.zeros(1 << n, dtype=np.complex128)
            psi[x] = 1
            oracle.apply_gate(psi, n, g)
            return int(np.argmax(np.abs(psi))), np.max(np.abs(psi))
        b = lambda q: (x >> q) & 1
        y, amp = run(W.Gate("SWAP", (1, 3)))
        exp = x & ~0b1010 | (b(1) << 3) | (b(3) << 1)
        assert y == exp and amp == 1
        y, _ = run(W.Gate("TOFFOLI", (2,), controls=(0, 3), control_values=(1, 1)))
        assert y == (x ^ (4 if b(0) and b(3) else 0))
        y, _ = run(W.Gate("FREDKIN", (0, 2), controls=(1,), control_values=(1,)))
        exp = x if not b(1) else (x & ~0b101 | (b(0) << 2) | (b(2) << 0))
        assert y == exp


# ------------------------------------------------------------------ named gates
def mat_of(name, params=()):
    return oracle.gate_action(W.Gate(name, (0,), params=tuple(params)))[2]


def test_named_gate_identities():
    X, Y, Z = oracle.PAULI[1], oracle.PAULI[2], oracle.PAULI[3]
    H, S, T = mat_of("H"), mat_of("S"), mat_of("T")
    assert np.allclose(H @ H, np.eye(2))
    assert np.allclose(H @ X @ H, Z)
    assert np.allclose(S @ S, Z)
    assert np.allclose(T @ T, S)
    assert np.allclose(mat_of("sqrtX") @ mat_of("sqrtX"), X)
    assert np.allclose(mat_of("sqrtY") @ mat_of("sqrtY"), Y)
    for g in ["S", "T", "sqrtX", "sqrtY"]:
        assert np.allclose(mat_of(g) @ mat_of(g + "dag"), np.eye(2))
    # Pauli algebra: XY = iZ, YZ = iX, ZX = iY, and anticommutation
    assert np.allclose(X @ Y, 1j * Z) and np.allclose(Y @ Z, 1j * X) and np.allclose(Z @ X, 1j * Y)
    assert np.allclose(X @ Z, -Z @ X)


@pytest.mark.parametrize("theta", [-2.7, -0.4, 0.0, 0.9, 3.1])
def test_rotations_are_matrix_exponentials(theta):
    """RX/RY/RZ = exp(+i theta P / 2), the sign of the paper's gate table, via scipy expm."""
    for name, pid in [("RX", 1), ("RY", 2), ("RZ", 3)]:
        ref = scipy.linalg.expm(1j * theta / 2 * oracle.PAULI[pid])
        assert np.allclose(mat_of(name, [theta]), ref, atol=1e-14)
    assert np.allclose(mat_of("RZ", [theta]), np.diag([np.exp(1j * theta / 2), np.exp(-1j * theta / 2)]))
    # multi-qubit Pauli rotation on local indices (bit j <-> ids[j])
    ids = (1, 3, 2)
    P = np.kron(oracle.PAULI[2], np.kron(oracle.PAULI[3], oracle.PAULI[1]))
    g = W.Gate("PAULIROT", (0, 1, 2), pauli=ids, params=(theta,))
    assert np.allclose(oracle.gate_action(g)[2], scipy.linalg.expm(1j * theta / 2 * P), atol=1e-13)


def test_u_gates_openqasm_relations():
    th, ph, la = 0.7, 1.9, -2.3
    U3 = mat_of("U3", [th, ph, la])
    assert np.allclose(U3.conj().T @ U3, np.eye(2))
    assert np.allclose(mat_of("U2", [ph, la]), mat_of("U3", [math.pi / 2, ph, la]))
    assert np.allclose(mat_of("U3", [0, 0, la]), np.diag(mat_of("U1", [la])))
    # U3(theta, -pi/2, pi/2) = exp(-i theta X / 2) = RX(-theta) in the paper's sign
    assert np.allclose(mat_of("U3", [th, -math.pi / 2, math.pi / 2]), mat_of("RX", [-th]))
    # U3(theta, 0, 0) = exp(-i theta Y / 2) = RY(-theta)
    assert np.allclose(mat_of("U3", [th, 0, 0]), mat_of("RY", [-th]))
    # U1 as a state update equals a phase on |1>
    psi = np.array([0.6, 0.8j])
    oracle.apply_gate(psi, 1, W.Gate("U1", (0,), params=(la,)))
    assert np.allclose(psi, [0.6, 0.8j * np.exp(1j * la)])


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 5, 10])
def test_ghz(n):
    gates = [W.Gate("H", (0,))] + [W.Gate("CNOT", (i,), controls=(0,), control_values=(1,)) for i in range(1, n)]
    psi = oracle.run_circuit(W.Circuit(n, gates))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


def qft_gates(n):
    """Textbook QFT: for q = n-1 down to 0: H(q), then controlled phase 2pi/2^(k+1) from each
    lower qubit; the output is bit-reversed (qubit q of the result carries bit n-1-q)."""
    gates = []
    for q in range(n - 1, -1, -1):
        gates.append(W.Gate("H", (q,)))
        for k, c in enumerate(range(q - 1, -1, -1), start=1):
            ph = 2 * math.pi / (1 << (k + 1))
            gates.append(W.Gate("DIAG", (q,), controls=(c,), control_values=(1,),
                                matrix=np.array([1, np.exp(1j * ph)])))
    return gates


@pytest.mark.parametrize("n,j", [(3, 5), (5, 0), (5, 19), (7, 100)])
def test_qft_of_basis_state(n, j):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[j] = 1
    psi = oracle.run_circuit(W.Circuit(n, qft_gates(n)), psi)
    N = 1 << n
    rev = [int(format(k, f"0{n}b")[::-1], 2) for k in range(N)]
    ref = np.array([np.exp(2j * math.pi * j * rev[k] / N) for k in range(N)]) / math.sqrt(N)
    assert np.max(np.abs(np.abs(psi) - N ** -0.5)) < 1e-13
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_x_on_all_qubits():
    n = 9
    psi = oracle.run_circuit(W.Circuit(n, [W.Gate("X", (q,)) for q in range(n)]))
    assert psi[-1] == 1 and np.count_nonzero(psi) == 1


def test_norm_preserved_by_unitary_circuits():
    for seed in range(3):
        c = W.u3cz_circuit(10, 6, seed)
        psi = oracle.run_circuit(c)
        assert abs(oracle.norm2(psi, 10) - 1.0) < 1e-13
    suite = W.random_gate_suite(7, 42)
    psi = oracle.run_circuit(W.Circuit(7, suite))
    assert abs(oracle.norm2(psi, 7) - 1.0) < 1e-13


def test_circuit_vs_full_unitary_product():
    """merge_all-style check (Sec. 5.4): the whole circuit as one 2^n x 2^n product of
    entry-wise gate operators, later gates on the left."""
    n = 5
    gates = W.random_gate_suite(n, 3)
    U = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        kind, t, data, c, cv = oracle.gate_action(g)
        K = data if kind == "dense" else np.diag(data)
        U = entrywise_operator(n, t, K, c, cv) @ U
    psi = oracle.run_circuit(W.Circuit(n, gates))
    assert np.max(np.abs(psi - U[:, 0])) < 1e-12


# ------------------------------------------------------------------ observables
def pauli_full(n, xm, zm):
    ops = {}
    for q in range(n):
        x, z = (xm >> q) & 1, (zm >> q) & 1
        pid = {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}[(x, z)]
        ops[q] = oracle.PAULI[pid]
    return kron_chain(ops, n)


def test_expectation_vs_full_matrix():
    rng = W.SplitMix64(77)
    for n in [1, 2, 4, 6]:
        obs = W.random_pauli_observable(n, 7, 1000 + n)
        v = W.random_state(n, 5 + n)
        O = sum(c * pauli_full(n, int(x), int(z)) for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
        ref = np.vdot(v, O @ v)
        re, im = oracle.expectation(v, obs)
        assert abs(re - ref.real) < 1e-13 and abs(im) < 1e-13 and abs(ref.imag) < 1e-13


def test_expectation_two_routes_and_identity_term():
    n = 6
    v = W.random_state(n, 8)
    v = v * 1.7                                           # not normalised
    obs = W.random_pauli_observable(n, 5, 31)
    total = 0.0
    for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask):
        total += c * oracle.inner(v, oracle.apply_pauli(v, n, int(x), int(z)), n).real
    assert abs(oracle.expectation(v, obs)[0] - total) < 1e-12
    ident = W.PauliObservable(n, np.array([0.37]), np.array([0], dtype=np.uint64), np.array([0], dtype=np.uint64))
    assert abs(oracle.expectation(v, ident)[0] - 0.37 * oracle.norm2(v, n)) < 1e-13


def test_pauli_apply_algebra():
    n = 3
    v = W.random_state(n, 3)
    # Y = i X Z on one qubit: apply Z then X then multiply by i
    y = oracle.apply_pauli(v, n, 0b010, 0b010)
    xz = 1j * oracle.apply_pauli(oracle.apply_pauli(v, n, 0, 0b010), n, 0b010, 0)
    assert np.allclose(y, xz)
    # P^2 = I
    p = oracle.apply_pauli(oracle.apply_pauli(v, n, 0b101, 0b110), n, 0b101, 0b110)
    assert np.allclose(p, v)


def load_printed_observable():
    coef, xm, zm = [], [], []
    with open(os.path.join(GOLDEN, "openfermion_4q_observable.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            coef.append(float(parts[0]))
            x = z = 0
            for tok in parts[1:]:
                if tok == "[]":
                    continue
                p, q = tok[0], int(tok[1:])
                if p in "XY":
                    x |= 1 << q
                if p in "YZ":
                    z |= 1 << q
            xm.append(x)
            zm.append(z)
    return W.PauliObservable(4, np.array(coef), np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64))


def test_printed_observable_on_basis_states():
    """The paper's printed 4-qubit observable: on a basis state only I/Z terms survive, each
    contributing coef * prod of Z eigenvalues; the file's header records three hand sums."""
    obs = load_printed_observable()
    assert obs.n_terms == 15
    hand = {0: 0.0, 3: -1.064939, 15: -0.361291}
    for b in range(16):
        psi = np.zeros(16, dtype=np.complex128)
        psi[b] = 1
        closed = 0.0
        for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask):
            if int(x) == 0:
                closed += c * (-1) ** bin(b & int(z)).count("1")
        re, im = oracle.expectation(psi, obs)
        assert abs(re - closed) < 1e-14 and abs(im) < 1e-15
        if b in hand:
            assert abs(re - hand[b]) < 1e-6
    # X/Y terms: against the full 16 x 16 matrix on a random state
    v = W.random_state(4, 12)
    O = sum(c * pauli_full(4, int(x), int(z)) for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
    assert np.allclose(O, O.conj().T)
    assert abs(oracle.expectation(v, obs)[0] - np.vdot(v, O @ v).real) < 1e-13


def test_inner_and_norm_vs_numpy():
    a = W.random_state(7, 1) * 2
    b = W.random_state(7, 2)
    assert abs(oracle.inner(a, b, 7) - np.vdot(a, b)) < 1e-13
    assert abs(oracle.norm2(a, 7) - np.vdot(a, a).real) < 1e-13


def test_z_expectation_on_basis():
    n = 5
    for b in [0, 7, 22, 31]:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[b] = 1
        for q in range(n):
            obs = W.PauliObservable(n, np.array([1.0]), np.array([0], dtype=np.uint64), np.array([1 << q], dtype=np.uint64))
            assert oracle.expectation(psi, obs)[0] == (-1 if (b >> q) & 1 else 1)


# ------------------------------------------------------------------ gradients
def test_parameter_shift_matches_finite_difference():
    c = W.hea_circuit(4, 3, 21)
    obs = W.tfim_observable(4, 1.0)
    idx = list(range(c.n_params))
    ps = oracle.grad_parameter_shift(c, obs, idx)
    fd = oracle.grad_finite_difference(c, obs, idx, h=1e-6)
    assert np.max(np.abs(ps - fd)) < 1e-8
    assert np.max(np.abs(ps)) > 1e-3


def test_parameter_shift_matches_brute_force_derivative():
    """d/dtheta of <0|U(theta)^+ O U(theta)|0> with U built from full matrices, where the
    derivative of exp(i theta P / 2) is (i/2) P exp(i theta P / 2)."""
    n = 3
    c = W.hea_circuit(n, 2, 4)
    obs = W.random_pauli_observable(n, 4, 6)
    O = sum(cf * pauli_full(n, int(x), int(z)) for cf, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
    theta = c.parameters()
    mats = []
    for g in c.bind(theta).gates:
        kind, t, data, cc, cv = oracle.gate_action(g)
        mats.append(entrywise_operator(n, t, data if kind == "dense" else np.diag(data), cc, cv))
    psi0 = np.zeros(1 << n, dtype=np.complex128); psi0[0] = 1
    grads = np.zeros(c.n_params)
    for gi, g in enumerate(c.gates):
        if g.param_index < 0:
            continue
        pid = {"RX": 1, "RY": 2, "RZ": 3}[g.name]
        P = entrywise_operator(n, g.targets, oracle.PAULI[pid])
        U = np.eye(1 << n, dtype=np.complex128)
        dU = np.eye(1 << n, dtype=np.complex128)
        for gj, M in enumerate(mats):
            U = M @ U
            dU = (M @ dU) if gj != gi else (0.5j * P @ M @ dU)
        grads[g.param_index] = 2 * np.vdot(U @ psi0, O @ (dU @ psi0)).real
    ps = oracle.grad_parameter_shift(c, obs, range(c.n_params))
    assert np.max(np.abs(ps - grads)) < 1e-12


# ---------------------------------------------------------------- Pauli and observable rotations
def random_masks(n, rng):
    xm = zm = 0
    while xm == 0 and zm == 0:
        for q in range(n):
            pid = int(rng.next_u64() % 4)
            if pid in (1, 2):
                xm |= 1 << q
            if pid in (2, 3):
                zm |= 1 << q
    return xm, zm


@pytest.mark.parametrize("n", [1, 3, 5])
def test_pauli_rotation_is_matrix_exponential(n):
    """exp(i angle P / 2) by the oracle's pass equals scipy's expm of the Kronecker-built Pauli
    string (Y strings, identity factors, every length)."""
    rng = W.SplitMix64(40 + n)
    for _ in range(6):
        xm, zm = random_masks(n, rng)
        angle = 4 * math.pi * rng.uniform() - 2 * math.pi
        v = rand_vec(n, rng)
        got = oracle.apply_pauli_rotation(v.copy(), n, xm, zm, angle)
        ref = scipy.linalg.expm(1j * angle / 2 * pauli_full(n, xm, zm)) @ v
        assert np.max(np.abs(got - ref)) < 1e-13
    # the identity string is the global phase exp(i angle / 2)
    v = rand_vec(n, rng)
    assert np.max(np.abs(oracle.apply_pauli_rotation(v.copy(), n, 0, 0, 0.8) - np.exp(0.4j) * v)) < 1e-15


def test_observable_rotation_commuting_terms_exact():
    """For commuting terms (Z strings and an identity term) every Trotter slicing equals
    expm(i angle H)."""
    n = 4
    obs = W.PauliObservable(n, np.array([0.7, -1.1, 0.4, 0.25]), np.zeros(4, dtype=np.uint64),
                            np.array([0b0011, 0b0110, 0b1001, 0], dtype=np.uint64))
    H = sum(c * pauli_full(n, int(x), int(z)) for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
    rng = W.SplitMix64(3)
    v = rand_vec(n, rng)
    ref = scipy.linalg.expm(1j * 0.9 * H) @ v
    for r in (1, 3, 10):
        assert np.max(np.abs(oracle.observable_rotation(v, n, obs, 0.9, r) - ref)) < 1e-13


def test_observable_rotation_trotter_error_falls_as_one_over_slices():
    """Non-commuting terms (transverse-field Ising chain): the first-order product approaches
    expm(i angle H) with an error falling like 1 / n_slices."""
    n = 4
    obs = W.tfim_observable(n, 1.0)
    H = sum(c * pauli_full(n, int(x), int(z)) for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
    rng = W.SplitMix64(4)
    v = rand_vec(n, rng)
    ref = scipy.linalg.expm(1j * 0.5 * H) @ v
    err = {r: np.max(np.abs(oracle.observable_rotation(v, n, obs, 0.5, r) - ref)) for r in (1, 4, 16, 64)}
    assert err[1] > 1e-3
    for r in (4, 16, 64):
        assert 0.15 < err[r] * r / err[1] < 2.0, err


# ---------------------------------------------------------------- analysis functions
def test_transition_amplitude_pins():
    """<bra|H|ket>: equals <psi|H|psi> (the oracle's expectation routine) when bra = ket, and
    vdot(bra, H ket) with H built from Kronecker products."""
    n = 4
    rng = W.SplitMix64(81)
    obs = W.random_pauli_observable(n, 6, 82)
    psi = rand_vec(n, rng)
    t = oracle.transition_amplitude(psi, psi, n, obs)
    e = oracle.expectation(psi, obs)
    assert abs(t - complex(e[0], e[1])) < 1e-13
    bra, ket = rand_vec(n, rng), rand_vec(n, rng)
    H = sum(float(c) * pauli_full(n, int(x), int(z)) for c, x, z in zip(obs.coef, obs.x_mask, obs.z_mask))
    assert abs(oracle.transition_amplitude(bra, ket, n, obs) - np.vdot(bra, H @ ket)) < 1e-13


def test_marginal_probability_pins():
    """Against slicing the state as an n-axis tensor (axis n-1-q is qubit q), the all-wildcard
    case is the squared norm, and a qubit's two outcomes add up to its wildcard."""
    n = 5
    rng = W.SplitMix64(83)
    psi = rand_vec(n, rng) * 1.3
    T = np.abs(psi.reshape((2,) * n)) ** 2
    for _ in range(10):
        mv = [int(rng.next_u64() % 3) for _ in range(n)]
        idx = tuple(slice(None) if mv[n - 1 - a] == 2 else mv[n - 1 - a] for a in range(n))
        assert abs(oracle.marginal_probability(psi, n, mv) - float(np.sum(T[idx]))) < 1e-13
        q = int(rng.next_u64() % n)
        m0, m1, m2 = list(mv), list(mv), list(mv)
        m0[q], m1[q], m2[q] = 0, 1, 2
        assert abs(oracle.marginal_probability(psi, n, m0) + oracle.marginal_probability(psi, n, m1) -
                   oracle.marginal_probability(psi, n, m2)) < 1e-13
    assert abs(oracle.marginal_probability(psi, n, [2] * n) - np.vdot(psi, psi).real) < 1e-13


def test_sampling_pins():
    """Inverse-CDF sampling: exact outcomes for a 1-qubit state with probabilities (1/4, 3/4) and
    for a basis state; outcome frequencies of many uniforms within 5 sigma of |psi_x|^2."""
    psi = np.array([0.5, math.sqrt(0.75)], dtype=np.complex128)
    assert list(oracle.sample(psi, [0.0, 0.1, 0.2499, 0.2501, 0.9])) == [0, 0, 0, 1, 1]
    e5 = np.zeros(8, dtype=np.complex128)
    e5[5] = 1j
    assert set(oracle.sample(e5, [0.0, 0.3, 0.99]).tolist()) == {5}
    n = 3
    rng = W.SplitMix64(84)
    v = rand_vec(n, rng)
    p = np.abs(v) ** 2 / np.vdot(v, v).real
    m = 20000
    u = np.array([rng.uniform() for _ in range(m)])
    counts = np.bincount(oracle.sample(v, u).astype(np.int64), minlength=8)
    assert np.all(np.abs(counts - m * p) < 5 * np.sqrt(m * p * (1 - p)) + 1)
