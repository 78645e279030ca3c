"""FP64 CPU oracle for the state-vector simulator.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the bench's
``cpu_baseline`` / ``--impl reference`` legs may import this package. It shares no
code with the CUDA path and never imports it.

State convention (Sec. 4.2.1, the initialisation listing): amplitude index x has
qubit i in bit i ("the right-most digit is the 0-th qubit"); the state is a
complex128 numpy array of length 2**n.

Gate matrices of the named gates follow the paper's gate table (Sec. 4.3.4) with
these readings where the table is terse:
  * RX, RY, RZ(theta) = exp(+i theta P / 2) (the table's sign), PAULIROT the same on a
    Pauli string;
  * U1, U2, U3 follow OpenQASM 2 (the table defers to it);
  * S = diag(1, i), T = diag(1, e^{i pi/4}), sqrtX / sqrtY the principal square roots of
    X / Y ("pi/4 rotations" up to global phase), the *dag variants their adjoints;
  * a DENSE matrix has row = output, bit j of its local index <-> targets[j].
The update itself is the C library (``qsim_oracle.c``), plain loops per Eq. (update_mat).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.c_void_p
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_apply_matrix.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int, ip, ip]
        L.oracle_apply_matrix.restype = ctypes.c_int
        L.oracle_apply_diagonal.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int, ip, ip]
        L.oracle_apply_diagonal.restype = ctypes.c_int
        L.oracle_apply_pauli.argtypes = [dp, dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_apply_pauli.restype = None
        L.oracle_pauli_expectation.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                               ctypes.POINTER(ctypes.c_double)]
        L.oracle_pauli_expectation.restype = ctypes.c_double
        L.oracle_inner.argtypes = [dp, dp, ctypes.c_int, dp]
        L.oracle_inner.restype = None
        L.oracle_norm2.argtypes = [dp, ctypes.c_int]
        L.oracle_norm2.restype = ctypes.c_double
        L.oracle_threads.argtypes = []
        L.oracle_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _iarr(v: Sequence[int]):
    a = (ctypes.c_int * max(1, len(v)))(*[int(x) for x in v])
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return lib().oracle_threads()


# ---------------------------------------------------------------- gate matrices
SQ2 = 1.0 / math.sqrt(2.0)
PAULI = {
    0: np.array([[1, 0], [0, 1]], dtype=np.complex128),
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),
    2: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    3: np.array([[1, 0], [0, -1]], dtype=np.complex128),
}
FIXED_1Q = {
    "X": PAULI[1],
    "Y": PAULI[2],
    "Z": PAULI[3],
    "H": SQ2 * np.array([[1, 1], [1, -1]], dtype=np.complex128),
    "S": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "Sdag": np.array([[1, 0], [0, -1j]], dtype=np.complex128),
    "T": np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128),
    "Tdag": np.array([[1, 0], [0, np.exp(-1j * math.pi / 4)]], dtype=np.complex128),
    "sqrtX": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128),
    "sqrtXdag": 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]], dtype=np.complex128),
    "sqrtY": 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128),
    "sqrtYdag": 0.5 * np.array([[1 - 1j, 1 - 1j], [-1 + 1j, 1 - 1j]], dtype=np.complex128),
}


def pauli_string_matrix(ids: Sequence[int]) -> np.ndarray:
    """Matrix of a Pauli string on local indices: bit j of the local index <-> ids[j]."""
    m = np.array([[1.0 + 0j]])
    for pid in ids:               # later ids are more significant bits -> kron on the left
        m = np.kron(PAULI[pid], m)
    return m


def rotation(P: np.ndarray, theta: float) -> np.ndarray:
    """exp(i theta P / 2) for a Pauli string P (P^2 = I): cos(theta/2) I + i sin(theta/2) P."""
    return math.cos(theta / 2) * np.eye(P.shape[0], dtype=np.complex128) + 1j * math.sin(theta / 2) * P


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def gate_action(g) -> Tuple[str, tuple, np.ndarray, tuple, tuple]:
    """Turn a gate record into (kind, targets, data, controls, control_values) where kind is
    'dense' (data = 2^m x 2^m matrix) or 'diag' (data = 2^m diagonal)."""
    name = g.name
    t, c, cv = tuple(g.targets), tuple(g.controls), tuple(g.control_values)
    p = g.params
    if name in FIXED_1Q:
        return "dense", t, FIXED_1Q[name], c, cv
    if name in ("RX", "RY", "RZ"):
        pid = {"RX": 1, "RY": 2, "RZ": 3}[name]
        return "dense", t, rotation(PAULI[pid], p[0]), c, cv
    if name == "U1":
        return "diag", t, np.array([1.0, np.exp(1j * p[0])]), c, cv
    if name == "U2":
        return "dense", t, u3(math.pi / 2, p[0], p[1]), c, cv
    if name == "U3":
        return "dense", t, u3(p[0], p[1], p[2]), c, cv
    if name == "CNOT":           # X on the target, controlled
        return "dense", t, PAULI[1], c, cv
    if name == "TOFFOLI":
        return "dense", t, PAULI[1], c, cv
    if name == "CZ":             # diag(1,1,1,-1) on (t0, t1)
        return "diag", t, np.array([1, 1, 1, -1], dtype=np.complex128), c, cv
    if name in ("SWAP", "FREDKIN"):
        sw = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
        return "dense", t, sw, c, cv
    if name == "DENSE":
        return "dense", t, np.asarray(g.matrix, dtype=np.complex128), c, cv
    if name == "DIAG":
        return "diag", t, np.asarray(g.matrix, dtype=np.complex128).reshape(-1), c, cv
    if name == "PAULI":
        return "dense", t, pauli_string_matrix(g.pauli), c, cv
    if name == "PAULIROT":
        return "dense", t, rotation(pauli_string_matrix(g.pauli), p[0]), c, cv
    raise ValueError(f"unknown gate {name}")


# ---------------------------------------------------------------- state updates
def zero_state(n: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = 1.0
    return v


def apply_matrix(psi: np.ndarray, n: int, targets, K: np.ndarray, controls=(), cvals=()) -> None:
    K = np.ascontiguousarray(K, dtype=np.complex128)
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    r = lib().oracle_apply_matrix(_ptr(psi), n, len(targets), _iarr(targets), _ptr(K),
                                  len(controls), _iarr(controls), _iarr(cvals))
    if r != 0:
        raise ValueError("invalid gate arguments")


def apply_diagonal(psi: np.ndarray, n: int, targets, d: np.ndarray, controls=(), cvals=()) -> None:
    d = np.ascontiguousarray(d, dtype=np.complex128)
    r = lib().oracle_apply_diagonal(_ptr(psi), n, len(targets), _iarr(targets), _ptr(d),
                                    len(controls), _iarr(controls), _iarr(cvals))
    if r != 0:
        raise ValueError("invalid gate arguments")


def apply_gate(psi: np.ndarray, n: int, g) -> None:
    kind, t, data, c, cv = gate_action(g)
    if kind == "dense":
        apply_matrix(psi, n, t, data, c, cv)
    else:
        apply_diagonal(psi, n, t, data, c, cv)


def run_circuit(circuit, psi0: Optional[np.ndarray] = None) -> np.ndarray:
    """Apply the gates in order (Sec. 4.4: a circuit is an ordered gate array)."""
    n = circuit.n
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    for g in circuit.gates:
        apply_gate(psi, n, g)
    return psi


def apply_pauli(psi: np.ndarray, n: int, xmask: int, zmask: int) -> np.ndarray:
    out = np.empty_like(psi)
    lib().oracle_apply_pauli(_ptr(psi), _ptr(out), n, int(xmask), int(zmask))
    return out


def apply_pauli_rotation(psi: np.ndarray, n: int, xmask: int, zmask: int, angle: float) -> np.ndarray:
    """exp(i angle P / 2) psi = cos(angle/2) psi + i sin(angle/2) P psi (Sec. 4.3.2 Pauli rotation,
    the half-angle convention of the rotation gates), P given by masks."""
    return math.cos(angle / 2) * psi + 1j * math.sin(angle / 2) * apply_pauli(psi, n, xmask, zmask)


def observable_rotation(psi: np.ndarray, n: int, obs, angle: float, n_slices: int) -> np.ndarray:
    """First-order Trotter product [prod_k exp(i (angle / r) coef_k P_k)]^r psi, terms in order
    (Sec. 4.5 observable rotation)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    for _ in range(n_slices):
        for c, xm, zm in zip(obs.coef, obs.x_mask, obs.z_mask):
            out = apply_pauli_rotation(out, n, int(xm), int(zm), 2.0 * angle * float(c) / n_slices)
    return out


# ---------------------------------------------------------------- reductions
def expectation(psi: np.ndarray, obs) -> Tuple[float, float]:
    """(Re, Im) of sum_k coef_k <psi|P_k|psi>."""
    coef = np.ascontiguousarray(obs.coef, dtype=np.float64)
    xm = np.ascontiguousarray(obs.x_mask, dtype=np.uint64)
    zm = np.ascontiguousarray(obs.z_mask, dtype=np.uint64)
    im = ctypes.c_double(0.0)
    re = lib().oracle_pauli_expectation(_ptr(psi), obs.n, len(coef), _ptr(coef), _ptr(xm), _ptr(zm),
                                        ctypes.byref(im))
    return re, im.value


def inner(a: np.ndarray, b: np.ndarray, n: int) -> complex:
    out = np.zeros(2)
    lib().oracle_inner(_ptr(a), _ptr(b), n, _ptr(out))
    return complex(out[0], out[1])


def transition_amplitude(bra: np.ndarray, ket: np.ndarray, n: int, obs) -> complex:
    """<bra|H|ket> = sum_k coef_k <bra|P_k|ket> (Sec. 4.5), each term by applying P_k to ket."""
    total = 0j
    for c, xm, zm in zip(obs.coef, obs.x_mask, obs.z_mask):
        total += float(c) * inner(bra, apply_pauli(np.ascontiguousarray(ket, dtype=np.complex128), n, int(xm), int(zm)), n)
    return total


def marginal_probability(psi: np.ndarray, n: int, measured) -> float:
    """Sum of |psi_x|^2 over the x whose bit q equals measured[q] wherever measured[q] is 0 or 1
    (2 = any value), Sec. 4.2.2."""
    x = np.arange(1 << n, dtype=np.uint64)
    keep = np.ones(1 << n, dtype=bool)
    for q, v in enumerate(measured):
        if v in (0, 1):
            keep &= ((x >> np.uint64(q)) & np.uint64(1)) == np.uint64(v)
    return float(np.sum(np.abs(np.asarray(psi)[keep]) ** 2))


def sample(psi: np.ndarray, uniforms) -> np.ndarray:
    """For each u in [0, 1): the first index whose cumulative probability exceeds u times the
    total (Sec. 4.2.2 sampling, with the random numbers given)."""
    cdf = np.cumsum(np.abs(np.asarray(psi)) ** 2)
    return np.searchsorted(cdf, np.asarray(uniforms, dtype=np.float64) * cdf[-1], side="right").astype(np.uint64)


def norm2(psi: np.ndarray, n: int) -> float:
    return lib().oracle_norm2(_ptr(psi), n)


# ---------------------------------------------------------------- gradients
def energy(circuit, obs, theta: Optional[Sequence[float]] = None) -> float:
    c = circuit if theta is None else circuit.bind(theta)
    return expectation(run_circuit(c), obs)[0]


def grad_parameter_shift(circuit, obs, indices: Iterable[int]) -> np.ndarray:
    """dE/dtheta_j = [E(theta_j + pi/2) - E(theta_j - pi/2)] / 2, exact for a parameter that
    enters through exactly one gate exp(+-i theta P / 2)."""
    theta = circuit.parameters()
    out = []
    for j in indices:
        tp = theta.copy(); tp[j] += math.pi / 2
        tm = theta.copy(); tm[j] -= math.pi / 2
        out.append(0.5 * (energy(circuit, obs, tp) - energy(circuit, obs, tm)))
    return np.array(out)


def grad_finite_difference(circuit, obs, indices: Iterable[int], h: float = 1e-6) -> np.ndarray:
    """Central difference [E(theta_j + h) - E(theta_j - h)] / (2h)."""
    theta = circuit.parameters()
    out = []
    for j in indices:
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        out.append((energy(circuit, obs, tp) - energy(circuit, obs, tm)) / (2 * h))
    return np.array(out)
