"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and lays out gate lists; it holds none of the
simulator's arithmetic (no gate matrices, no state updates). Both the oracle and
the CUDA path turn a ``Gate`` record into their own gate matrix.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles as (x >> 11) * 2**-53.

Workload shapes follow the paper's benchmark circuits (Sec. 6.6, random
rotation layers + CZ brickwork) and the variational usage it describes (Sec. 3.1,
Sec. 4.4 parametric circuits), with the sizes of the configured workloads:

* ``u3cz_circuit``: every layer applies U3 to each qubit, then CZ on (i, i+1) for
  i of the layer's parity (layer 0 starts at even i).
* ``hea_circuit``: hardware-efficient ansatz, RY then RZ on every qubit, then a CZ
  ladder (i, i+1) for i = 0..n-2, every rotation a distinct parameter.
* ``tfim_observable``: sum_i Z_i Z_{i+1} (open chain) + h sum_i X_i.
* ``random_pauli_observable``: random Pauli strings with weights in [-1, 1].
* ``batch_workload``: many small HEA circuits of uneven width and depth.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; one 64-bit output per call."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection-free modulo of 64 bits."""
        span = hi - lo + 1
        return lo + (self.next_u64() % span)

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass(frozen=True)
class Gate:
    """One gate of a circuit, as data.

    name: one of X Y Z H S Sdag T Tdag sqrtX sqrtXdag sqrtY sqrtYdag
          RX RY RZ U1 U2 U3 CNOT CZ SWAP TOFFOLI FREDKIN DENSE DIAG PAULI PAULIROT
    targets: target qubits in the order that defines the local index of ``matrix``
             (target j <-> bit j of the local index).
    controls / control_values: control qubits and the value each must hold.
    params: rotation angles (RX/RY/RZ/U1/U2/U3/PAULIROT).
    matrix: complex 2^m x 2^m (DENSE, row = output) or length-2^m diagonal (DIAG).
    pauli: Pauli ids 0..3 (I X Y Z) per target (PAULI, PAULIROT).
    param_index: index into a parameter vector for a parametric rotation, else -1.
    """

    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    control_values: Tuple[int, ...] = ()
    params: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = field(default=None, compare=False)
    pauli: Tuple[int, ...] = ()
    param_index: int = -1

    def with_param(self, theta: float) -> "Gate":
        return Gate(self.name, self.targets, self.controls, self.control_values, (theta,),
                    self.matrix, self.pauli, self.param_index)


@dataclass
class Circuit:
    n: int
    gates: List[Gate]
    n_params: int = 0

    def parameters(self) -> np.ndarray:
        out = np.zeros(self.n_params)
        for g in self.gates:
            if g.param_index >= 0:
                out[g.param_index] = g.params[0]
        return out

    def bind(self, theta: Sequence[float]) -> "Circuit":
        gates = [g.with_param(float(theta[g.param_index])) if g.param_index >= 0 else g
                 for g in self.gates]
        return Circuit(self.n, gates, self.n_params)


@dataclass
class PauliObservable:
    """O = sum_k coef[k] P_k, P_k given by bit masks: x_mask bit q set for X or Y on q,
    z_mask bit q set for Z or Y on q (Y sets both)."""

    n: int
    coef: np.ndarray
    x_mask: np.ndarray
    z_mask: np.ndarray

    @property
    def n_terms(self) -> int:
        return len(self.coef)


def pauli_masks(ids: Sequence[int], qubits: Sequence[int]) -> Tuple[int, int]:
    """Masks of a Pauli string given as ids (0..3 = I X Y Z) on the listed qubits."""
    xm = zm = 0
    for pid, q in zip(ids, qubits):
        if pid in (1, 2):
            xm |= 1 << q
        if pid in (2, 3):
            zm |= 1 << q
    return xm, zm


def u3cz_circuit(n: int, depth: int, seed: int) -> Circuit:
    """Layered random circuit: U3 angles drawn (theta, phi, lambda) per qubit, in [0, 2pi)."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    two_pi = 2.0 * math.pi
    for layer in range(depth):
        for q in range(n):
            th = two_pi * rng.uniform()
            ph = two_pi * rng.uniform()
            la = two_pi * rng.uniform()
            gates.append(Gate("U3", (q,), params=(th, ph, la)))
        for i in range(layer % 2, n - 1, 2):
            gates.append(Gate("CZ", (i, i + 1)))
    return Circuit(n, gates)


def rzrxrz_cnot_circuit(n: int, reps: int, seed: int) -> Circuit:
    """Comparison-benchmark shape (Sec. 7): rotation layer RZ RX RZ on each qubit and a CNOT
    layer (target i, control (i+1) mod n), repeated, then a final rotation layer; the first RZ
    of the first layer and the last RZ of the last layer are dropped."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    two_pi = 2.0 * math.pi
    for r in range(reps + 1):
        for q in range(n):
            a1, a2, a3 = (two_pi * rng.uniform() for _ in range(3))
            if r != 0:
                gates.append(Gate("RZ", (q,), params=(a1,)))
            gates.append(Gate("RX", (q,), params=(a2,)))
            if r != reps:
                gates.append(Gate("RZ", (q,), params=(a3,)))
        if r == reps:
            break
        for i in range(n):
            gates.append(Gate("CNOT", (i,), controls=((i + 1) % n,), control_values=(1,)))
    return Circuit(n, gates)


def iqp_circuit(n: int, layers: int, seed: int) -> Circuit:
    """Commuting (IQP-like) circuit: H on every qubit, then `layers` diagonal layers (RZ with a
    seeded angle in [0, 2 pi) on every qubit, CZ(i, i+1) for i of the layer's parity), then H on
    every qubit. Every gate between the two H layers is diagonal."""
    rng = SplitMix64(seed)
    gates: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for layer in range(layers):
        for q in range(n):
            gates.append(Gate("RZ", (q,), params=(2.0 * math.pi * rng.uniform(),)))
        for i in range(layer % 2, n - 1, 2):
            gates.append(Gate("CZ", (i, i + 1)))
    gates += [Gate("H", (q,)) for q in range(n)]
    return Circuit(n, gates)


def hea_circuit(n: int, layers: int, seed: int, lo: float = -math.pi, hi: float = math.pi) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) on all qubits, RZ(theta) on all qubits,
    CZ ladder (i, i+1) for i = 0..n-2. Every rotation is its own parameter."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("RY", (q,), params=(rng.uniform_range(lo, hi),), param_index=p))
            p += 1
        for q in range(n):
            gates.append(Gate("RZ", (q,), params=(rng.uniform_range(lo, hi),), param_index=p))
            p += 1
        for i in range(n - 1):
            gates.append(Gate("CZ", (i, i + 1)))
    return Circuit(n, gates, n_params=p)


def tfim_observable(n: int, h: float = 1.0) -> PauliObservable:
    """sum_{i=0}^{n-2} Z_i Z_{i+1} + h sum_i X_i on an open chain."""
    coef, xm, zm = [], [], []
    for i in range(n - 1):
        coef.append(1.0)
        xm.append(0)
        zm.append((1 << i) | (1 << (i + 1)))
    for i in range(n):
        coef.append(h)
        xm.append(1 << i)
        zm.append(0)
    return PauliObservable(n, np.array(coef, dtype=np.float64), np.array(xm, dtype=np.uint64),
                           np.array(zm, dtype=np.uint64))


def random_pauli_observable(n: int, n_terms: int, seed: int) -> PauliObservable:
    """Each term: per qubit a uniform id in {I, X, Y, Z}; weight uniform in [-1, 1]."""
    rng = SplitMix64(seed)
    coef, xm, zm = [], [], []
    for _ in range(n_terms):
        ids = [rng.randint(0, 3) for _ in range(n)]
        x, z = pauli_masks(ids, range(n))
        coef.append(rng.uniform_range(-1.0, 1.0))
        xm.append(x)
        zm.append(z)
    return PauliObservable(n, np.array(coef, dtype=np.float64), np.array(xm, dtype=np.uint64),
                           np.array(zm, dtype=np.uint64))


def random_complex_matrix(dim: int, rng: SplitMix64) -> np.ndarray:
    """Gaussian complex matrix (input data for DENSE gates; not unitary in general)."""
    a = np.empty((dim, dim), dtype=np.complex128)
    for i in range(dim):
        for j in range(dim):
            a[i, j] = complex(rng.normal(), rng.normal())
    return a


def random_unitary(dim: int, rng: SplitMix64) -> np.ndarray:
    """Haar-distributed unitary from the QR decomposition of a Gaussian matrix
    (Mezzadri, Notices AMS 2007): Q with the phases of diag(R) divided out."""
    q, r = np.linalg.qr(random_complex_matrix(dim, rng))
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised Gaussian random state vector (complex128)."""
    rng = SplitMix64(seed)
    v = np.array([complex(rng.normal(), rng.normal()) for _ in range(1 << n)], dtype=np.complex128)
    return v / np.linalg.norm(v)


def random_state_fast(n: int, seed: int) -> np.ndarray:
    """Normalised random state for large n, drawn with numpy's Philox from the SplitMix64 seed."""
    rs = np.random.Generator(np.random.Philox(SplitMix64(seed).next_u64()))
    v = rs.standard_normal(1 << n) + 1j * rs.standard_normal(1 << n)
    return v / np.linalg.norm(v)


@dataclass
class BatchItem:
    circuit: Circuit
    observable: PauliObservable


def batch_workload(count: int, seed: int, n_lo: int = 8, n_hi: int = 20, l_lo: int = 2,
                   l_hi: int = 12, n_terms: int = 4) -> List[BatchItem]:
    """Independent (circuit, observable) pairs: n ~ U{n_lo..n_hi}, layers ~ U{l_lo..l_hi},
    HEA circuits with angles in [-pi, pi], random n_terms-term Pauli observables."""
    rng = SplitMix64(seed)
    items: List[BatchItem] = []
    for _ in range(count):
        n = rng.randint(n_lo, n_hi)
        layers = rng.randint(l_lo, l_hi)
        cseed = rng.next_u64()
        oseed = rng.next_u64()
        items.append(BatchItem(hea_circuit(n, layers, cseed), random_pauli_observable(n, n_terms, oseed)))
    return items


def random_gate_suite(n: int, seed: int) -> List[Gate]:
    """Every gate kind at random placements (for parity sweeps): named gates, rotations,
    dense 1..6-qubit unitaries, diagonal gates, controlled dense gates, Pauli strings."""
    rng = SplitMix64(seed)

    def pick(k: int) -> Tuple[int, ...]:
        qs = list(range(n))
        out = []
        for _ in range(k):
            j = rng.randint(0, len(qs) - 1)
            out.append(qs.pop(j))
        return tuple(out)

    gates: List[Gate] = []
    for name in ["X", "Y", "Z", "H", "S", "Sdag", "T", "Tdag", "sqrtX", "sqrtXdag", "sqrtY", "sqrtYdag"]:
        gates.append(Gate(name, pick(1)))
    for name in ["RX", "RY", "RZ", "U1"]:
        gates.append(Gate(name, pick(1), params=(rng.uniform_range(-math.pi, math.pi),)))
    gates.append(Gate("U2", pick(1), params=(rng.uniform_range(0, 6.28), rng.uniform_range(0, 6.28))))
    gates.append(Gate("U3", pick(1), params=tuple(rng.uniform_range(0, 6.28) for _ in range(3))))
    if n >= 2:
        c, t = pick(2)
        gates.append(Gate("CNOT", (t,), controls=(c,), control_values=(1,)))
        gates.append(Gate("CZ", pick(2)))
        gates.append(Gate("SWAP", pick(2)))
    if n >= 3:
        c1, c2, t = pick(3)
        gates.append(Gate("TOFFOLI", (t,), controls=(c1, c2), control_values=(1, 1)))
        c, t1, t2 = pick(3)
        gates.append(Gate("FREDKIN", (t1, t2), controls=(c,), control_values=(1,)))
    for m in range(1, min(n, 6) + 1):
        gates.append(Gate("DENSE", pick(m), matrix=random_unitary(1 << m, rng)))
    for m in range(1, min(n, 4) + 1):
        d = np.exp(1j * np.array([rng.uniform_range(-3.14, 3.14) for _ in range(1 << m)]))
        gates.append(Gate("DIAG", pick(m), matrix=d))
    if n >= 3:
        qs = pick(3)
        gates.append(Gate("DENSE", (qs[0],), controls=qs[1:], control_values=(0, 1),
                          matrix=random_unitary(2, rng)))
        qs = pick(3)
        gates.append(Gate("DENSE", qs[:2], controls=qs[2:], control_values=(1,),
                          matrix=random_unitary(4, rng)))
        qs = pick(3)
        gates.append(Gate("DIAG", qs[:1], controls=qs[1:], control_values=(1, 0),
                          matrix=np.exp(1j * np.array([0.3, -1.1]))))
    for m in range(1, min(n, 4) + 1):
        qs = pick(m)
        ids = tuple(rng.randint(1, 3) for _ in range(m))
        gates.append(Gate("PAULI", qs, pauli=ids))
        qs = pick(m)
        ids = tuple(rng.randint(1, 3) for _ in range(m))
        gates.append(Gate("PAULIROT", qs, pauli=ids, params=(rng.uniform_range(-3, 3),)))
    return gates
