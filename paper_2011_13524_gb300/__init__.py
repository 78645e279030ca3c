"""Python binding of libqsim_gb300.so, the GB300 state-vector simulator.

Argument marshalling only: every gate update, reduction and gradient runs in the
library's CUDA kernels. PyTorch supplies device memory and streams (a ``State`` can wrap
a ``torch.complex64`` / ``torch.complex128`` CUDA tensor, whose layout matches the
library's interleaved (re, im) amplitudes with qubit i in bit i of the index).

Gate records are any objects with the attributes of ``workloads.Gate`` (name, targets,
controls, control_values, params, matrix, pauli, param_index); circuits have ``n``,
``gates`` and ``n_params``; observables have ``n``, ``coef``, ``x_mask`` and ``z_mask``.
If the shared library is missing it is built with nvcc; if that fails the import fails:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

QS_OK = 0
QS_ERR_INVALID_ARG = 1
QS_ERR_OOM = 2
QS_ERR_CUDA = 3
QS_ERR_UNSUPPORTED = 4
QS_ERR_TIMEOUT = 5
QS_ERR_NUMERIC = 6

QS_C64 = 1
QS_C128 = 2
QS_MATH_FP64 = 0
QS_MATH_DF = 1

QS_MAX_TARGETS = 6
QS_MAX_CONTROLS = 8

QS_GATE_DENSE, QS_GATE_DIAG, QS_GATE_PAULI, QS_GATE_NAMED = 0, 1, 2, 3
QS_DEBUG_NONE, QS_DEBUG_TC_LATE, QS_DEBUG_BATCH_HOLD = 0, 1, 2
KERNEL_NAMES = {0: "dense_reg", 1: "dense_smem", 2: "diag", 3: "phase", 4: "pauli", 5: "swap", 6: "dense_df",
                8: "dense_oz", 9: "pauli_rot", 10: "dense_oz5", 11: "dense_bz"}
NAMED = {
    "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "Sdag": 6, "T": 7, "Tdag": 8, "sqrtX": 9,
    "sqrtXdag": 10, "sqrtY": 11, "sqrtYdag": 12, "RX": 13, "RY": 14, "RZ": 15, "U1": 16,
    "U2": 17, "U3": 18, "CNOT": 19, "CZ": 20, "SWAP": 21, "TOFFOLI": 22, "FREDKIN": 23,
    "PAULIROT": 24,
}


class QsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qsim error {code}: {msg}")
        self.code = code


class QsGate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("named", ctypes.c_int32), ("m", ctypes.c_int32),
        ("targets", ctypes.c_int32 * QS_MAX_TARGETS), ("mc", ctypes.c_int32),
        ("controls", ctypes.c_int32 * QS_MAX_CONTROLS),
        ("control_values", ctypes.c_int32 * QS_MAX_CONTROLS),
        ("pauli", ctypes.c_int32 * QS_MAX_TARGETS), ("param_index", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("params", ctypes.c_double * 3),
        ("mat", ctypes.POINTER(ctypes.c_double)),
    ]


class QsCircuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_gates", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("gates", ctypes.POINTER(QsGate))]


class QsPauliObs(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("coef", ctypes.POINTER(ctypes.c_double)),
                ("x_mask", ctypes.POINTER(ctypes.c_uint64)),
                ("z_mask", ctypes.POINTER(ctypes.c_uint64))]


_lib = None
_VOIDP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_version": ([], ctypes.c_char_p),
    "qs_set_c128_math": ([ctypes.c_int], ctypes.c_int),
    "qs_get_c128_math": ([ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qs_set_tensor_cores": ([ctypes.c_int], ctypes.c_int),
    "qs_get_tensor_cores": ([ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qs_state_set_arith": ([_VOIDP, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "qs_state_get_arith": ([_VOIDP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qs_create_state": ([ctypes.c_int, ctypes.c_int, _VOIDP, ctypes.POINTER(_VOIDP)], ctypes.c_int),
    "qs_wrap_state": ([_VOIDP, ctypes.c_int, ctypes.c_int, _VOIDP, ctypes.POINTER(_VOIDP)], ctypes.c_int),
    "qs_destroy_state": ([_VOIDP], ctypes.c_int),
    "qs_state_info": ([_VOIDP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(_VOIDP)], ctypes.c_int),
    "qs_set_stream": ([_VOIDP, _VOIDP], ctypes.c_int),
    "qs_set_basis": ([_VOIDP, ctypes.c_uint64], ctypes.c_int),
    "qs_load": ([_VOIDP, _VOIDP, ctypes.c_int], ctypes.c_int),
    "qs_get_vector": ([_VOIDP, _VOIDP], ctypes.c_int),
    "qs_copy_state": ([_VOIDP, _VOIDP], ctypes.c_int),
    "qs_synchronize": ([_VOIDP], ctypes.c_int),
    "qs_apply_gate": ([_VOIDP, ctypes.POINTER(QsGate)], ctypes.c_int),
    "qs_apply_pauli_rotation": ([_VOIDP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
    "qs_transition_amplitude": ([_VOIDP, ctypes.POINTER(QsPauliObs), _VOIDP, _DP], ctypes.c_int),
    "qs_marginal_probability": ([_VOIDP, ctypes.POINTER(ctypes.c_int32), _DP], ctypes.c_int),
    "qs_sample": ([_VOIDP, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qs_apply_observable_rotation": ([_VOIDP, ctypes.POINTER(QsPauliObs), ctypes.c_double, ctypes.c_int], ctypes.c_int),
    "qs_apply_fused": ([_VOIDP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP], ctypes.c_int),
    "qs_run_circuit": ([_VOIDP, ctypes.POINTER(QsCircuit), ctypes.c_int], ctypes.c_int),
    "qs_plan_fusion": ([ctypes.POINTER(QsCircuit), ctypes.c_int, ctypes.POINTER(_VOIDP)], ctypes.c_int),
    "qs_clear_plan_cache": ([], ctypes.c_int),
    "qs_debug_set_wait_limit": ([ctypes.c_longlong], ctypes.c_int),
    "qs_debug_set_tile_rows": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "qs_dense_tile_rows": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                           ctypes.c_int),
    "qs_debug_set_fault": ([ctypes.c_int], ctypes.c_int),
    "qs_debug_fail_alloc": ([ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "qs_fused_info": ([_VOIDP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qs_fused_block": ([_VOIDP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _DP],
                       ctypes.c_int),
    "qs_apply_fused_circuit": ([_VOIDP, _VOIDP], ctypes.c_int),
    "qs_destroy_fused": ([_VOIDP], ctypes.c_int),
    "qs_fused_layout_passes": ([_VOIDP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "qs_fused_block_cost": ([_VOIDP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), _DP], ctypes.c_int),
    "qs_apply_fused_circuit_timed": ([_VOIDP, _VOIDP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "qs_autotune_fusion": ([ctypes.POINTER(QsCircuit), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP],
                           ctypes.c_int),
    "qs_expectation": ([_VOIDP, ctypes.POINTER(QsPauliObs), _DP], ctypes.c_int),
    "qs_expectation_plan": ([ctypes.c_int, ctypes.POINTER(QsPauliObs), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                            ctypes.c_int),
    "qs_expectation_noalloc": ([_VOIDP, ctypes.c_int, ctypes.c_int, _VOIDP, ctypes.POINTER(QsPauliObs), _DP],
                               ctypes.c_int),
    "qs_inner_product": ([_VOIDP, _VOIDP, _DP], ctypes.c_int),
    "qs_batch_create": ([_VOIDP, _VOIDP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VOIDP)], ctypes.c_int),
    "qs_batch_run": ([_VOIDP, _DP, _VOIDP, ctypes.c_int, _DP, _DP], ctypes.c_int),
    "qs_batch_info": ([_VOIDP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "qs_batch_destroy": ([_VOIDP], ctypes.c_int),
    "qs_batch_traffic": ([_VOIDP, _DP], ctypes.c_int),
    "qs_norm2": ([_VOIDP, _DP], ctypes.c_int),
    "qs_adjoint_grad": ([ctypes.POINTER(QsCircuit), _DP, ctypes.POINTER(QsPauliObs), ctypes.c_int, _VOIDP,
                         _DP, _DP], ctypes.c_int),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded shared library (built in-tree with nvcc if missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != QS_OK:
        raise QsError(rc, lib().qs_last_error().decode())


def exported_symbols() -> Sequence[str]:
    return list(_SIGNATURES)


def set_c128_math(mode: int) -> None:
    check(lib().qs_set_c128_math(int(mode)))


QS_TENSOR_C128 = 2
QS_TENSOR_C64X = 4


def set_tensor_cores(mask: int) -> None:
    """Tensor-core paths as a bit mask of QS_TENSOR_C128 / QS_TENSOR_C64X (0: CUDA cores only)."""
    check(lib().qs_set_tensor_cores(int(mask)))


def get_tensor_cores() -> int:
    m = ctypes.c_int(0)
    check(lib().qs_get_tensor_cores(ctypes.byref(m)))
    return m.value


def get_c128_math() -> int:
    m = ctypes.c_int(0)
    check(lib().qs_get_c128_math(ctypes.byref(m)))
    return m.value


# ------------------------------------------------------------------ marshalling
class _Keep:
    """Holds numpy buffers referenced by C structs for the lifetime of a call."""

    def __init__(self):
        self.refs = []

    def dptr(self, a) -> ctypes.POINTER(ctypes.c_double):
        a = np.ascontiguousarray(a)
        self.refs.append(a)
        return a.ctypes.data_as(_DP)


def fill_gate(cg: QsGate, g, keep: _Keep) -> None:
    ctypes.memset(ctypes.byref(cg), 0, ctypes.sizeof(cg))
    name = g.name
    cg.m = len(g.targets)
    if cg.m > QS_MAX_TARGETS or len(g.controls) > QS_MAX_CONTROLS:
        raise QsError(QS_ERR_INVALID_ARG, "too many targets or controls")
    for j, t in enumerate(g.targets):
        cg.targets[j] = int(t)
    cg.mc = len(g.controls)
    cvals = tuple(g.control_values) if g.control_values else (1,) * cg.mc
    for j, (c, v) in enumerate(zip(g.controls, cvals)):
        cg.controls[j] = int(c)
        cg.control_values[j] = int(v)
    for j, p in enumerate(g.params[:3]):
        cg.params[j] = float(p)
    cg.param_index = int(getattr(g, "param_index", -1))
    for j, p in enumerate(getattr(g, "pauli", ()) or ()):
        cg.pauli[j] = int(p)
    if name == "DENSE":
        cg.kind = QS_GATE_DENSE
        m = np.ascontiguousarray(g.matrix, dtype=np.complex128)
        cg.mat = keep.dptr(m.view(np.float64).reshape(-1))
    elif name == "DIAG":
        cg.kind = QS_GATE_DIAG
        d = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128).reshape(-1))
        cg.mat = keep.dptr(d.view(np.float64))
    elif name == "PAULI":
        cg.kind = QS_GATE_PAULI
    else:
        cg.kind = QS_GATE_NAMED
        cg.named = NAMED[name]


def make_gate(g) -> Tuple[QsGate, _Keep]:
    keep = _Keep()
    cg = QsGate()
    fill_gate(cg, g, keep)
    return cg, keep


def make_circuit(circuit) -> Tuple[QsCircuit, _Keep]:
    """Marshals a circuit into a qs_circuit. The gate array of a circuit without matrix gates is
    kept on the circuit object and reused while its gate list holds the same (immutable) gates,
    so a loop over parameter vectors does not rebuild it."""
    gates = circuit.gates
    cache = getattr(circuit, "_qs_marshal", None)
    if cache is not None and cache[0] == len(gates) and all(a is b for a, b in zip(cache[1], gates)):
        arr, keep = cache[2], cache[3]
    else:
        keep = _Keep()
        arr = (QsGate * max(1, len(gates)))()
        for i, g in enumerate(gates):
            fill_gate(arr[i], g, keep)
        keep.refs.append(arr)
        if all(g.name not in ("DENSE", "DIAG") for g in gates):
            try:
                circuit._qs_marshal = (len(gates), list(gates), arr, keep)
            except AttributeError:  # a circuit type that takes no new attributes
                pass
    c = QsCircuit(int(circuit.n), len(gates), int(getattr(circuit, "n_params", 0)), 0,
                  ctypes.cast(arr, ctypes.POINTER(QsGate)))
    return c, keep


def make_obs(obs) -> Tuple[QsPauliObs, _Keep]:
    keep = _Keep()
    coef = np.ascontiguousarray(obs.coef, dtype=np.float64)
    xm = np.ascontiguousarray(obs.x_mask, dtype=np.uint64)
    zm = np.ascontiguousarray(obs.z_mask, dtype=np.uint64)
    keep.refs += [coef, xm, zm]
    o = QsPauliObs(len(coef), 0, coef.ctypes.data_as(_DP), xm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                   zm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return o, keep


def expectation_plan(n: int, obs):
    """How qs_expectation reads an n-qubit state for obs (host only): (tile qubit masks of the
    tiled reads, number of single-group reads)."""
    o, keep = make_obs(obs)
    npass, nsingle = ctypes.c_int(0), ctypes.c_int(0)
    masks = (ctypes.c_uint64 * 64)()
    check(lib().qs_expectation_plan(int(n), ctypes.byref(o), ctypes.byref(npass), masks, 64, ctypes.byref(nsingle)))
    del keep
    return [int(masks[i]) for i in range(min(npass.value, 64))], nsingle.value


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ states
class State:
    """A 2^n-amplitude state vector on the GPU.

    ``State(n, dtype)`` allocates through torch (the library wraps the tensor);
    ``State(n, dtype, owned=True)`` lets the library allocate (qs_create_state).
    Either way the state starts as |0...0>.
    """

    def __init__(self, n: int, dtype: int = QS_C128, stream=None, owned: bool = False, tensor=None):
        import torch
        self.n = int(n)
        self.dtype = int(dtype)
        self.tensor = None
        h = ctypes.c_void_p()
        sp = _stream_ptr(stream)
        if owned:
            check(lib().qs_create_state(self.n, self.dtype, sp, ctypes.byref(h)))
        else:
            tdt = torch.complex64 if self.dtype == QS_C64 else torch.complex128
            fresh = tensor is None
            if fresh:
                tensor = torch.empty(1 << self.n, dtype=tdt, device="cuda")
            assert tensor.dtype == tdt and tensor.is_cuda and tensor.is_contiguous()
            assert tensor.numel() == (1 << self.n)
            self.tensor = tensor
            check(lib().qs_wrap_state(tensor.data_ptr(), self.n, self.dtype, sp, ctypes.byref(h)))
            if fresh:
                check(lib().qs_set_basis(h, 0))
        self.handle = h

    def set_arith(self, math: int = -1, tensor: int = -1) -> None:
        """This state's own complex128 arithmetic (QS_MATH_*) and tensor-core mask (QS_TENSOR_*);
        -1 follows the process-wide setting."""
        check(lib().qs_state_set_arith(self.handle, int(math), int(tensor)))

    def get_arith(self) -> Tuple[int, int]:
        m, t = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().qs_state_get_arith(self.handle, ctypes.byref(m), ctypes.byref(t)))
        return m.value, t.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            check(lib().qs_destroy_state(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- contents
    def set_basis(self, j: int):
        check(lib().qs_set_basis(self.handle, int(j)))

    def load(self, vec: np.ndarray):
        dt = np.complex64 if self.dtype == QS_C64 else np.complex128
        v = np.ascontiguousarray(vec, dtype=dt)
        assert v.size == (1 << self.n)
        check(lib().qs_load(self.handle, v.ctypes.data_as(_VOIDP), 0))
        check(lib().qs_synchronize(self.handle))

    def get_vector(self) -> np.ndarray:
        dt = np.complex64 if self.dtype == QS_C64 else np.complex128
        out = np.empty(1 << self.n, dtype=dt)
        check(lib().qs_get_vector(self.handle, out.ctypes.data_as(_VOIDP)))
        return out

    def synchronize(self):
        check(lib().qs_synchronize(self.handle))

    def copy_from(self, other: "State"):
        check(lib().qs_copy_state(other.handle, self.handle))

    # -- updates
    def apply_gate(self, g):
        cg, keep = make_gate(g)
        check(lib().qs_apply_gate(self.handle, ctypes.byref(cg)))

    def apply_fused(self, targets: Sequence[int], mat: np.ndarray):
        t = (ctypes.c_int * len(targets))(*targets)
        m = np.ascontiguousarray(np.asarray(mat, dtype=np.complex128)).view(np.float64).reshape(-1)
        check(lib().qs_apply_fused(self.handle, len(targets), t, m.ctypes.data_as(_DP)))

    def run(self, circuit, fusion_k: int = 0):
        c, keep = make_circuit(circuit)
        check(lib().qs_run_circuit(self.handle, ctypes.byref(c), int(fusion_k)))

    def apply_plan(self, plan: "FusedCircuit"):
        check(lib().qs_apply_fused_circuit(self.handle, plan.handle))

    def apply_plan_timed(self, plan: "FusedCircuit") -> np.ndarray:
        """Apply a plan with a CUDA event after every block; per-block device ms."""
        out = (ctypes.c_float * max(1, plan.n_blocks))()
        check(lib().qs_apply_fused_circuit_timed(self.handle, plan.handle, out))
        return np.array(out[: plan.n_blocks], dtype=np.float64)

    # -- reductions
    def apply_pauli_rotation(self, x_mask: int, z_mask: int, angle: float) -> None:
        """psi <- exp(i angle P / 2) psi for the Pauli string given by the masks (any length)."""
        check(lib().qs_apply_pauli_rotation(self.handle, int(x_mask), int(z_mask), float(angle)))

    def apply_observable_rotation(self, obs, angle: float, n_slices: int = 1) -> None:
        """First-order Trotter evolution exp(i angle H) of the observable H in n_slices steps."""
        o, keep = make_obs(obs)
        check(lib().qs_apply_observable_rotation(self.handle, ctypes.byref(o), float(angle), int(n_slices)))

    def transition_amplitude(self, obs, ket: "State") -> complex:
        """<self|H|ket> for the observable H."""
        o, keep = make_obs(obs)
        out = (ctypes.c_double * 2)()
        check(lib().qs_transition_amplitude(self.handle, ctypes.byref(o), ket.handle, out))
        return complex(out[0], out[1])

    def marginal_probability(self, measured_value: Sequence[int]) -> float:
        """Probability of the measured values (0, 1, or 2 for any) of qubits 0 .. n-1."""
        mv = np.ascontiguousarray(measured_value, dtype=np.int32)
        if mv.size != self.n:
            raise QsError(QS_ERR_INVALID_ARG, "one measured value per qubit")
        out = ctypes.c_double(0)
        check(lib().qs_marginal_probability(self.handle, mv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            ctypes.byref(out)))
        return out.value

    def sample(self, uniforms) -> np.ndarray:
        """Z-basis samples: for each uniform u in [0, 1), the first index whose cumulative
        probability exceeds u times the squared norm."""
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        out = np.zeros(max(1, u.size), dtype=np.uint64)
        check(lib().qs_sample(self.handle, int(u.size), u.ctypes.data_as(_DP),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out[: u.size]

    def expectation(self, obs) -> Tuple[float, float]:
        o, keep = make_obs(obs)
        out = (ctypes.c_double * 2)()
        check(lib().qs_expectation(self.handle, ctypes.byref(o), out))
        return out[0], out[1]

    def norm2(self) -> float:
        out = ctypes.c_double(0)
        check(lib().qs_norm2(self.handle, ctypes.byref(out)))
        return out.value

    def inner(self, other: "State") -> complex:
        out = (ctypes.c_double * 2)()
        check(lib().qs_inner_product(self.handle, other.handle, out))
        return complex(out[0], out[1])


class FusedCircuit:
    """A fusion plan (qs_plan_fusion) that can be applied many times."""

    def __init__(self, circuit, k: int):
        c, keep = make_circuit(circuit)
        h = ctypes.c_void_p()
        check(lib().qs_plan_fusion(ctypes.byref(c), int(k), ctypes.byref(h)))
        self.handle = h
        nb, ns = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().qs_fused_info(h, ctypes.byref(nb), ctypes.byref(ns)))
        self.n_blocks, self.n_source_gates = nb.value, ns.value

    def block(self, b: int):
        w = ctypes.c_int(0)
        t = (ctypes.c_int * QS_MAX_TARGETS)()
        check(lib().qs_fused_block(self.handle, b, ctypes.byref(w), t, None))
        mat = np.zeros((1 << w.value) ** 2 * 2)
        check(lib().qs_fused_block(self.handle, b, None, None, mat.ctypes.data_as(_DP)))
        return list(t[: w.value]), mat.view(np.complex128).reshape(1 << w.value, 1 << w.value)

    def block_cost(self, b: int, dtype: int):
        """(kernel name, launches, algorithmic bytes) of block b for a state of `dtype`."""
        k, l, by = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        check(lib().qs_fused_block_cost(self.handle, b, int(dtype), ctypes.byref(k), ctypes.byref(l),
                                        ctypes.byref(by)))
        return KERNEL_NAMES[k.value], l.value, by.value

    def layout_passes(self, dtype: int) -> int:
        """Separate layout-change passes a run of this plan adds (double-float complex128)."""
        p = ctypes.c_int(0)
        check(lib().qs_fused_layout_passes(self.handle, int(dtype), ctypes.byref(p)))
        return p.value

    def widths(self):
        out = []
        for b in range(self.n_blocks):
            w = ctypes.c_int(0)
            check(lib().qs_fused_block(self.handle, b, ctypes.byref(w), None, None))
            out.append(w.value)
        return out

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                lib().qs_destroy_fused(self.handle)
                self.handle = None
        except Exception:
            pass


def clear_plan_cache() -> None:
    """Forget the cached fusion partitions (the next run of any circuit plans it afresh)."""
    check(lib().qs_clear_plan_cache())


def dense_tile_rows(dtype: int, m: int):
    """(rows per thread of the shared-memory dense kernel for dtype and m targets under the current
    arithmetic setting, whether the autotuner timed it or a test set it)."""
    r, t = ctypes.c_int(0), ctypes.c_int(0)
    check(lib().qs_dense_tile_rows(int(dtype), int(m), ctypes.byref(r), ctypes.byref(t)))
    return r.value, bool(t.value)


def autotune_fusion(circuit, dtype: int = QS_C128):
    """(best width, predicted ms per candidate: index 0 = gate by gate, 1..6 = fused widths)."""
    c, keep = make_circuit(circuit)
    k = ctypes.c_int(0)
    pred = (ctypes.c_double * 7)()
    check(lib().qs_autotune_fusion(ctypes.byref(c), int(dtype), ctypes.byref(k), pred))
    return k.value, list(pred)


class Batch:
    """Many (circuit, observable) pairs evaluated in one persistent launch (qs_batch_*)."""

    def __init__(self, circuits, observables, dtype: int = QS_C64):
        assert len(circuits) == len(observables) and len(circuits) > 0
        self.count = len(circuits)
        keep = []
        carr = (QsCircuit * self.count)()
        oarr = (QsPauliObs * self.count)()
        for i, (c, o) in enumerate(zip(circuits, observables)):
            cc, k1 = make_circuit(c)
            oo, k2 = make_obs(o)
            carr[i] = cc
            oarr[i] = oo
            keep += [k1, k2]
        self.n_params = [int(c.n_params) for c in circuits]
        h = ctypes.c_void_p()
        check(lib().qs_batch_create(ctypes.cast(carr, _VOIDP), ctypes.cast(oarr, _VOIDP), self.count, int(dtype),
                                    ctypes.byref(h)))
        self.handle = h
        tp, npass, ws = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_size_t(0)
        check(lib().qs_batch_info(h, ctypes.byref(tp), ctypes.byref(npass), ctypes.byref(ws)))
        self.total_params, self.total_passes, self.workspace_bytes = tp.value, npass.value, ws.value
        tr = ctypes.c_double(0)
        check(lib().qs_batch_traffic(h, ctypes.byref(tr)))
        self.traffic_bytes = tr.value

    def run(self, theta=None, use_graph: bool = True, stream=None):
        """(energies, list of per-circuit gradient arrays)."""
        e = np.zeros(self.count)
        g = np.zeros(max(1, self.total_params))
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        assert th is None or th.size == self.total_params
        check(lib().qs_batch_run(self.handle, None if th is None else th.ctypes.data_as(_DP), _stream_ptr(stream),
                                 int(use_graph), e.ctypes.data_as(_DP), g.ctypes.data_as(_DP)))
        out, off = [], 0
        for p in self.n_params:
            out.append(g[off:off + p].copy())
            off += p
        return e, out

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                lib().qs_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def adjoint_grad(circuit, obs, theta: Optional[Sequence[float]] = None, dtype: int = QS_C128,
                 stream=None) -> Tuple[float, np.ndarray]:
    """Energy and full gradient by the library's reverse-sweep adjoint kernels."""
    c, keep = make_circuit(circuit)
    o, keep2 = make_obs(obs)
    P = int(circuit.n_params)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    grad = np.zeros(max(P, 1))
    e = ctypes.c_double(0)
    check(lib().qs_adjoint_grad(ctypes.byref(c), None if th is None else th.ctypes.data_as(_DP), ctypes.byref(o),
                                int(dtype), _stream_ptr(stream), ctypes.byref(e), grad.ctypes.data_as(_DP)))
    return e.value, grad[:P]


def _autograd():
    import torch

    class AdjointEnergy(torch.autograd.Function):
        """E(theta) = <psi(theta)|H|psi(theta)> with dE/dtheta from the adjoint kernels."""

        @staticmethod
        def forward(ctx, theta, circuit, obs, dtype=QS_C128):
            th = theta.detach().to("cpu", torch.float64).numpy()
            e, g = adjoint_grad(circuit, obs, th, dtype)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return torch.tensor(e, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None

    return AdjointEnergy


def __getattr__(name):
    if name == "AdjointEnergy":
        return _autograd()
    raise AttributeError(name)
