"""The allocation-free expectation entry point (qs_expectation_noalloc) through the C ABI.

It serves callers that cannot allocate device memory: processes whose device memory is all held
by another allocator or a fixed budget, and loops that must not call the allocator because
cudaMalloc and cudaFree can synchronise the device. Its value must match qs_expectation, the
allocating entry point, within the tolerance of the other parity tests, on two calls in a row
(the fixed scratch array keeps the previous call's contents), and the FP64 oracle's value on
the same vector. Collected last, so a stop at the first failure has already run every other
test; it also passes alone in a fresh process.
"""
import ctypes

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


def noalloc(qs, st, obs):
    import torch
    o, keep = qs.make_obs(obs)
    out = (ctypes.c_double * 2)()
    stream = torch.cuda.current_stream().cuda_stream
    rc = qs.lib().qs_expectation_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), st.n, st.dtype,
                                         ctypes.c_void_p(stream), ctypes.byref(o), out)
    return rc, (out[0], out[1])


def noalloc_ptr(qs, ptr, n, dtype, obs):
    import torch
    o, keep = qs.make_obs(obs)
    out = (ctypes.c_double * 2)()
    stream = torch.cuda.current_stream().cuda_stream
    rc = qs.lib().qs_expectation_noalloc(ctypes.c_void_p(ptr), n, dtype, ctypes.c_void_p(stream), ctypes.byref(o), out)
    return rc, (out[0], out[1])


@pytest.fixture(params=["default", "double-float+tensor-cores"])
def settings(qs, request):
    """The library defaults, and the benchmark's complex128 arithmetic (double-float with the
    tensor-core blocks); the entry point reads IEEE vectors either way."""
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    if request.param != "default":
        qs.set_c128_math(qs.QS_MATH_DF)
        qs.set_tensor_cores(old_t | qs.QS_TENSOR_C128)
    yield request.param
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


@pytest.mark.parametrize("dtype", [2, 1])
def test_noalloc_matches_allocating_entry_point(qs, settings, dtype):
    tol = 1e-12 if dtype == 2 else 1e-6
    for n, seed in [(3, 1), (12, 2), (21, 3)]:
        st = qs.State(n, dtype)
        psi = W.random_state_fast(n, seed)
        st.load(psi)
        obs_list = [W.random_pauli_observable(n, 60, 10 + seed), W.tfim_observable(n, 0.7)]
        for obs in obs_list:
            ref = st.expectation(obs)
            e_oracle = oracle.expectation(st.get_vector().astype(np.complex128), obs)[0]
            scale = max(1.0, float(np.sum(np.abs(obs.coef))))
            for call in range(2):
                rc, got = noalloc(qs, st, obs)
                assert rc == qs.QS_OK, qs.lib().qs_last_error()
                assert abs(got[0] - ref[0]) < tol * max(1.0, abs(ref[0])), (n, call, got, ref)
                assert abs(got[1] - ref[1]) < tol * max(1.0, abs(ref[0]))
                # the oracle sums the same vector in FP64: the GPU's FP64-class sums agree to rounding
                assert abs(got[0] - e_oracle) < (1e-12 if dtype == 2 else 1e-10) * scale, (n, got, e_oracle)
        st.close()


def test_noalloc_after_tensor_core_run(qs, settings):
    """A state left by a fused complex128 run (tensor-core blocks under double-float) is read in
    the IEEE layout: the value matches the oracle's on the oracle's own run of the circuit."""
    n = 14
    c = W.u3cz_circuit(n, 6, 77)
    ref = oracle.run_circuit(c)
    obs = W.tfim_observable(n, 1.0)
    e_ref = oracle.expectation(ref, obs)[0]
    st = qs.State(n, 2)
    st.run(c, 5)
    for call in range(2):
        rc, got = noalloc(qs, st, obs)
        assert rc == qs.QS_OK, qs.lib().qs_last_error()
        assert abs(got[0] - e_ref) < 1e-11, (call, got, e_ref)
    st.close()


@pytest.mark.parametrize("dtype", [2, 1])
def test_noalloc_state_16_bytes_into_a_32_byte_aligned_buffer(qs, dtype):
    """The header asks for 16-byte alignment only: a vector that starts 16 bytes into a
    32-byte-aligned buffer gives the same value as an aligned copy and as the oracle."""
    import torch
    n = 13
    psi = W.random_state_fast(n, 8)
    tdt = torch.complex128 if dtype == 2 else torch.complex64
    shift = 16 // (16 if dtype == 2 else 8)
    buf = torch.zeros((1 << n) + shift, dtype=tdt, device="cuda")
    assert buf.data_ptr() % 32 == 0
    view = buf[shift:]
    view.copy_(torch.from_numpy(psi.astype(np.complex128 if dtype == 2 else np.complex64)).cuda())
    assert view.data_ptr() % 32 == 16
    obs = W.random_pauli_observable(n, 40, 5)
    rc, got = noalloc_ptr(qs, view.data_ptr(), n, dtype, obs)
    assert rc == qs.QS_OK, qs.lib().qs_last_error()
    aligned = view.clone()
    rc2, got2 = noalloc_ptr(qs, aligned.data_ptr(), n, dtype, obs)
    assert rc2 == qs.QS_OK
    e_oracle = oracle.expectation(view.cpu().numpy().astype(np.complex128), obs)[0]
    tol = 1e-12 if dtype == 2 else 1e-6
    assert abs(got[0] - got2[0]) < tol
    assert abs(got[0] - e_oracle) < tol * max(1.0, float(np.sum(np.abs(obs.coef))))


def wide_masks(n, count):
    """The first `count` flip masks with 10 or more X positions above qubit 2: none fits a tile,
    so each takes a launch of its own."""
    out = []
    f = 0
    while len(out) < count:
        f += 1
        if bin(f >> 3).count("1") >= 10:
            out.append(f)
    return np.array(out, dtype=np.uint64)


def test_noalloc_rejects_oversized_observable(qs):
    n = 20
    st = qs.State(n, 2)
    m = 33000                     # single-group launches beyond the 32767 block partials
    obs = W.PauliObservable(n, np.ones(m), wide_masks(n, m), np.zeros(m, dtype=np.uint64))
    rc, _ = noalloc(qs, st, obs)
    assert rc == qs.QS_ERR_INVALID_ARG
    assert b"launches" in qs.lib().qs_last_error()
    # still usable afterwards
    rc, got = noalloc(qs, st, W.tfim_observable(n, 1.0))
    assert rc == qs.QS_OK
    assert abs(got[0] - st.expectation(W.tfim_observable(n, 1.0))[0]) < 1e-12
    st.close()
