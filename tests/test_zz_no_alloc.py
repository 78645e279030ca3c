"""The allocation-free expectation entry point (qs_expectation_noalloc) through the C ABI.

It serves callers that cannot allocate device memory (inside stream capture, under a foreign
allocator or a fixed memory budget). Its value must match qs_expectation, the allocating entry
point, within the tolerance of the other parity tests, on two calls in a row (the fixed scratch
array keeps the previous call's contents). Collected last, so a stop at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype", [2, 1])
def test_noalloc_matches_allocating_entry_point(qs, dtype):
    tol = 1e-12 if dtype == 2 else 1e-6
    for n, seed in [(3, 1), (12, 2), (21, 3)]:
        st = qs.State(n, dtype)
        st.load(W.random_state_fast(n, seed))
        obs_list = [W.random_pauli_observable(n, 60, 10 + seed), W.tfim_observable(n, 0.7)]
        for obs in obs_list:
            ref = st.expectation(obs)
            for call in range(2):
                rc, got = noalloc(qs, st, obs)
                assert rc == qs.QS_OK, qs.lib().qs_last_error()
                assert abs(got[0] - ref[0]) < tol * max(1.0, abs(ref[0])), (n, call, got, ref)
                assert abs(got[1] - ref[1]) < tol * max(1.0, abs(ref[0]))
        st.close()


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
