"""Failure paths, made to happen without faulting or hanging the GPU.

* Bounded device-side waits: the tensor-core kernels' accumulator waits and the batch kernel's
  grid barrier give up after a limit that a test hook makes small, or a hook makes the first
  accumulator wait report late (while the kernel's final wait for its own MMAs keeps the full
  limit). The call that synchronises reports QS_ERR_TIMEOUT, and the next run with the hooks off
  is correct: the GPU and the library stay usable.
* Device allocations: a hook makes the k-th allocation of a call fail as if memory had run out;
  for every k up to the call's last allocation the call returns QS_ERR_OOM and the library holds
  no more allocations than before it, and the call succeeds once k passes its allocations.
"""
import ctypes
import gc

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


@pytest.fixture
def hooks(qs):
    """Every hook off again after the test, whatever happened."""
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    yield qs
    qs.check(qs.lib().qs_debug_set_fault(qs.QS_DEBUG_NONE))
    qs.check(qs.lib().qs_debug_set_wait_limit(-1))
    qs.check(qs.lib().qs_debug_fail_alloc(-1, None))
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


def held(qs):
    h = ctypes.c_longlong(0)
    qs.check(qs.lib().qs_debug_fail_alloc(-1, ctypes.byref(h)))
    return h.value


# ---------------------------------------------------------------- bounded waits
@pytest.mark.parametrize("dtype,k", [(2, 5), (2, 4), (1, 6)])
def test_tensor_core_wait_reports_timeout_and_recovers(hooks, dtype, k):
    qs = hooks
    qs.set_c128_math(qs.QS_MATH_DF)
    qs.set_tensor_cores(qs.QS_TENSOR_C128 | qs.QS_TENSOR_C64X)
    n = 14
    c = W.u3cz_circuit(n, 6, 900 + k)
    ref = oracle.run_circuit(c)
    plan = qs.FusedCircuit(c, k)
    want = {5: "dense_oz5", 4: "dense_oz", 6: "dense_bz"}[k]
    assert want in {plan.block_cost(b, dtype)[0] for b in range(plan.n_blocks)}
    st = qs.State(n, dtype)
    qs.check(qs.lib().qs_debug_set_fault(qs.QS_DEBUG_TC_LATE))
    st.apply_plan(plan)
    with pytest.raises(qs.QsError) as e:
        st.synchronize()
    assert e.value.code == qs.QS_ERR_TIMEOUT
    qs.check(qs.lib().qs_debug_set_fault(qs.QS_DEBUG_NONE))
    st.synchronize()  # the error was reported once and cleared
    st.set_basis(0)
    st.apply_plan(plan)
    got = st.get_vector()
    assert float(np.max(np.abs(got - ref))) < (1e-12 if dtype == 2 else 1e-5)
    st.close()


def test_tensor_core_short_wait_limit_never_hangs(hooks):
    """A limit of one poll per wait: the launch either finishes or reports a timeout; either way
    the state is usable again and the next run with the default limit is correct."""
    qs = hooks
    qs.set_c128_math(qs.QS_MATH_DF)
    n = 16
    c = W.u3cz_circuit(n, 6, 77)
    ref = oracle.run_circuit(c)
    plan = qs.FusedCircuit(c, 5)
    st = qs.State(n, qs.QS_C128)
    qs.check(qs.lib().qs_debug_set_wait_limit(0))
    st.apply_plan(plan)
    try:
        st.synchronize()
    except qs.QsError as e:
        assert e.code == qs.QS_ERR_TIMEOUT
    qs.check(qs.lib().qs_debug_set_wait_limit(-1))
    st.set_basis(0)
    st.apply_plan(plan)
    assert float(np.max(np.abs(st.get_vector() - ref))) < 1e-12
    st.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_grid_barrier_timeout_and_recovery(hooks, use_graph):
    qs = hooks
    items = W.batch_workload(5, 31, n_lo=14, n_hi=15, l_lo=1, l_hi=3)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    e_ok, g_ok = b.run(theta, use_graph=use_graph)
    qs.check(qs.lib().qs_debug_set_wait_limit(2000))       # 2000 polls of 256 ns: about 0.5 ms
    qs.check(qs.lib().qs_debug_set_fault(qs.QS_DEBUG_BATCH_HOLD))
    for _ in range(2):
        with pytest.raises(qs.QsError) as e:
            b.run(theta, use_graph=use_graph)
        assert e.value.code == qs.QS_ERR_TIMEOUT
    qs.check(qs.lib().qs_debug_set_fault(qs.QS_DEBUG_NONE))
    qs.check(qs.lib().qs_debug_set_wait_limit(-1))
    e2, g2 = b.run(theta, use_graph=use_graph)
    assert np.array_equal(e2, e_ok)
    assert all(np.array_equal(a, c) for a, c in zip(g2, g_ok))
    for k, it in enumerate(items):
        assert abs(e2[k] - oracle.energy(it.circuit, it.observable)) < 2e-5


# ---------------------------------------------------------------- allocation failures
def sweep_allocation_failures(qs, op, cleanup, limit=60):
    """Runs op with the k-th allocation failing, k = 0, 1, ...: every failing run reports
    QS_ERR_OOM and leaves the library holding what it held before; returns the first k at which
    op succeeds (its allocation count)."""
    gc.collect()  # objects left by earlier tests release their allocations now, not mid-sweep
    base = held(qs)
    for k in range(limit):
        objs = []
        qs.check(qs.lib().qs_debug_fail_alloc(k, None))
        try:
            op(objs)
            ok = True
        except qs.QsError as e:
            assert e.code == qs.QS_ERR_OOM, (k, e)
            ok = False
        finally:
            qs.check(qs.lib().qs_debug_fail_alloc(-1, None))
            cleanup(objs)
            gc.collect()
        assert held(qs) == base, (k, held(qs), base)
        if ok:
            return k
    raise AssertionError("the call never succeeded")


def test_allocation_failures_state_circuit_expectation(hooks):
    import torch
    qs = hooks
    qs.set_c128_math(qs.QS_MATH_DF)
    n = 14
    c = W.u3cz_circuit(n, 6, 41)
    ref = oracle.run_circuit(c)
    obs = W.tfim_observable(n, 1.0)
    rng = W.SplitMix64(2)
    uni = [rng.uniform() for _ in range(16)]

    def op(objs):
        st = qs.State(n, qs.QS_C128, owned=True)
        objs.append(st)
        st.run(c, 5)       # block matrices uploaded (tensor-core form), double-float layout
        st.expectation(obs)
        st.norm2()
        st.sample(uni)
        objs.append(st.get_vector())

    def cleanup(objs):
        for o in objs:
            if hasattr(o, "close"):
                o.close()
        torch.cuda.synchronize()

    k = sweep_allocation_failures(qs, op, cleanup)
    assert k >= 3  # the state, the matrices, the reduction scratch at least
    st = qs.State(n, qs.QS_C128, owned=True)
    st.run(c, 5)
    assert float(np.max(np.abs(st.get_vector() - ref))) < 1e-12
    st.close()


def test_allocation_failures_adjoint_and_batch(hooks):
    import torch
    qs = hooks
    hea = W.hea_circuit(8, 2, 5)
    H = W.tfim_observable(8, 1.0)

    def op_adj(objs):
        objs.append(qs.adjoint_grad(hea, H))

    def cleanup(objs):
        torch.cuda.synchronize()

    assert sweep_allocation_failures(qs, op_adj, cleanup) >= 2
    e, g = qs.adjoint_grad(hea, H)
    assert abs(e - oracle.energy(hea, H)) < 1e-12

    items = W.batch_workload(6, 8, n_lo=8, n_hi=15, l_lo=1, l_hi=3)

    def op_batch(objs):
        b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
        objs.append(b)
        b.run(np.concatenate([i.circuit.parameters() for i in items]), use_graph=False)

    def cleanup_batch(objs):
        for o in objs:
            o.__del__()
        torch.cuda.synchronize()

    assert sweep_allocation_failures(qs, op_batch, cleanup_batch) >= 5
