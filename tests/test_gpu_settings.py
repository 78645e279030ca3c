"""Arithmetic settings per state and per call (qs_state_set_arith, qs_set_c128_math).

A state with settings of its own runs with them whatever the process-wide settings are; a
call reads the settings once, at entry, so threads that change the process-wide settings while
other threads apply circuits do not change those circuits' results. Results are compared bit
for bit with single-threaded runs under the same settings, and with the FP64 oracle.
"""
import threading

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
def restore(qs):
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    yield
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


def run(qs, c, k, math=-1, tensor=-1):
    st = qs.State(c.n, qs.QS_C128)
    st.set_arith(math, tensor)
    st.run(c, k)
    out = st.get_vector()
    st.close()
    return out


def test_state_settings_override_process_settings(qs, restore):
    c = W.u3cz_circuit(14, 6, 515)
    ref = oracle.run_circuit(c)
    qs.set_c128_math(qs.QS_MATH_DF)
    qs.set_tensor_cores(qs.QS_TENSOR_C128)
    df_tc = run(qs, c, 5)
    qs.set_c128_math(qs.QS_MATH_FP64)
    qs.set_tensor_cores(0)
    fp64 = run(qs, c, 5)
    own = run(qs, c, 5, qs.QS_MATH_DF, qs.QS_TENSOR_C128)  # its own settings, unlike the process's
    assert np.array_equal(own, df_tc)
    assert not np.array_equal(df_tc, fp64)  # the two arithmetics round differently
    for v in (df_tc, fp64, own):
        assert float(np.max(np.abs(v - ref))) < 1e-12
    st = qs.State(5, qs.QS_C128)
    assert st.get_arith() == (-1, -1)
    st.set_arith(qs.QS_MATH_FP64, qs.QS_TENSOR_C128)
    assert st.get_arith() == (qs.QS_MATH_FP64, qs.QS_TENSOR_C128)
    with pytest.raises(qs.QsError) as e:
        st.set_arith(5, -1)
    assert e.value.code == qs.QS_ERR_INVALID_ARG
    with pytest.raises(qs.QsError):
        st.set_arith(-1, 1)
    st.close()


def test_threads_with_own_settings_while_process_settings_change(qs, restore):
    import torch
    c = W.u3cz_circuit(14, 6, 616)
    ref = oracle.run_circuit(c)
    configs = [(qs.QS_MATH_FP64, 0, 2), (qs.QS_MATH_DF, qs.QS_TENSOR_C128, 5), (qs.QS_MATH_DF, 0, 3),
               (qs.QS_MATH_DF, qs.QS_TENSOR_C128, 4)]
    expected = [run(qs, c, k, m, t) for m, t, k in configs]
    stop = threading.Event()
    results = [[] for _ in configs]
    follow = []
    errors = []

    def worker(i):
        try:
            m, t, k = configs[i]
            torch.cuda.set_device(0)
            with torch.cuda.stream(torch.cuda.Stream()):
                for _ in range(6):
                    results[i].append(run(qs, c, k, m, t))
                    follow.append(run(qs, c, k))  # follows whatever the process setting is
        except Exception as e:  # surfaced in the main thread
            errors.append(repr(e))

    def toggler():
        j = 0
        while not stop.is_set():
            qs.set_c128_math(qs.QS_MATH_FP64 if j % 2 else qs.QS_MATH_DF)
            qs.set_tensor_cores(qs.QS_TENSOR_C128 if j % 3 else 0)
            j += 1

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(len(configs))]
    tg = threading.Thread(target=toggler)
    tg.start()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    stop.set()
    tg.join()
    assert not errors, errors
    for i, outs in enumerate(results):
        assert len(outs) == 6
        for v in outs:
            assert np.array_equal(v, expected[i]), configs[i]
    for v in follow:
        assert float(np.max(np.abs(v - ref))) < 1e-12
