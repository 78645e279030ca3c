"""Tile shapes of the shared-memory dense kernel (4..6 targets on the CUDA cores): the autotuner
times rows per thread 4, 8 and 16 on the GPU and keeps the fastest; every shape gives the same
bits, and each matches the oracle. Complex64 (tensor cores off), complex128 in FP64 and in
double-float (tensor cores off)."""
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
def settings(qs):
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    yield qs
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


CASES = [("c64", 1, None, (5, 6)), ("c128_fp64", 2, "FP64", (4, 5, 6)), ("c128_df", 2, "DF", (4, 5, 6))]


def setup_arith(qs, math):
    qs.set_tensor_cores(0)  # the CUDA-core kernels for every width
    if math is not None:
        qs.set_c128_math(qs.QS_MATH_FP64 if math == "FP64" else qs.QS_MATH_DF)


def test_autotuner_picks_a_tile_shape(settings):
    qs = settings
    for name, dtype, math, widths in CASES:
        setup_arith(qs, math)
        c = W.u3cz_circuit(14, 4, 3)
        qs.autotune_fusion(c, dtype)
        for m in widths:
            rows, tuned = qs.dense_tile_rows(dtype, m)
            assert tuned and rows in (4, 8, 16), (name, m, rows, tuned)


@pytest.mark.parametrize("name,dtype,math,widths", CASES)
def test_tile_shapes_same_bits_and_oracle(settings, name, dtype, math, widths):
    qs = settings
    setup_arith(qs, math)
    n = 11
    rng = W.SplitMix64(77)
    psi0 = W.random_state(n, 5)
    for m in widths:
        saved = qs.dense_tile_rows(dtype, m)
        for targets, controls in (((0, 3, 7, 9, 10, 2)[:m], ()), ((10, 1, 5, 8, 4, 6)[:m], (2,))):
            K = W.random_complex_matrix(1 << m, rng) * 0.3
            g = W.Gate("DENSE", targets, matrix=K, controls=controls, control_values=(1,) * len(controls))
            ref = psi0.copy()
            oracle.apply_gate(ref, n, g)
            outs = []
            for rows in (4, 8, 16):
                qs.check(qs.lib().qs_debug_set_tile_rows(dtype, m, rows))
                st = qs.State(n, dtype)
                st.load(psi0)
                st.apply_gate(g)
                outs.append(st.get_vector())
                st.close()
            for o in outs[1:]:
                assert np.array_equal(o, outs[0]), (name, m, targets)
            got = outs[0].astype(np.complex128)
            tol = 1e-12 if dtype == 2 else 1e-5
            assert float(np.max(np.abs(got - ref))) < tol * max(1.0, float(np.max(np.abs(ref)))), (name, m)
        qs.check(qs.lib().qs_debug_set_tile_rows(dtype, m, saved[0] if saved[1] else 0))


def test_tile_rows_invalid(settings):
    qs = settings
    with pytest.raises(qs.QsError):
        qs.check(qs.lib().qs_debug_set_tile_rows(2, 4, 6))
    with pytest.raises(qs.QsError):
        qs.dense_tile_rows(2, 3)
