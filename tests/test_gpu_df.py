"""GPU parity of the complex128 double-float arithmetic (QS_MATH_DF) against the FP64 oracle.

In this mode a circuit run converts the state in place to double-float pairs, applies every
gate on the FP32 pipes and converts back; the result must still meet the complex128 bound
(1e-12 max-abs amplitude error) and the state seen at every entry point is IEEE complex128.
"""
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
def df(qs):
    old = qs.get_c128_math()
    qs.set_c128_math(qs.QS_MATH_DF)
    yield qs
    qs.set_c128_math(old)


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


@pytest.mark.parametrize("n", [1, 2, 3, 6, 9, 12])
def test_df_every_gate_kind(df, n):
    qs = df
    for seed in range(2):
        gates = W.random_gate_suite(n, 500 * n + seed)
        psi0 = W.random_state(n, seed + 3)
        for g in gates:
            ref = psi0.copy()
            oracle.apply_gate(ref, n, g)
            st = qs.State(n, qs.QS_C128)
            st.load(psi0)
            st.run(W.Circuit(n, [g]), 0)
            assert maxabs(st.get_vector(), ref) < 1e-12, (g.name, g.targets)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6])
def test_df_circuits(df, k):
    qs = df
    for n, c in [(12, W.u3cz_circuit(12, 10, 2021)), (15, W.Circuit(15, W.random_gate_suite(15, 8))),
                 (17, W.rzrxrz_cnot_circuit(17, 4, 2))]:
        ref = oracle.run_circuit(c)
        st = qs.State(n, qs.QS_C128)
        st.run(c, k)
        got = st.get_vector()
        assert maxabs(got, ref) < 1e-12
        # the buffer is IEEE complex128 again after the run
        assert abs(st.norm2() - oracle.norm2(ref, n)) < 1e-12


def test_df_deep_circuit_error_growth(df):
    """890-gate depth-20 family at n = 20: error after the whole circuit within the bound."""
    qs = df
    c = W.u3cz_circuit(20, 20, 11)
    ref = oracle.run_circuit(c)
    for k in (0, 2, 3):
        st = qs.State(20, qs.QS_C128)
        st.run(c, k)
        err = maxabs(st.get_vector(), ref)
        assert err < 1e-12, (k, err)


def test_df_non_unitary_and_small_values(df):
    """K need not be unitary: scaled matrices and tiny amplitudes keep their relative accuracy."""
    qs = df
    n = 8
    rng = W.SplitMix64(4)
    psi0 = W.random_state(n, 2) * 1e-3
    gates = [W.Gate("DENSE", (1, 6), matrix=W.random_complex_matrix(4, rng) * 3.0),
             W.Gate("DENSE", (0,), matrix=W.random_complex_matrix(2, rng) * 1e-4),
             W.Gate("DENSE", (7, 2, 4), matrix=W.random_complex_matrix(8, rng))]
    c = W.Circuit(n, gates)
    ref = oracle.run_circuit(c, psi0)
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(c, 0)
    got = st.get_vector()
    scale = np.max(np.abs(ref))
    assert maxabs(got, ref) < 1e-13 * max(scale, 1.0) * 8


def test_df_adjoint(df):
    qs = df
    c = W.hea_circuit(7, 3, 5)
    obs = W.tfim_observable(7, 1.0)
    e, g = qs.adjoint_grad(c, obs)
    assert abs(e - oracle.energy(c, obs)) < 1e-12
    ps = oracle.grad_parameter_shift(c, obs, range(c.n_params))
    assert np.max(np.abs(g - ps)) < 1e-11


def test_df_full_size_sampled(df):
    import torch
    from test_gpu_parity import product_then_cz, sampled_amplitudes
    qs = df
    n = 30
    circ, u3, cz = product_then_cz(n, 20, 777)
    st = qs.State(n, qs.QS_C128)
    st.run(circ, 2)
    st.synchronize()
    rng = W.SplitMix64(6)
    xs = [rng.next_u64() & ((1 << n) - 1) for _ in range(2000)] + [0, (1 << n) - 1]
    ref = sampled_amplitudes(n, u3, cz, xs)
    idx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    got = st.tensor[idx].cpu().numpy()
    assert maxabs(got, ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-11
    st.close()
    del st
    torch.cuda.empty_cache()


def test_precision_c64_c128_vs_oracle(qs):
    """The precision comparison on the depth-20 circuit family at n = 20: complex64 (FP32 gates,
    FP64-built matrices, FP64 sums) and complex128 in both arithmetics against the FP64 oracle:
    max-abs amplitude error, 1 - fidelity and the transverse-field Ising energy error (h = 1)."""
    n = 20
    c = W.u3cz_circuit(n, 20, 2020)
    ref = oracle.run_circuit(c)
    tf = W.tfim_observable(n, 1.0)
    e_ref = oracle.expectation(ref, tf)[0]
    old = qs.get_c128_math()
    try:
        for dtype, math_mode, k, amp_tol, e_tol in ((2, qs.QS_MATH_FP64, 2, 1e-12, 1e-11),
                                                    (2, qs.QS_MATH_DF, 2, 1e-12, 1e-11),
                                                    (1, qs.QS_MATH_FP64, 4, 1e-5, 1e-4)):
            qs.set_c128_math(math_mode)
            st = qs.State(n, dtype)
            st.run(c, k)
            got = st.get_vector().astype(np.complex128)
            err = maxabs(got, ref)
            fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real)
            assert err < amp_tol, (dtype, math_mode, err)
            assert 1 - fid < (1e-12 if dtype == 2 else 1e-6)
            assert abs(st.expectation(tf)[0] - e_ref) < e_tol
    finally:
        qs.set_c128_math(old)


def test_df_layout_round_trip_wide_range(df):
    """The in-place layout change and back (an empty circuit run) keeps every amplitude between
    1e-28 and 1e30 to 2^-47 relative (both conversion branches, signs), zeros exactly, and values
    below the FP32 exponent range (1e-300 .. 1e-40) to 1e-37 absolute."""
    qs = df
    n = 12
    rng = W.SplitMix64(12)
    N = 1 << n
    mags = np.array([10.0 ** (-28 + 58 * rng.uniform()) for _ in range(N)])
    tiny = np.array([10.0 ** (-300 + 260 * rng.uniform()) for _ in range(N)])
    signs = np.array([1 if rng.next_u64() & 1 else -1 for _ in range(2 * N)]).reshape(2, -1)
    psi0 = signs[0] * mags + 1j * signs[1] * mags[::-1]
    psi0[::97] = 0.0
    psi0[5::7] = signs[0][5::7] * tiny[5::7] + 1j * tiny[::-1][5::7]
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(W.Circuit(n, []), 0)
    got = st.get_vector()
    small = np.zeros(N, dtype=bool)
    small[5::7] = True
    small[::97] = False
    zero = np.zeros(N, dtype=bool)
    zero[::97] = True
    normal = ~(small | zero)
    assert np.all(got[zero] == 0)
    rel = np.abs(got[normal] - psi0[normal]) / np.abs(psi0[normal])
    assert float(np.max(rel)) < 2.0 ** -47
    assert float(np.max(np.abs(got[small] - psi0[small]))) < 1e-37


def test_df_layout_round_trip_bit_exact(df):
    """In place to double-float and back: every amplitude in FP32's normal range comes back as
    exactly RN(hi + lo) with hi = RN_float(x), lo = RN_float(x - hi) (numpy's float32 rounding and
    FP64 sum), whichever path (integer pipes or the FP64 add) the join takes."""
    qs = df
    n = 13
    rng = np.random.default_rng(1313)
    N = 1 << n
    mags = 10.0 ** rng.uniform(-25, 25, 2 * N)
    vals = rng.choice([-1.0, 1.0], 2 * N) * mags
    vals[::37] *= (1 - 2.0 ** -30)   # significands with long runs of ones
    vals[5::41] = np.ldexp(1.0, rng.integers(-60, 60, len(vals[5::41])))  # powers of two
    psi0 = vals[0::2] + 1j * vals[1::2]
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(W.Circuit(n, []), 0)
    got = st.get_vector()
    re = np.ascontiguousarray(psi0).view(np.float64)
    hi = re.astype(np.float32)
    lo = (re - hi.astype(np.float64)).astype(np.float32)
    want = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(np.ascontiguousarray(got).view(np.float64).view(np.uint64), want.view(np.uint64))
    st.close()


def test_df_layout_round_trip_small_magnitudes_bit_exact(df):
    """Magnitudes from 2^-126 to 2^-70, where the low word of the split can be subnormal in FP32:
    in place to double-float and back still gives exactly RN(hi + lo) of numpy's float32 split
    (one rounding of lo, also when it is subnormal)."""
    qs = df
    n = 12
    rng = np.random.default_rng(2718)
    N = 1 << n
    mags = np.ldexp(1.0, rng.integers(-126, -70, 2 * N)) * rng.uniform(1.0, 2.0, 2 * N)
    vals = rng.choice([-1.0, 1.0], 2 * N) * mags
    vals[::29] = np.ldexp(1.0, rng.integers(-126, -70, len(vals[::29])))  # powers of two
    vals[3::31] *= (1 + 2.0 ** -40)  # remainders far below hi
    psi0 = vals[0::2] + 1j * vals[1::2]
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(W.Circuit(n, []), 0)
    got = st.get_vector()
    re = np.ascontiguousarray(psi0).view(np.float64)
    hi = re.astype(np.float32)
    lo = (re - hi.astype(np.float64)).astype(np.float32)
    want = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(np.ascontiguousarray(got).view(np.float64).view(np.uint64), want.view(np.uint64))
    st.close()


def test_df_layout_round_trip_near_powers_of_two(df):
    """Doubles just below and above powers of two (hi = 2^k with lo of either sign, the join's
    binade edge and its FP64 fallback), long runs of ones, and lo exponents 24..60 below hi's:
    in place to double-float and back gives exactly RN(hi + lo) of numpy's float32 split."""
    qs = df
    n = 12
    rng = np.random.default_rng(4242)
    N = 1 << n
    k = rng.integers(-60, 60, 2 * N)
    eps = np.ldexp(1.0, -rng.integers(24, 61, 2 * N))
    kind = rng.integers(0, 4, 2 * N)
    base = np.ldexp(1.0, k)
    vals = np.where(kind == 0, base * (1 - eps), np.where(kind == 1, base * (1 + eps),
                    np.where(kind == 2, base * (1 - eps) * (1 - 2.0 ** -53), base * (1.5 + eps))))
    vals *= rng.choice([-1.0, 1.0], 2 * N)
    psi0 = vals[0::2] + 1j * vals[1::2]
    st = qs.State(n, qs.QS_C128)
    st.load(psi0)
    st.run(W.Circuit(n, []), 0)
    got = st.get_vector()
    re = np.ascontiguousarray(psi0).view(np.float64)
    hi = re.astype(np.float32)
    lo = (re - hi.astype(np.float64)).astype(np.float32)
    want = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(np.ascontiguousarray(got).view(np.float64).view(np.uint64), want.view(np.uint64))
    st.close()
