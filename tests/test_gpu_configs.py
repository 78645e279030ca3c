"""The benchmark configurations themselves, checked against the FP64 oracle at their own sizes.

* Differentiation: the 20-qubit hardware-efficient ansatz with 20 layers (800 parameters, RY and
  RZ on every qubit then a CZ ladder) and H = sum Z_i Z_{i+1} + sum X_i on the open chain, through
  qs_adjoint_grad in the double-float arithmetic the benchmark times: the energy against the
  oracle, 20 seeded-sampled gradient components against the parameter-shift rule (exact for
  exp(i theta P / 2), so it pins each component to rounding) and against central finite
  differences with step 1e-6.
* Batching: circuits of 18..20 qubits (the level-synchronous whole-grid path of the persistent
  kernel) and a seeded sample of 20 circuits out of the 4096-circuit batch that the benchmark
  times, energies and sampled gradient components against the oracle.
* The 33-qubit complex128 state (128 GiB, in place): sampled amplitudes of a circuit with a closed
  form, run through the double-float path with 5-qubit tensor-core blocks.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

BENCH_SEED = 20201127  # seed of the benchmark's workloads (bench.py --seed default)


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_13524_gb300 as qs
    qs.lib()
    return qs


@pytest.fixture
def df_tc(qs):
    """Double-float complex128 arithmetic with the tensor-core blocks, restored afterwards."""
    old_m, old_t = qs.get_c128_math(), qs.get_tensor_cores()
    qs.set_c128_math(qs.QS_MATH_DF)
    qs.set_tensor_cores(old_t | qs.QS_TENSOR_C128)
    yield qs
    qs.set_c128_math(old_m)
    qs.set_tensor_cores(old_t)


def sample_indices(count, total, seed):
    rng = W.SplitMix64(seed)
    out = []
    while len(out) < count:
        j = int(rng.next_u64() % total)
        if j not in out:
            out.append(j)
    return sorted(out)


# ---------------------------------------------------------------- differentiation, n = 20
@pytest.fixture(scope="module")
def hea20():
    c = W.hea_circuit(20, 20, BENCH_SEED)
    H = W.tfim_observable(20, 1.0)
    idx = sample_indices(20, c.n_params, 4)
    return c, H, idx


@pytest.fixture(scope="module")
def hea20_oracle(hea20):
    c, H, idx = hea20
    return {"energy": oracle.energy(c, H),
            "shift": oracle.grad_parameter_shift(c, H, idx),
            "fd": oracle.grad_finite_difference(c, H, idx, h=1e-6)}


def test_config_adjoint_n20_800_parameters(df_tc, hea20, hea20_oracle):
    qs = df_tc
    c, H, idx = hea20
    assert c.n_params == 800 and len(c.gates) == 1180
    e, g = qs.adjoint_grad(c, H)
    assert g.shape == (800,)
    assert abs(e - hea20_oracle["energy"]) < 1e-12, (e, hea20_oracle["energy"])
    err_shift = float(np.max(np.abs(g[idx] - hea20_oracle["shift"])))
    err_fd = float(np.max(np.abs(g[idx] - hea20_oracle["fd"])))
    assert err_shift < 1e-11, err_shift
    # central difference: truncation h^2/6 |E'''| < 1e-11, rounding ~ eps |E| / h ~ 1e-9
    assert err_fd < 1e-7, err_fd


def test_config_adjoint_n20_ieee_fp64(qs, hea20, hea20_oracle):
    """The same gradient with IEEE FP64 gate arithmetic: both arithmetics meet the bound."""
    c, H, idx = hea20
    old = qs.get_c128_math()
    try:
        qs.set_c128_math(qs.QS_MATH_FP64)
        e, g = qs.adjoint_grad(c, H)
    finally:
        qs.set_c128_math(old)
    assert abs(e - hea20_oracle["energy"]) < 1e-12
    assert float(np.max(np.abs(g[idx] - hea20_oracle["shift"]))) < 1e-11


def test_config_adjoint_n20_complex64(qs, hea20, hea20_oracle):
    """complex64 storage with FP64-class sums: energy and gradient within the complex64 bounds."""
    c, H, idx = hea20
    e, g = qs.adjoint_grad(c, H, dtype=qs.QS_C64)
    assert abs(e - hea20_oracle["energy"]) < 1e-4
    assert float(np.max(np.abs(g[idx] - hea20_oracle["shift"]))) < 1e-4


# ---------------------------------------------------------------- batching
def check_batch(items, energies, grads, thetas, n_grad, e_tol=2e-5, g_tol=5e-5):
    worst_e = worst_g = 0.0
    for k, it in enumerate(items):
        c = it.circuit.bind(thetas[k])
        e_ref = oracle.energy(c, it.observable)
        worst_e = max(worst_e, abs(energies[k] - e_ref) / max(1.0, abs(e_ref)))
        idx = sample_indices(min(n_grad, c.n_params), c.n_params, 100 + k)
        ps = oracle.grad_parameter_shift(c, it.observable, idx)
        worst_g = max(worst_g, float(np.max(np.abs(grads[k][idx] - ps))))
    assert worst_e < e_tol, worst_e
    assert worst_g < g_tol, worst_g


def test_config_batch_wide_circuits_18_to_20(qs):
    """Circuits of 18..20 qubits run level-synchronously over the whole grid."""
    items = W.batch_workload(4, 1820, n_lo=18, n_hi=20, l_lo=2, l_hi=12)
    assert max(i.circuit.n for i in items) >= 19
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    e, g = b.run(theta, use_graph=True)
    offs = np.cumsum([0] + [i.circuit.n_params for i in items])
    check_batch(items, e, g, [theta[offs[k]:offs[k + 1]] for k in range(len(items))], n_grad=3)


def test_config_batch_4096_sampled(qs):
    """The benchmark's own batch (4096 circuits, n ~ U{8..20}, 2..12 layers, 4-term Pauli
    observables) in one graph-replayed persistent launch; 20 seeded-sampled circuits checked."""
    items = W.batch_workload(4096, BENCH_SEED)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    b.run(theta, use_graph=True)
    e, g = b.run(theta, use_graph=True)  # replay
    assert np.all(np.isfinite(e))
    pick = sample_indices(20, len(items), 5096)
    assert any(items[k].circuit.n >= 17 for k in pick)
    offs = np.cumsum([0] + [i.circuit.n_params for i in items])
    check_batch([items[k] for k in pick], e[pick], [g[k] for k in pick],
                [theta[offs[k]:offs[k + 1]] for k in pick], n_grad=2)


# ---------------------------------------------------------------- n = 33 complex128
def test_config_n33_sampled_amplitudes(df_tc):
    """33 qubits (128 GiB): 20 U3 layers then every CZ brickwork layer, fused at width 5 on the
    tensor cores; amplitude x = prod_q phi_q[x_q] (-1)^(CZ pairs set in x)."""
    import torch
    from test_gpu_parity import product_then_cz, sampled_amplitudes
    qs = df_tc
    n = 33
    free, _ = torch.cuda.mem_get_info()
    if free < (16 << n) + (4 << 30):
        pytest.skip("needs 132 GiB of free device memory")
    circ, u3, cz = product_then_cz(n, 20, 3333)
    plan = qs.FusedCircuit(circ, 5)
    kinds = {plan.block_cost(b, qs.QS_C128)[0] for b in range(plan.n_blocks)}
    assert "dense_oz5" in kinds, kinds
    st = qs.State(n, qs.QS_C128)
    st.apply_plan(plan)
    st.synchronize()
    rng = W.SplitMix64(33)
    xs = [rng.next_u64() & ((1 << n) - 1) for _ in range(2000)] + [0, (1 << n) - 1, 1 << 32, (1 << 32) - 1]
    ref = sampled_amplitudes(n, u3, cz, xs)
    idx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    got = st.tensor[idx].cpu().numpy()
    assert float(np.max(np.abs(got - ref))) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-11
    st.close()
    del st
    torch.cuda.empty_cache()
