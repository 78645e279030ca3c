"""Batched persistent execution (qs_batch_*) against the FP64 oracle: energies and adjoint
gradients of many independent parametric circuits, complex64 storage with FP64-class sums.
Covers shared-memory-resident circuits (n <= 13) and multi-pass chunked ones (n > 13), graph
replay with new parameters, and graph vs. direct launch."""
import math

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


def check_items(items, energies, grads, theta_of, e_tol=2e-5, g_tol=5e-5, sample=6):
    for k, it in enumerate(items):
        c = it.circuit.bind(theta_of(k))
        e_ref = oracle.energy(c, it.observable)
        assert abs(energies[k] - e_ref) < e_tol * max(1.0, abs(e_ref)), (k, it.circuit.n, energies[k], e_ref)
        idx = list(range(0, c.n_params, max(1, c.n_params // sample)))[:sample]
        ps = oracle.grad_parameter_shift(c, it.observable, idx)
        assert np.max(np.abs(grads[k][idx] - ps)) < g_tol, (k, it.circuit.n)


def test_batch_resident_small(qs):
    items = W.batch_workload(24, 7, n_lo=4, n_hi=11, l_lo=1, l_hi=4)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    e, g = b.run(theta, use_graph=False)
    offs = np.cumsum([0] + [i.circuit.n_params for i in items])
    check_items(items, e, g, lambda k: theta[offs[k]:offs[k + 1]])


def test_batch_chunked_large(qs):
    items = W.batch_workload(6, 9, n_lo=14, n_hi=17, l_lo=2, l_hi=4)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    assert b.total_passes > len(items)
    theta = np.concatenate([i.circuit.parameters() for i in items])
    e, g = b.run(theta, use_graph=True)
    offs = np.cumsum([0] + [i.circuit.n_params for i in items])
    check_items(items, e, g, lambda k: theta[offs[k]:offs[k + 1]], sample=4)


def test_batch_graph_replay_new_theta(qs):
    items = W.batch_workload(40, 3, n_lo=4, n_hi=15, l_lo=1, l_hi=5)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    rng = W.SplitMix64(1)
    offs = np.cumsum([0] + [i.circuit.n_params for i in items])
    for rep in range(3):
        theta = np.array([rng.uniform_range(-math.pi, math.pi) for _ in range(b.total_params)])
        e1, g1 = b.run(theta, use_graph=True)
        e2, g2 = b.run(theta, use_graph=False)
        assert np.array_equal(e1, e2)
        assert all(np.array_equal(a, c) for a, c in zip(g1, g2))
        if rep == 2:
            check_items(items[::7], e1[::7], g1[::7], lambda k: theta[offs[7 * k]:offs[7 * k + 1]], sample=3)


def test_batch_other_gates_and_fixed_angles(qs):
    n = 5
    gates = [W.Gate("H", (0,)), W.Gate("CNOT", (1,), controls=(0,), control_values=(1,)),
             W.Gate("RX", (2,), params=(0.3,), param_index=0), W.Gate("RY", (3,), params=(1.1,)),
             W.Gate("X", (4,)), W.Gate("Y", (1,)), W.Gate("Z", (2,)), W.Gate("RZ", (4,), params=(-0.7,), param_index=1),
             W.Gate("CZ", (3, 4))]
    c = W.Circuit(n, gates, n_params=2)
    obs = W.random_pauli_observable(n, 5, 3)
    b = qs.Batch([c], [obs])
    e, g = b.run(c.parameters(), use_graph=False)
    assert abs(e[0] - oracle.energy(c, obs)) < 2e-6
    assert np.max(np.abs(g[0] - oracle.grad_parameter_shift(c, obs, [0, 1]))) < 2e-6


def test_batch_rejects_unsupported(qs):
    c = W.Circuit(5, [W.Gate("U3", (0,), params=(0.1, 0.2, 0.3))])
    with pytest.raises(qs.QsError) as e:
        qs.Batch([c], [W.tfim_observable(5)])
    assert e.value.code == qs.QS_ERR_UNSUPPORTED
    small = W.Circuit(3, [W.Gate("H", (0,))])
    with pytest.raises(qs.QsError) as e:
        qs.Batch([small], [W.tfim_observable(3)])
    assert e.value.code == qs.QS_ERR_INVALID_ARG
