"""Multi-process host logic over gloo on the CPU (world_size 2).

The multi-GPU headline run of bench.py is independent replicas: each rank simulates its own
seeded circuit, ranks meet only for the barrier and the max-over-ranks timing. The batched
workload is split across ranks by pair cost, with no exchange but the gather of the results on
rank 0. Both are run here with the oracle standing in for the GPU kernels."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)

    class A:
        n, depth, seed = 6, 3, 100

    c = bench.replica_circuit(A, rank)
    psi = oracle.run_circuit(c)
    local_ms = 10.0 * (rank + 1)
    dist.barrier()
    mx = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(world, len(c.gates), 3, mx)
    out[rank] = (mx, rate, float(np.abs(psi[0])), c.gates[0].params)
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, free_port(), out), nprocs=world, start_method="spawn", join=True)
    (mx0, rate0, a0, p0), (mx1, rate1, a1, p1) = out[0], out[1]
    assert mx0 == mx1 == 20.0                       # the slowest rank's time on both ranks
    gates = 6 * 3 + (3 + 2 + 3)                     # U3 layers + CZ brickwork of n = 6, depth 3
    assert rate0 == rate1 == pytest.approx(2 * gates * 3 / 0.020)
    assert p0 != p1 and a0 != a1                    # independent replicas (different seeds)


def _batch_rank(rank, world, port, out):
    """One rank of a sharded batch: its pairs by the cost split, evaluated (here by the oracle,
    standing in for the GPU kernel), results gathered on every rank in the batch's order."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import workloads as W
    from paper_2011_13524_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = W.batch_workload(12, 77, n_lo=3, n_hi=8, l_lo=1, l_hi=3)
    parts = shard.split([shard.pair_cost(i.circuit) for i in items], world)
    idx = parts[rank]
    e = [oracle.energy(items[i].circuit, items[i].observable) for i in idx]
    g = [oracle.grad_parameter_shift(items[i].circuit, items[i].observable, range(2)) for i in idx]
    e_all, g_all = shard.gather(dist, len(items), idx, e, g)
    out[rank] = (parts, list(e_all), [list(x) for x in g_all])
    dist.destroy_process_group()


def test_batch_split_by_cost_and_gathered_over_gloo():
    """world_size 2: the split is the same on both ranks, disjoint, covers every pair and balances
    the cost within one pair's cost; the gathered energies and gradients equal a single process's
    evaluation of the whole batch, in the batch's order."""
    import oracle
    import workloads as W
    from paper_2011_13524_gb300 import shard
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_batch_rank, args=(world, free_port(), out), nprocs=world, start_method="spawn", join=True)
    (parts0, e0, g0), (parts1, e1, g1) = out[0], out[1]
    assert parts0 == parts1
    flat = sorted(parts0[0] + parts0[1])
    items = W.batch_workload(12, 77, n_lo=3, n_hi=8, l_lo=1, l_hi=3)
    assert flat == list(range(len(items))) and not set(parts0[0]) & set(parts0[1])
    costs = [shard.pair_cost(i.circuit) for i in items]
    loads = [sum(costs[i] for i in p) for p in parts0]
    assert abs(loads[0] - loads[1]) <= max(costs)
    ref_e = [oracle.energy(i.circuit, i.observable) for i in items]
    ref_g = [oracle.grad_parameter_shift(i.circuit, i.observable, range(2)) for i in items]
    assert e0 == e1 == ref_e
    assert all(np.array_equal(a, b) and np.array_equal(a, c) for a, b, c in zip(g0, g1, ref_g))


def test_split_single_rank_and_errors():
    from paper_2011_13524_gb300 import shard
    assert shard.split([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    assert shard.split([5.0, 4.0, 3.0, 3.0], 2) == [[0, 3], [1, 2]]
    with pytest.raises(ValueError):
        shard.split([1.0], 0)
    with pytest.raises(ValueError):
        shard.gather(None, 3, [0, 1], [1.0, 2.0], [np.zeros(1), np.zeros(1)])
