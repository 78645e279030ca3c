"""The multi-GPU path of bench.py is independent replicas: each rank simulates its own seeded
circuit, ranks meet only for the barrier and the max-over-ranks timing. This runs that host
logic with world_size 2 over gloo on the CPU (the simulation itself replaced by the oracle)."""
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
