"""Splitting a batch of independent circuits across ranks (one process per GPU), and gathering
the results on rank 0.

A batch of (circuit, observable) pairs needs no exchange between GPUs: every pair is simulated
whole on one rank. The split balances the work (longest-processing-time first: pairs in order
of decreasing cost, each to the rank with the least work so far; ties to the lower rank), which
matters because the cost of a pair grows as 2^n with its qubit count. Every rank computes the
same split from the same workload, so the split itself needs no communication either; the only
collective is the gather of the results.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def pair_cost(circuit) -> float:
    """Work of one pair: its gates times its amplitudes."""
    return float(max(1, len(circuit.gates))) * float(2 ** int(circuit.n))


def split(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the pairs each rank runs (ascending within a rank)."""
    if world < 1:
        raise ValueError("world size must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(ix) for ix in out]


def gather(pg, count: int, idx: Sequence[int], energies: Sequence[float],
           grads: Sequence[np.ndarray]) -> Tuple[np.ndarray, List[np.ndarray]]:
    """All ranks' (indices, energies, gradients) collected in the original order of the batch.
    pg: torch.distributed (gloo or nccl) or None for a single process."""
    parts = [(list(idx), [float(e) for e in energies], [np.asarray(g) for g in grads])]
    if pg is not None and pg.get_world_size() > 1:
        allp = [None] * pg.get_world_size()
        pg.all_gather_object(allp, parts[0])
        parts = allp
    e_all = np.full(count, np.nan)
    g_all: List[np.ndarray] = [np.zeros(0)] * count
    seen = np.zeros(count, dtype=bool)
    for ix, es, gs in parts:
        for i, e, g in zip(ix, es, gs):
            if seen[i]:
                raise ValueError(f"pair {i} evaluated twice")
            seen[i] = True
            e_all[i] = e
            g_all[i] = g
    if not seen.all():
        raise ValueError("some pairs were evaluated by no rank")
    return e_all, g_all
