"""Partition of independent runs across ranks (one process per GPU).

Runs of an ensemble do not interact, so a multi-GPU job shards them with no
collective on the data path: each rank steps its own runs, and only the
timing (max over ranks) and per-run diagnostics are gathered at the end.
The partition balances the transform work, which grows as P log2 P for a
run of P grid points.
"""
from __future__ import annotations

import math


def run_cost(n: int, d: int = 2) -> float:
    p = float(n) ** d
    return p * math.log2(p)


def shard_runs(ns, world: int, d: int = 2):
    """Longest-processing-time-first assignment of runs (grid sizes `ns`) to
    `world` ranks: runs in decreasing cost (ties by index) each go to the rank
    with the least load so far (ties to the lowest rank). Returns one sorted
    list of run indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(ns)), key=lambda i: (-run_cost(ns[i], d), i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += run_cost(ns[i], d)
    return [sorted(x) for x in out]


def max_over_ranks(value: float, dist=None) -> float:
    """The maximum of a per-rank float over the process group (the value
    itself without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
