"""Sharding of independent runs across ranks (host logic; gloo on CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2012_15133_gb300.sharding import run_cost, shard_runs, max_over_ranks

ENSEMBLE_NS = [(64, 128, 256, 512)[i % 4] for i in range(256)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_are_disjoint_complete_and_balanced(world):
    sh = shard_runs(ENSEMBLE_NS, world)
    flat = [i for s in sh for i in s]
    assert sorted(flat) == list(range(len(ENSEMBLE_NS)))
    loads = [sum(run_cost(ENSEMBLE_NS[i]) for i in s) for s in sh]
    assert max(loads) <= 1.05 * (sum(loads) / world)


def test_shard_of_uneven_runs_is_deterministic():
    ns = [512, 16, 16, 16, 16, 256, 32]
    assert shard_runs(ns, 2) == shard_runs(list(ns), 2)
    assert shard_runs(ns, 2)[0] == [0]          # the one large run alone
    assert shard_runs([], 3) == [[], [], []]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_runs(ENSEMBLE_NS, world)[rank]
    t = torch.zeros(len(ENSEMBLE_NS), dtype=torch.int64)
    t[mine] = 1
    dist.all_reduce(t)                       # every run claimed exactly once
    m = max_over_ranks(10.0 + rank, dist)    # slowest rank's time
    q.put((rank, t.tolist(), m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_every_run_once_and_agree_on_the_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, claimed, m in res:
        assert claimed == [1] * len(ENSEMBLE_NS)
        assert m == 10.0 + world - 1
