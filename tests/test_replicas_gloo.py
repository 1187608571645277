"""Replica bookkeeping on world_size 2 (gloo, CPU processes): shards of the
request stream, the max-time / sum-work combination of the bench, and the
final min-reduce of (cost, rank)."""
import os

import pytest

from paper_2402_03640_gb300 import replicas
from synth import serving_stream


def test_shard_partitions_the_stream():
    reqs = serving_stream(101, rate_per_s=100.0, seed=3)
    parts = [replicas.shard(reqs, r, 4) for r in range(4)]
    ids = sorted(q.rid for p in parts for q in p)
    assert ids == list(range(101))
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        replicas.shard(reqs, 4, 4)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = replicas.combine(seconds=1.0 + rank, units=10.0 * (rank + 1))
        c, who = replicas.best_over_ranks(best_cost=[7, 3][rank], rank=rank)
        mine = [r.rid for r in replicas.shard(serving_stream(10, 50.0, seed=1), rank, world)]
        q.put((rank, t, u, c, who, mine))
    finally:
        dist.destroy_process_group()


def test_combine_and_reduce_over_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, c, who, mine in out:
        assert t == 2.0 and u == 30.0          # slowest rank's time, all ranks' work
        assert (c, who) == (3, 1)              # lowest best cost and its rank
    assert sorted(out[0][5] + out[1][5]) == list(range(10))
    assert not set(out[0][5]) & set(out[1][5])


def test_combine_without_process_group_is_identity():
    assert replicas.combine(2.5, 7.0) == (2.5, 7.0)
    assert replicas.best_over_ranks(5, 0) == (5, 0)
