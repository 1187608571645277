"""Replicas on several GPUs: restarts and serving requests are independent,
so N processes (one per GPU) each run their own share with no collective on
the data path.  Only the timing is combined: the job's time is the slowest
rank's, its work the sum over ranks.  The functions take any initialised
torch.distributed process group (NCCL between GPUs, gloo on the CPU)."""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard(items: Sequence, rank: int, world: int) -> List:
    """Rank `rank`'s share of `items`: every world-th item from position rank
    (round robin keeps each share's size mix close to the whole stream's)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(items[rank::world])


def combine(seconds: float, units: float, device=None) -> Tuple[float, float]:
    """(max over ranks of seconds, sum over ranks of units); the identity
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def best_over_ranks(best_cost: int, rank: int, device=None) -> Tuple[int, int]:
    """The one reduction of a replicated solve: the smallest best cost over
    ranks and the lowest rank holding it."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(best_cost), int(rank)
    # cost in the high part, rank in the low part: one MIN gives both
    key = torch.tensor([int(best_cost) * 65536 + int(rank)], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    k = int(key.item())
    return k // 65536, k % 65536
