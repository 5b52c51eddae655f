"""Multi-GPU layout: independent shards, no data-path collective.

Instances (and subtrees) are independent, so N processes (one per GPU) each
run their own shard; the only cross-rank traffic is the reduction of the
timing (max) and of the node/solution counts (sum) at the end.
"""
from __future__ import annotations

from typing import Sequence, Tuple


def shard_bounds(count: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced shard [lo, hi) of `count` items for `rank`."""
    if world < 1 or not (0 <= rank < world) or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard(items: Sequence, rank: int, world: int):
    lo, hi = shard_bounds(len(items), rank, world)
    return list(items[lo:hi])


def reduce_max_sum(values_max: float, values_sum: float, world: int, device: str = "cpu"):
    """(max over ranks, sum over ranks) with the current process group."""
    if world == 1:
        return values_max, values_sum
    import torch
    import torch.distributed as dist
    t = torch.tensor([values_max], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([values_sum], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())
