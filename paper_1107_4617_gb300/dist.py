"""Multi-GPU orchestration for independent images (one process per GPU).

The filter has no exchange step between images: with several GPUs each rank
filters its own images and no collective touches the data path. Ranks only
meet to time a run (a barrier before and after, then the slowest rank's time).
These helpers hold that host logic; they work with any torch.distributed
backend (NCCL on GPUs, gloo on CPU for the tests).
"""
from __future__ import annotations

import heapq


def shard(costs, rank: int, world: int):
    """Indices of the items rank `rank` of `world` processes, assigned by
    longest-processing-time-first: items sorted by decreasing cost, each given
    to the currently least-loaded rank (ties to the lowest rank). Deterministic,
    so every rank computes the same partition without communicating."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(units_this_rank: float, seconds_this_rank: float, device=None) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest
    rank's time."""
    total = sum_over_ranks(units_this_rank, device)
    slowest = max_over_ranks(seconds_this_rank, device)
    return total / slowest if slowest > 0 else 0.0
