"""Weak-scaling helpers for runs with one process per GPU (host logic only).

The method shards over independent solves: every instance of a batch, every request of
a served stream, is a Helmholtz problem of its own, so ranks exchange nothing on the
data path.  What the ranks share is the timing protocol: a barrier before and after the
timed region, and the maximum of the ranks' times, from which the whole-job throughput
is (units all ranks processed) / (max time).

The process group is whatever the caller created (NCCL on GPUs; gloo on CPU in the
tests); these functions only use ``barrier`` and ``all_reduce`` / ``all_gather_object``.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, rank: int, ws: int) -> range:
    """Contiguous block of `count` units owned by `rank` (sizes differ by at most one)."""
    if ws < 1 or not 0 <= rank < ws or count < 0:
        raise ValueError(f"bad shard request count={count} rank={rank} ws={ws}")
    base, extra = divmod(count, ws)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist=None, device=None) -> float:
    """Sum of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(units_this_rank: float, seconds_this_rank: float, dist=None, device=None) -> float:
    """Whole-job units per second: units summed over ranks / the slowest rank's time."""
    units = sum_over_ranks(units_this_rank, dist, device)
    secs = max_over_ranks(seconds_this_rank, dist, device)
    return units / secs if secs > 0 else float("inf")
