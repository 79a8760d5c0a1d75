"""Channel sharding across GPUs (one process per GPU).

Channels are imaged independently (Sec. 2.2: the GPU blocks run in parallel
across time and frequency; Sec. 5: each of a server's two GPUs images its own
band), so the multi-GPU form of the imaging path is a partition of channels
with no exchange on the data path.  Two uses:

* weak scaling: every rank images a band of the same shape next to the others
  (`rank_first_channel`);
* a fixed band split across ranks (`shard_channels`), balanced by the
  per-channel cost N^2 log2 N of the grid side.

The only collective is on the control path: the slowest rank's time
(`max_over_ranks`).
"""
from __future__ import annotations

import math


def rank_first_channel(channels_per_rank: int, rank: int) -> int:
    """First channel index of rank `rank` when every rank images its own band
    of `channels_per_rank` adjacent channels."""
    if channels_per_rank < 1 or rank < 0:
        raise ValueError("channels_per_rank must be >= 1 and rank >= 0")
    return rank * channels_per_rank


def channel_cost(n: int) -> float:
    """Relative cost of one channel of grid side n (transform-dominated)."""
    return float(n) * n * math.log2(n)


def shard_channels(grid_n, world: int, rank: int) -> list[int]:
    """Contiguous, cost-balanced block of channel indices for `rank`.

    Every channel goes to exactly one rank; channel order is kept so each rank's
    output is one contiguous slice of the packed image array.  A rank may get
    no channel when there are fewer channels than ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    costs = [channel_cost(int(n)) for n in grid_n]
    total = sum(costs)
    bounds = [0]
    acc = 0.0
    c = 0
    for r in range(1, world):
        target = total * r / world
        while c < len(costs) and acc + costs[c] / 2 <= target:
            acc += costs[c]
            c += 1
        bounds.append(c)
    bounds.append(len(costs))
    return list(range(bounds[rank], bounds[rank + 1]))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Aggregate throughput: the units every rank processed over the slowest
    rank's time."""
    if max_seconds <= 0:
        raise ValueError("max_seconds must be positive")
    return world * units_per_rank / max_seconds
