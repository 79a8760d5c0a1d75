"""Channel sharding across GPUs (one process per GPU).

Channels are imaged independently (Sec. 2.2: the GPU blocks run in parallel
across time and frequency; Sec. 5: each of a server's two GPUs images its own
band), so the multi-GPU form of the imaging path is a partition of channels
with no exchange on the data path.  Two uses:

* weak scaling: every rank images a band of the same shape next to the others
  (`rank_first_channel`);
* a fixed band split across ranks (`shard_channels`), balanced by the
  per-channel cost N^2 log2 N of the grid side.  Each rank plans and images
  only its channels (`band_slice` gives their place in the whole band's packed
  output) and `assemble_band` collects the slices into the band's packed
  layout once the integration is done.

Imaging itself needs no exchange.  The collectives are the slowest rank's time
(`max_over_ranks`) and, for a split band, the one gather of the finished
images (`assemble_band`).
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


def packed_offsets(grid_n, n_pol: int) -> list[int]:
    """Offsets (complex elements) of every channel's [NP][N][N] block in a
    plan's packed output, with the total size as the last entry (NP = 4 products
    for dual polarisation, 1 for single)."""
    NP = 4 if int(n_pol) == 2 else 1
    offs = [0]
    for n in grid_n:
        offs.append(offs[-1] + NP * int(n) * int(n))
    return offs


def band_slice(grid_n, n_pol: int, world: int, rank: int) -> tuple[list[int], int, int]:
    """Rank `rank`'s part of a fixed band split across `world` ranks: its
    channels (`shard_channels`) and the [start, stop) range of complex elements
    their images occupy in the whole band's packed output.  A plan made of
    exactly these channels, in this order, writes that range contiguously."""
    ch = shard_channels(grid_n, world, rank)
    offs = packed_offsets(grid_n, n_pol)
    if not ch:
        return ch, 0, 0
    return ch, offs[ch[0]], offs[ch[-1] + 1]


def assemble_band(local, grid_n, n_pol: int, dst: int = 0, group=None):
    """Collect every rank's packed slice (a 1-D complex tensor from a plan of
    its `band_slice` channels; empty for a rank without channels) into the whole
    band's packed output on rank `dst` (None on the others).

    One all_gather of equal-length buffers (each slice padded to the longest),
    as complex values viewed as float pairs so that gloo and NCCL both carry it;
    without torch.distributed (one rank) the slice is the band."""
    import torch
    import torch.distributed as dist
    offs = packed_offsets(grid_n, n_pol)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        if local.numel() != offs[-1]:
            raise ValueError("a single rank's slice must be the whole band")
        return local
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    spans = [band_slice(grid_n, n_pol, world, r)[1:] for r in range(world)]
    mine = spans[rank][1] - spans[rank][0]
    if local.numel() != mine:
        raise ValueError(f"rank {rank}: slice has {local.numel()} elements, its channels need {mine}")
    longest = max(b - a for a, b in spans)
    buf = torch.zeros(max(longest, 1), 2, dtype=torch.float32, device=local.device)
    if mine:
        buf[:mine] = torch.view_as_real(local.reshape(-1).to(torch.complex64))
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    if rank != dst:
        return None
    out = torch.empty(offs[-1], dtype=torch.complex64, device=local.device)
    for (a, b), part in zip(spans, parts):
        if b > a:
            out[a:b] = torch.view_as_complex(part[:b - a].contiguous())
    return out


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
