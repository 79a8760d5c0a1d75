"""The multi-GPU (one process per GPU) host logic, run as world_size-2 gloo
ranks on the CPU: channel partition, the max-over-ranks timing, the whole-job
rate, and a fixed band split across ranks whose per-rank images (here from the
oracle, the stand-in for each rank's GPU plan) reassemble into the one-rank
packed output.  No GPU is involved."""
import os
import socket

import pytest

from paper_2301_09662_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, grid_n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.shard_channels(grid_n, world, rank)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        # a rank-dependent "step time": the slowest rank decides
        t = 1.0 + 0.5 * rank
        tmax = shard.max_over_ranks(t)
        rate = shard.whole_job_rate(1000, world, tmax)
        q.put((rank, everyone, tmax, rate, shard.rank_first_channel(64, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_time():
    import torch.multiprocessing as mp
    grid_n = [64] * 64 + [96] * 64 + [128] * 64
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, grid_n, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    shards = results[0][1]
    assert results[1][1] == shards
    flat = [c for s in shards for c in s]
    assert flat == list(range(len(grid_n)))          # every channel once, in order
    costs = [sum(shard.channel_cost(grid_n[c]) for c in s) for s in shards]
    assert max(costs) / min(costs) < 1.1              # balanced by N^2 log N
    assert all(r[2] == 1.5 for r in results)          # max over ranks
    assert all(abs(r[3] - 2 * 1000 / 1.5) < 1e-9 for r in results)
    assert [r[4] for r in results] == [0, 64]


def _band():
    """A small dual-pol band with uneven grid sides (32 and 64), so that the
    channels' packed blocks differ in size."""
    import numpy as np
    from paper_2301_09662_gb300 import synth
    wl = synth.random_small(A=6, P=2, C=5, T=3, N=32, K=3, seed=91)
    wl.grid_n = np.array([32, 64, 32, 64, 64], np.int32)
    return wl


def _band_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _band()
        ch, a, b = shard.band_slice(wl.grid_n, wl.n_pol, world, rank)
        local = oracle.workload_image(wl, channels=ch) if ch else np.zeros(0, np.complex128)
        assert local.size == b - a
        full = shard.assemble_band(torch.from_numpy(local.astype(np.complex64)), wl.grid_n, wl.n_pol)
        q.put((rank, ch, a, b, None if full is None else full.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_fixed_band_split_reassembles_the_one_rank_output(world):
    """Each rank images only its `band_slice` channels; assemble_band on rank 0
    equals the whole band imaged by one rank, block for block (world 3 also has
    ranks of unequal slice length)."""
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    wl = _band()
    want = oracle.workload_image(wl).astype(np.complex64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [c for r in results for c in r[1]] == list(range(wl.C))
    assert results[0][2] == 0 and results[-1][3] == want.size
    assert all(results[i][3] == results[i + 1][2] for i in range(world - 1))   # slices tile the band
    assert all(r[4] is None for r in results[1:])
    assert np.array_equal(results[0][4], want)


def test_band_slice_single_rank_is_the_band():
    import numpy as np
    import torch
    grid_n = [32, 64, 96]
    ch, a, b = shard.band_slice(grid_n, 1, 1, 0)
    assert ch == [0, 1, 2] and (a, b) == (0, 32 * 32 + 64 * 64 + 96 * 96)
    assert shard.packed_offsets(grid_n, 2)[-1] == 4 * (32 * 32 + 64 * 64 + 96 * 96)
    x = torch.arange(b, dtype=torch.float32).to(torch.complex64)
    assert shard.assemble_band(x, grid_n, 1) is x
    with pytest.raises(ValueError):
        shard.assemble_band(x[:-1], grid_n, 1)
    assert np.array_equal(shard.band_slice([128, 128], 2, 4, 3)[1:], (0, 0))


@pytest.mark.parametrize("world", [1, 3, 8])
def test_shard_channels_covers_everything(world):
    grid_n = [128] * 10 + [64] * 7
    parts = [shard.shard_channels(grid_n, world, r) for r in range(world)]
    assert [c for p in parts for c in p] == list(range(len(grid_n)))


def test_more_ranks_than_channels():
    parts = [shard.shard_channels([128, 128], 4, r) for r in range(4)]
    assert sorted(c for p in parts for c in p) == [0, 1]


def test_select_channels_is_the_same_band_subset():
    """The per-rank workload of a split band (synth.select_channels) images to
    the same values as those channels of the whole band."""
    import numpy as np
    import oracle
    from paper_2301_09662_gb300 import synth
    wl = _band()
    ch, a, b = shard.band_slice(wl.grid_n, wl.n_pol, 2, 1)
    sub = synth.select_channels(wl, ch)
    assert sub.C == len(ch) and sub.T == wl.T and np.array_equal(sub.grid_n, wl.grid_n[ch])
    assert np.array_equal(oracle.workload_image(sub), oracle.workload_image(wl)[a:b])
