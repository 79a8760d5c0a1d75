"""The multi-GPU (one process per GPU) host logic, run as world_size-2 gloo
ranks on the CPU: channel partition, the max-over-ranks timing and the
whole-job rate.  No GPU and no data-path collective is involved."""
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


@pytest.mark.parametrize("world", [1, 3, 8])
def test_shard_channels_covers_everything(world):
    grid_n = [128] * 10 + [64] * 7
    parts = [shard.shard_channels(grid_n, world, r) for r in range(world)]
    assert [c for p in parts for c in p] == list(range(len(grid_n)))


def test_more_ranks_than_channels():
    parts = [shard.shard_channels([128, 128], 4, r) for r in range(4)]
    assert sorted(c for p in parts for c in p) == [0, 1]
