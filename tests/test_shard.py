"""Host logic of the multi-GPU layout, on CPU with gloo (world size 2 and 3)."""
import os
import socket

import pytest

from paper_2508_08702_gb300.shard import reduce_max_sum, shard, shard_bounds


@pytest.mark.parametrize("count,world", [(64, 1), (64, 2), (64, 8), (7, 3), (0, 4), (5, 8)])
def test_shards_partition_the_batch(count, world):
    seen = []
    for r in range(world):
        lo, hi = shard_bounds(count, r, world)
        assert 0 <= lo <= hi <= count
        seen.extend(range(lo, hi))
    assert seen == list(range(count))
    sizes = [shard_bounds(count, r, world)[1] - shard_bounds(count, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = list(range(64))
    mine = shard(items, rank, world)
    # each rank "times" its shard and counts its items
    t_max, n_sum = reduce_max_sum(float(rank + 1), float(len(mine)), world)
    out.put((rank, mine, t_max, n_sum))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reduce_timing_and_counts(world):
    import torch.multiprocessing as mp
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
    res.sort()
    assert sorted(x for _, mine, _, _ in res for x in mine) == list(range(64))
    for _, _, t_max, n_sum in res:
        assert t_max == float(world)
        assert n_sum == 64.0
