"""Multi-rank logic on the CPU: LPT sharding of uneven pairs and the max over
ranks, with world_size = 2 gloo process groups."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2506_00976_gb300 import shard


def test_lpt_covers_every_pair_once_and_balances():
    sizes = [32, 64, 128, 256] * 50
    for world in (1, 2, 3, 8):
        shards = shard.lpt_shards(sizes, world)
        flat = sorted(t for s in shards for t in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(shard.pair_cost(sizes[t]) for t in s) for s in shards]
        assert max(loads) - min(loads) <= shard.pair_cost(max(sizes))


def test_lpt_equal_pairs_split_evenly():
    shards = shard.lpt_shards([128] * 180, 4)
    assert [len(s) for s in shards] == [45, 45, 45, 45]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [32, 64, 128, 256, 64, 32, 128]
        mine = shard.lpt_shards(sizes, world)[rank]
        # every rank derives the same partition without communication
        assert mine == shard.lpt_shards(sizes, world)[rank]
        out[rank] = (mine, shard.max_over_ranks(10.0 + rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_gloo_sharding_and_max():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    parts = [out[r][0] for r in range(world)]
    assert sorted(parts[0] + parts[1]) == list(range(7))
    assert not set(parts[0]) & set(parts[1])
    assert out[0][1] == out[1][1] == 11.0
