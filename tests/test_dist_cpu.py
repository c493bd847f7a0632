"""Multi-rank host logic on CPU (gloo, world size 2): problem sharding is a
partition, and the benchmark's max-over-ranks timing reduction works."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_math_9809043_gb300 import dist as D


def test_shard_partitions():
    items = list(range(17))
    for world in (1, 2, 3, 8):
        parts = [D.shard(items, r, world) for r in range(world)]
        assert sorted(sum(parts, [])) == items
        assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_shard_by_work_balances():
    works = [512 ** 2, 64 ** 2, 256 ** 2, 128 ** 2, 384 ** 2, 96 ** 2, 192 ** 2] * 5
    parts = [D.shard_by_work(works, r, 2) for r in range(2)]
    assert sorted(sum(parts, [])) == list(range(len(works)))
    loads = [sum(works[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(works)


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
    try:
        mine = D.shard(list(range(10)), rank, world)
        m = D.max_over_ranks(float(rank * 3 + 1))
        D.barrier()
        out[rank] = (mine, m)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gloo_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][1] == out[1][1] == 4.0
    assert sorted(out[0][0] + out[1][0]) == list(range(10))
