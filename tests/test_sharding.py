"""Multi-rank host logic on CPU (gloo, world size 2): disjoint frame shards
covering the batch, per-rank seeds, and the max/sum reductions bench.py uses."""
import os

import pytest
import torch.multiprocessing as mp

from paper_1206_3362_gb300.sharding import frame_seed, shard_range


@pytest.mark.parametrize("F,world", [(10, 3), (1 << 20, 8), (1, 2), (0, 4)])
def test_shard_range_partitions(F, world):
    covered = []
    for r in range(world):
        lo, hi = shard_range(F, r, world)
        covered.extend(range(lo, hi))
        assert 0 <= hi - lo <= F // world + 1
    assert covered == list(range(F))


def test_frame_seeds_distinct():
    assert len({frame_seed(7, r) for r in range(64)}) == 64


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_1206_3362_gb300.sharding import max_over_ranks, sum_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mx = max_over_ranks(float(rank + 1) * 1.5)
    sm = sum_over_ranks(float(rank + 1))
    out[rank] = (mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_reductions_gloo_world2():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mgr = mp.get_context("spawn").Manager()  # no fork of a process that may already run threads
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (3.0, 3.0) and out[1] == (3.0, 3.0)
