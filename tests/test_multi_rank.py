"""The N > 1 path on CPU: two gloo ranks split the views, render nothing on a GPU, and reduce timing
(max) and work (sum) the way bench.py does under torchrun."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2603_02887_gb300.distributed import shard_views


def test_shard_views_partition():
    for n in (0, 1, 7, 32):
        for world in (1, 2, 3, 8):
            got = [v for r in range(world) for v in shard_views(n, r, world)]
            assert got == list(range(n))
            sizes = [len(shard_views(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_views(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2603_02887_gb300.distributed import max_over_ranks, sum_over_ranks, shard_views

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    views = shard_views(32, rank, world)
    fake_ms = 10.0 + rank  # a rank-dependent "step time"
    pixels = sum(640 * 360 for _ in views)
    out[rank] = (views, max_over_ranks(fake_ms), sum_over_ranks(pixels))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    assert res[0][0] + res[1][0] == list(range(32))
    assert res[0][1] == res[1][1] == 11.0
    assert res[0][2] == res[1][2] == 32 * 640 * 360
