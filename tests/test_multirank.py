"""Two-rank (gloo, CPU) checks of the multi-GPU path: curves shard across ranks
with no data-path collective; only timing is reduced (max time, summed work)."""
from __future__ import annotations

import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batches = bench.shard_batches(13, world, rank, 10)
        ms, ev = bench.reduce_timing(dist, "cpu", 100.0 + rank, 1e12 * (rank + 1))
        gathered = [None] * world
        dist.all_gather_object(gathered, batches)
        out[rank] = (ms, ev, gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_disjoint_batches_and_reduce_timing():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, ev, gathered = out[r]
        assert ms == 101.0 and ev == 3e12  # max over ranks, sum over ranks
    b0, b1 = out[0][2]
    for s in range(13):
        assert b0[s] != b1[s]  # disjoint within every step
    assert set(b0[:5]) | set(b1[:5]) == set(range(10))  # five steps of two ranks cover the ten batches


def test_single_rank_is_identity():
    assert bench.reduce_timing(None, "cpu", 5.0, 7.0) == (5.0, 7.0)
    assert bench.shard_batches(12, 1, 0, 10) == [s % 10 for s in range(12)]
