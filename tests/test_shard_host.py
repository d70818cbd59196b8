"""Host-side sharding over ranks (paper_2502_00243_gb300.shard) on CPU: two gloo
ranks, each computing its part with the oracle in place of its GPU, must give
the single-process oracle's per-curve top-k (curves split by cost) and the
full-grid top-k of one curve whose frequencies are split with a halo."""
from __future__ import annotations

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import lightcurves as L  # noqa: E402
import oracle  # noqa: E402
from paper_2502_00243_gb300 import shard  # noqa: E402


def oracle_compute(M):
    def run(offsets, t, x, sigma, freqs, k):
        _, idx, S = oracle.fpw_batch(offsets, t, x, sigma, freqs, M, dense=False, k=k)
        return idx, S.astype(np.float32)
    return run


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = L.ragged(5, [900, 40, 2500, 0, 333, 1200, 77], 3000, M=20, k=5)
        bi, bs = shard.batch_topk_sharded(oracle_compute(20), w.offsets, w.t, w.x, w.sigma, w.freqs, 5, rank, world,
                                          dist)
        one = L.ragged(6, [1500], 4001, M=12)
        t, x, s = one.curve(0)
        ci, cs = shard.curve_topk_split(oracle_compute(12), t, x, s, one.freqs, 7, rank, world, dist)
        out[rank] = (bi, bs, ci, cs)
    finally:
        dist.destroy_process_group()


def test_two_ranks_reproduce_the_single_process_top_k():
    world = 2
    port = 31500 + (os.getpid() % 2000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    w = L.ragged(5, [900, 40, 2500, 0, 333, 1200, 77], 3000, M=20, k=5)
    _, ri, rs = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 20, dense=False, k=5)
    one = L.ragged(6, [1500], 4001, M=12)
    t, x, s = one.curve(0)
    S_full = oracle.fpw(t, x, s, one.freqs, 12)
    ci_ref, cs_ref = oracle.topk(S_full, 7)
    for r in range(world):
        bi, bs, ci, cs = out[r]
        np.testing.assert_array_equal(bi, ri)
        np.testing.assert_array_equal(bs, rs.astype(np.float32))
        np.testing.assert_array_equal(ci, ci_ref)
        np.testing.assert_allclose(cs, cs_ref.astype(np.float32))


def test_lpt_partition_balances_cost_and_covers_every_curve():
    rng = np.random.default_rng(3)
    n = rng.integers(0, 3000, 1000)
    off = np.concatenate(([0], np.cumsum(n)))
    parts = shard.lpt_partition(off, 100, 4)
    allc = np.sort(np.concatenate(parts))
    np.testing.assert_array_equal(allc, np.arange(1000))
    loads = [float(np.sum(n[p] + 32)) for p in parts]
    assert max(loads) - min(loads) <= float(np.max(n) + 32)  # LPT: within one job of balance


def test_frequency_parts_own_every_frequency_once_with_halos():
    for F, P in ((10, 3), (4001, 2), (5, 8), (1, 2)):
        parts = shard.frequency_parts(F, P)
        owned = np.concatenate([np.arange(lo, hi) for lo, hi, a, b in parts])
        np.testing.assert_array_equal(owned, np.arange(F))
        for lo, hi, a, b in parts:
            assert a == max(lo - 1, 0) and b == min(hi + 1, F)


def test_merge_ranks_by_S_then_lower_index():
    idx, S = shard.merge_topk([[(7, 2.0), (3, 1.0)], [(5, 2.0), (9, 0.5)]], 5)
    assert list(idx) == [5, 7, 3, 9, -1] and np.isnan(S[4])


def test_chunked_run_resumes_after_an_interruption(tmp_path):
    w = L.ragged(7, [300, 0, 1200, 50, 800, 999, 31, 450, 2000], 1500, M=10, k=4)
    full_i, full_s = shard.run_chunked(oracle_compute(10), w.offsets, w.t, w.x, w.sigma, w.freqs, 4, 100)
    calls = []

    def flaky(offsets, t, x, sigma, freqs, k):
        if len(calls) == 2:
            raise RuntimeError("interrupted")
        calls.append(len(offsets) - 1)
        return oracle_compute(10)(offsets, t, x, sigma, freqs, k)

    with pytest.raises(RuntimeError):
        shard.run_chunked(flaky, w.offsets, w.t, w.x, w.sigma, w.freqs, 4, 2, state_dir=str(tmp_path))
    assert calls == [2, 2] and len(list(tmp_path.glob("chunk_*.npz"))) == 2
    done = []

    def counted(offsets, t, x, sigma, freqs, k):
        done.append(len(offsets) - 1)
        return oracle_compute(10)(offsets, t, x, sigma, freqs, k)

    ri, rs = shard.run_chunked(counted, w.offsets, w.t, w.x, w.sigma, w.freqs, 4, 2, state_dir=str(tmp_path))
    assert done == [2, 2, 1]  # the two saved chunks are not recomputed
    np.testing.assert_array_equal(ri, full_i)
    np.testing.assert_array_equal(rs, full_s)
    assert not list(tmp_path.glob("*.tmp.npz"))
