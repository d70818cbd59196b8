"""The no-allocation batched entry point against the regular one.

fpw_periodogram_batch_noalloc serves callers that cannot call cudaMalloc
(inside another framework's memory pool, plugins that may not allocate after
start-up, real-time pipelines that must not allocate mid-run): its scratch is a
fixed device array inside the library. This file is collected last so that a
run stopping at the first failure has already run every other test."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
from gpu_util import check_topk, run_batch, s_bound, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(G, w, d, offsets_host):
    C, k = w.ncurves, w.k
    idx = torch.full((C * k,), -7, dtype=torch.int32, device="cuda")
    S = torch.full((C * k,), -7.0, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_noalloc(None, None, d["offsets"], offsets_host, d["t"], d["x"], d["sigma"], d["freqs"],
                                    w.M, k, idx, S)
    return idx.cpu().numpy().reshape(C, k), S.cpu().numpy().reshape(C, k)


def test_noalloc_matches_batch_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G
    w = L.ragged(31, [0, 1, 40, 700, 1500, 3100, 333], 20_000, M=20, k=5)
    d = to_dev(w)
    ctx = G.Context(0)
    ref_idx, ref_S, _, st = run_batch(ctx, w, d=d)
    assert st == 0
    ctx.close()
    # second call without the host offsets (the library reads offsets[C] back)
    for offsets_host in (w.offsets, None):
        idx, S = _noalloc(G, w, d, offsets_host)
        for c in range(w.ncurves):
            t, x, s = w.curve(c)
            check_topk(idx[c], S[c], ref_idx[c], ref_S[c].astype(np.float64), abs_tol=1e-7 * s_bound(x, s),
                       what=f"noalloc curve {c}")
            np.testing.assert_allclose(S[c][idx[c] >= 0], ref_S[c][ref_idx[c] >= 0], rtol=1e-4)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G
    n = 5_000_000  # 8 B of weights per observation exceeds the 32 MiB array
    off = np.array([0, n], dtype=np.int64)
    big = torch.ones(n, dtype=torch.float64, device="cuda")
    freqs = torch.linspace(0.1, 1.0, 8, dtype=torch.float64, device="cuda")
    idx = torch.empty(2, dtype=torch.int32, device="cuda")
    S = torch.empty(2, dtype=torch.float32, device="cuda")
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram_batch_noalloc(None, None, torch.from_numpy(off).cuda(), off, big, big, big, freqs, 4, 2,
                                        idx, S)
    assert ei.value.code == G.FPW_EINVAL
