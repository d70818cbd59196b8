"""Precision study on the 2000-day, 500 1/d workload (t f up to 10^6 cycles) and
autotuner parity, on the GPU against the oracle.

Per phase mode: the bin-mismatch rate (kernel bins vs oracle bins), how many
mismatches sit farther than 1e-9 cycles from an edge, and the S relative error
on windows of the 2e6-point grid near 100, 250, 400 and 499 1/d."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, check_topk, run_batch, run_single, s_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WINDOWS = (100.0, 250.0, 400.0, 499.0)
NWIN = 2048


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


def _study(G, ctx, mode, K):
    w = L.make("precision", range(3))
    full = L.freq_grid("precision")
    p = G.fpw_params_default(phase_mode=mode, K=K)
    total = far = bad_S = 0
    errs = []
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        for f0 in WINDOWS:
            a = int(np.searchsorted(full, f0))
            fr = full[a:a + NWIN]
            tt, ff = torch.from_numpy(t).cuda(), torch.from_numpy(fr).cuda()
            out = torch.empty(NWIN * t.size, dtype=torch.int32, device="cuda")
            G.fpw_debug_bins(ctx, None, p, tt, ff, w.M, out)
            g = out.cpu().numpy().reshape(NWIN, t.size)
            b, e = oracle.bins(t, fr, w.M)
            mm = g != b
            total += int(mm.sum())
            far += int((mm & (e > 1e-9)).sum())
            S_or = oracle.fpw(t, x, s, fr, w.M)
            S_g, st = run_single(ctx, t, x, s, fr, w.M, p)
            assert st == 0
            errs.append(np.abs(S_g - S_or) / np.maximum(np.abs(S_or), 1e-300))
    errs = np.concatenate(errs)
    pairs = w.ncurves * len(WINDOWS) * NWIN * 1500
    return total, far, pairs, float(errs.max()), float(np.median(errs))


@pytest.mark.parametrize("mode,K", [(0, 256), (1, 256), (2, 64), (2, 256), (2, 1024)])
def test_precision_study(G, mode, K):
    ctx = G.Context(0)
    total, far, pairs, emax, emed = _study(G, ctx, mode, K)
    name = {0: "fixed64", 1: "fp64-plain", 2: f"fp32 K={K}"}[mode]
    print(f"\n[precision] {name:14s} mismatches {total} / {pairs} ({total / pairs:.2e}); beyond 1e-9 cycles: {far}; "
          f"S rel err max {emax:.2e} median {emed:.2e}")
    if mode == 0:
        assert far == 0 and emed < 1e-5
    if mode == 1:
        assert total == 0 and emax == 0.0
    ctx.close()


def test_autotuner_installs_shapes_and_keeps_parity(G):
    from paper_2502_00243_gb300 import autotune
    ctx = G.Context(0)
    entries = autotune.tune(ctx, Ms=(20,), buckets=((0, 1 << 40),), nfreq=5000, evals_per_case=2e9,
                            candidates=((128, 4), (128, 2), (64, 8), (256, 1)))
    assert len(entries) == 1 and entries[0]["M_lo"] == 1 and entries[0]["geval_s"] > 0
    w = L.ragged(40, [900, 40, 2500, 333], 3000, M=20, k=5)
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 20, k=9)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        near = oracle.min_edge(t, w.freqs, 20) <= 1e-9
        assert_S_close(Sd[c], S_or[c], s_bound(x, s), mask=~near, what=f"tuned curve {c}")
        check_topk(idx[c], Sk[c], o_idx[c], o_S[c], o_dense=S_or[c], abs_tol=1e-7 * s_bound(x, s))
    ctx.clear_shapes()
    ctx.close()
