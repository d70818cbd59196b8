"""Edge cases of the GPU path against the oracle: very large M (one frequency
per thread), huge t*f, negative times, one-observation curves, k larger than
the number of peaks, and unsupported combinations rejected cleanly."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, check_topk, run_batch, run_single, s_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G
    c = G.Context(0)
    yield c
    c.close()


def test_large_bin_count_uses_one_frequency_per_thread(ctx):
    w = L.ragged(90, [1500, 300], 700, M=200, k=5)
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 200, k=9)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        near = oracle.min_edge(t, w.freqs, 200) <= 1e-9
        assert_S_close(Sd[c], S_or[c], s_bound(x, s), mask=~near, what=f"M=200 curve {c}")
        check_topk(idx[c], Sk[c], o_idx[c], o_S[c], o_dense=S_or[c], abs_tol=1e-7 * s_bound(x, s))


def test_huge_phases_and_negative_times(ctx):
    rng = np.random.default_rng(5)
    n = 400
    t = np.concatenate([rng.uniform(-3e4, 0, n // 2), rng.uniform(1e5, 3e5, n // 2)])  # |t f| up to ~3e8 cycles
    sigma = rng.uniform(0.05, 0.2, n)
    x = rng.normal(0, 1, n) * sigma
    freqs = np.linspace(900.0, 1000.0, 1500)
    S_or = oracle.fpw(t, x, sigma, freqs, 16)
    S_g, st = run_single(ctx, t, x, sigma, freqs, 16)
    assert st == 0
    # the oracle rounds t*f to binary64 (half an ulp = 3e-8 cycles at 3e8 cycles), so its own bins are
    # exact only beyond that distance from an edge; the GPU's exact anchor (this grid is not linear to
    # 2e-10 cycles at |t| = 3e5, so every pair is anchored directly) is exact to 2^-32 cycles
    near = oracle.min_edge(t, freqs, 16) <= 1e-7
    assert (~near).sum() > 100
    assert_S_close(S_g, S_or, s_bound(x, sigma), mask=~near, what="huge t f")


def test_single_observation_curves_and_k_beyond_peaks(ctx):
    w = L.ragged(91, [1, 1, 2, 3], 40, M=8, k=30)
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 8, k=34)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        # two observations in one bin leave a binary64 rounding residue (~1e-32) of the mean-subtracted
        # flux where FP32 gives 0: the absolute floor of the other parity tests covers it
        assert_S_close(Sd[c], S_or[c], s_bound(x, s), what=f"curve {c} (n={t.size})")
        check_topk(idx[c], Sk[c], o_idx[c], o_S[c], o_dense=S_or[c], abs_tol=1e-7 * s_bound(x, s))
        valid = idx[c] >= 0
        nv = int(valid.sum())
        assert nv < 30 and valid[:nv].all()  # fewer peaks than k on 40 frequencies: the rest trail as -1
        if t.size == 1:  # one observation: S is identically 0; the flat periodogram's one peak is its left end
            assert np.all(S_or[c] == 0.0) and np.all(Sd[c] == 0.0)
            assert nv == 1 and idx[c][0] == 0 and Sk[c][0] == 0.0


def test_plain_form_rejects_bins_beyond_shared_memory(ctx):
    import paper_2502_00243_gb300 as G
    w = L.ragged(92, [50], 16, M=300, k=1)
    with pytest.raises(G.FPWError) as ei:
        run_batch(ctx, w, params=G.fpw_params_default(phase_mode=G.FPW_PHASE_FP64))
    assert ei.value.code == G.FPW_ENOTSUP
