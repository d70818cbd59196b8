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


def test_bin_terms_with_denominators_far_outside_the_reciprocal_range(ctx):
    """FP32 bin terms A^2 / (B + 1/alpha^2) whose denominators lie outside
    [2^-100, 2^100] (there the kernel scales numerator and denominator before
    its reciprocal-based quotient): x and sigma scaled by 2^-45 (S is invariant,
    B per bin ~1e32), 1/alpha^2 = 1e38 (every denominator ~1e38), and 1/alpha^2
    = 3e-38 with short curves (empty bins whose denominator is 1/alpha^2 alone).
    The batched call and the several-M call against the oracle."""
    import paper_2502_00243_gb300 as G
    lam = 2.0 ** -45
    w = L.ragged(95, [1500, 900, 2400], 3001, M=20, k=5)
    w.x, w.sigma = w.x * lam, w.sigma * lam
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 20, k=9)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        assert np.sum(1.0 / s ** 2) / 20 > 2.0 ** 100  # the mean bin's B is beyond the reciprocal's range
        near = oracle.min_edge(t, w.freqs, 20) <= 1e-9
        assert_S_close(Sd[c], S_or[c], s_bound(x, s), mask=~near, what=f"scaled sigma curve {c}")
        check_topk(idx[c], Sk[c], o_idx[c], o_S[c], o_dense=S_or[c], abs_tol=1e-7 * s_bound(x, s))
    mi, mo, ms_, md = _multi(G, ctx, w, 20, (1, 4), 5)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        for q, g in enumerate((1, 4)):
            Sg = oracle.fpw_multi(t, x, s, w.freqs, 20, g).max(axis=0)
            assert_S_close(md[c, q], Sg, s_bound(x, s), rel=1e-4, mask=~(oracle.min_edge(t, w.freqs, 20) <= 1e-9),
                           what=f"scaled sigma several-M g={g} curve {c}")
    for ia2, ns in ((1e38, [1500, 900]), (3e-38, [5, 3, 40, 1500])):
        w = L.ragged(96, ns, 2001, M=20, k=5)
        idx, Sk, Sd, st = run_batch(ctx, w, dense=True, params=G.fpw_params_default(inv_alpha2=ia2))
        assert st == 0
        S_or, _, _ = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 20, ia2)
        assert np.isfinite(Sd).all()
        for c in range(w.ncurves):
            t, x, s = w.curve(c)
            ok = ~(oracle.min_edge(t, w.freqs, 20) <= 1e-9)
            if ia2 < 1.0:
                assert_S_close(Sd[c], S_or[c], s_bound(x, s), mask=ok, what=f"1/alpha^2={ia2} curve {c}")
            else:
                # S ~ 1e-32 here: the absolute floor is 1e-7 of the largest S this curve can have,
                # (sum |x| / sigma^2)^2 / (1/alpha^2), instead of 1e-7 sum w x^2
                floor = 1e-7 * np.sum(np.abs(x) / s ** 2) ** 2 / ia2
                err = np.abs(Sd[c] - S_or[c])[ok]
                assert (err <= 1e-4 * np.abs(S_or[c][ok]) + floor).all(), f"1/alpha^2={ia2} curve {c}: {err.max()}"
                assert np.median(Sd[c][ok]) > 1e3 * floor


def _multi(G, ctx, w, M_max, groups, k):
    from gpu_util import to_dev
    d = to_dev(w)
    C, F, ng = w.ncurves, w.nfreq, len(groups)
    idx = torch.empty(C * ng * k, dtype=torch.int32, device="cuda")
    off = torch.empty(C * ng * k, dtype=torch.int32, device="cuda")
    S = torch.empty(C * ng * k, dtype=torch.float32, device="cuda")
    Sd = torch.empty(C * ng * F, dtype=torch.float64, device="cuda")
    G.fpw_periodogram_batch_multi(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"],
                                  M_max, groups, k, idx, off, S, Sd)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return (idx.cpu().numpy().reshape(C, ng, k), off.cpu().numpy().reshape(C, ng, k),
            S.cpu().numpy().reshape(C, ng, k), Sd.cpu().numpy().reshape(C, ng, F))
