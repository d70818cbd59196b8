"""The baseline-drift statistic (Appendix A.1-A.2) on the GPU against the dense
oracle: ragged batches with empty and one-observation curves, tile tails,
K = 0..4 basis functions, finite and infinite alpha, invalid curves, the
no-baseline limit against the batched Eq. 1 path, and rejected arguments."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, check_topk, run_batch, s_bound, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def run_drift(G, ctx, w, M, K, beta, k, params=None, dense=True):
    d = to_dev(w)
    C, F = w.ncurves, w.nfreq
    idx = torch.empty(max(C * k, 1), dtype=torch.int32, device="cuda")
    S = torch.empty(max(C * k, 1), dtype=torch.float32, device="cuda")
    Sd = torch.empty(C * F, dtype=torch.float64, device="cuda") if dense else None
    G.fpw_periodogram_drift(ctx, None, params, d["offsets"], d["t"], d["x"], d["sigma"], d["freqs"], M, K, beta, k,
                            idx if k else None, S if k else None, Sd)
    torch.cuda.synchronize()
    st = ctx.status()
    return (idx.cpu().numpy()[:C * k].reshape(C, k), S.cpu().numpy()[:C * k].reshape(C, k),
            Sd.cpu().numpy().reshape(C, F) if dense else None, st)


CASES = [  # (ns, F, M, K, beta, inv_alpha2)
    ([0, 1, 40, 230, 300], 517, 20, 3, 1.0, 0.0),
    ([120, 250], 300, 7, 1, 2.0, 0.3),
    ([200, 64], 260, 12, 4, 0.5, 0.0),
    ([150], 129, 50, 2, 1.0, 1.0),
    ([90, 180], 400, 10, 0, 1.0, 0.0),
]


@pytest.mark.parametrize("ns,F,M,K,beta,ia2", CASES)
def test_drift_dense_and_topk_against_oracle(G, ctx, ns, F, M, K, beta, ia2):
    w = L.ragged(300 + M + K, ns, F, M=M, k=5)
    k = 5
    idx, Sk, Sd, st = run_drift(G, ctx, w, M, K, beta, k, params=G.fpw_params_default(inv_alpha2=ia2))
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, M, K, beta, ia2)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, M) <= 1e-9 if t.size else np.zeros(F, bool)
        assert_S_close(Sd[c], S_or, bound, mask=~near, what=f"drift M={M} K={K} curve {c} (n={t.size})")
        o_idx, o_S = oracle.topk(S_or, k + 4)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * max(bound, 1e-30), o_dense=S_or,
                   what=f"drift curve {c} peaks")


def test_drift_without_basis_matches_batched_path(G, ctx):
    w = L.ragged(310, [400, 150, 700], 2000, M=20, k=5)
    _, _, Sd, st = run_drift(G, ctx, w, 20, 0, 1.0, 0)
    assert st == 0
    _, _, Sb, st = run_batch(ctx, w, k=0, dense=True)
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        assert_S_close(Sd[c], Sb[c], s_bound(x, s), rel=2e-4, what=f"K=0 curve {c}")


def test_drift_invalid_curve_and_arguments(G, ctx):
    w = L.ragged(311, [60, 80, 50], 200, M=10, k=3)
    w.sigma = w.sigma.copy()
    w.sigma[w.offsets[1] + 3] = -1.0
    idx, Sk, Sd, st = run_drift(G, ctx, w, 10, 2, 1.0, 3)
    assert st == G.FPW_EDATA
    assert np.isnan(Sd[1]).all() and np.all(idx[1] == -1)
    for c in (0, 2):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, 10, 2, 1.0)
        assert_S_close(Sd[c], S_or, s_bound(x, s), mask=~(oracle.min_edge(t, w.freqs, 10) <= 1e-9),
                       what=f"neighbour {c}")
    with pytest.raises(G.FPWError) as ei:
        run_drift(G, ctx, w, 10, 5, 1.0, 3)
    assert ei.value.code == G.FPW_EINVAL
    with pytest.raises(G.FPWError) as ei:
        run_drift(G, ctx, w, 10, 2, 1.0, 3, params=G.fpw_params_default(accum=1))
    assert ei.value.code == G.FPW_ENOTSUP


def test_drift_ragged_10k_full_size_sampled(G, ctx):
    """All 10^4 curves of the ragged workload with K = 3 (beta = 1), top-5 per
    curve as the benchmark launches it; for sampled curves the oracle evaluates
    the reported peaks and their neighbours one frequency at a time."""
    w = L.make("ragged_10k")
    idx, Sk, _, st = run_drift(G, ctx, w, 20, 3, 1.0, 5, dense=False)
    assert st == 0
    sample = np.random.default_rng(12).choice(w.ncurves, 6, replace=False)
    for c in sample:
        t, x, s = w.curve(c)
        bound = s_bound(x, s)
        for j in range(5):
            fi = int(idx[c, j])
            assert 0 <= fi < w.nfreq
            nb = np.arange(max(fi - 1, 0), min(fi + 2, w.nfreq))
            So = oracle.fpw_drift(t, x, s, w.freqs[nb], 20, 3, 1.0)
            near = oracle.min_edge(t, w.freqs[nb], 20) <= 1e-9
            Sc = So[list(nb).index(fi)]
            if not near[list(nb).index(fi)]:
                assert abs(Sk[c, j] - Sc) <= 1e-4 * abs(Sc) + 1e-7 * bound, (c, j, Sk[c, j], Sc)
            # a local maximum of the oracle's periodogram up to the FP32 tolerance
            assert np.all(Sc >= So - (2e-4 * np.abs(So) + 2e-7 * bound)), (c, fi, So)
        assert np.all(np.diff(Sk[c]) <= 1e-4 * np.abs(Sk[c][:-1]) + 1e-7 * bound)  # ranked by S


def test_drift_zero_prior_width_is_eq1(G, ctx):
    """beta = 0 removes the baseline (C_B = 0): with K = 3 the statistic is Eq. 1,
    as the batched path computes it."""
    w = L.ragged(312, [350, 90, 600], 1500, M=20, k=5)
    _, _, Sd, st = run_drift(G, ctx, w, 20, 3, 0.0, 0)
    assert st == 0
    _, _, Sb, st = run_batch(ctx, w, k=0, dense=True)
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        assert_S_close(Sd[c], Sb[c], s_bound(x, s), rel=2e-4, what=f"beta=0 curve {c}")


@pytest.mark.parametrize("ia2", [2.0 ** 110, 1e-35])
def test_drift_extreme_inv_alpha2(G, ctx, ia2):
    """1/alpha^2 far outside the range where a bin's 1/L comes from the FP32
    reciprocal (above 2^100), and tiny: S against the dense oracle."""
    w = L.ragged(313, [120, 260], 300, M=10, k=3)
    _, _, Sd, st = run_drift(G, ctx, w, 10, 3, 1.0, 0, params=G.fpw_params_default(inv_alpha2=ia2))
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, 10, 3, 1.0, ia2)
        near = oracle.min_edge(t, w.freqs, 10) <= 1e-9
        assert_S_close(Sd[c], S_or, s_bound(x, s), mask=~near, what=f"ia2={ia2:g} curve {c}")


def test_drift_irregular_grid(G, ctx):
    """A grid that is not linear: every (observation, frequency) pair takes its
    exact anchor; a linear head and an irregular tail in one call."""
    w = L.ragged(314, [300, 45, 800], 700, M=16, k=4)
    rng = np.random.default_rng(5)
    w.freqs = np.concatenate([np.linspace(0.02, 5.0, 300), np.sort(rng.uniform(5.01, 35.0, 400))])
    idx, Sk, Sd, st = run_drift(G, ctx, w, 16, 3, 1.5, 4)
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, 16, 3, 1.5)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, 16) <= 1e-9
        assert_S_close(Sd[c], S_or, bound, mask=~near, what=f"irregular grid curve {c}")
        o_idx, o_S = oracle.topk(S_or, 8)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * bound, o_dense=S_or, what=f"irregular grid curve {c}")


def drifting(seed, ns, F, K):
    """Ragged curves with a polynomial baseline of ~100 noise sigmas added
    (degree K - 1 in the curve's scaled time, random coefficients)."""
    w = L.ragged(seed, ns, F, M=16, k=3)
    rng = np.random.default_rng([17, seed])
    x = w.x.copy()
    for c in range(w.ncurves):
        a, b = w.offsets[c], w.offsets[c + 1]
        t, s = w.t[a:b], w.sigma[a:b]
        tau = 2.0 * (t - t.min()) / np.ptp(t) - 1.0
        coef = rng.uniform(-1.0, 1.0, 3) * 100.0 * np.median(s)
        x[a:b] += coef[0] * tau + coef[1] * (2 * tau ** 2 - 1) + (coef[2] * (4 * tau ** 3 - 3 * tau) if K >= 4 else 0.0)
    w.x = x
    return w


@pytest.mark.parametrize("K,beta", [(2, 1.0), (3, 1.0), (4, 0.5)])
def test_drift_strong_baseline(G, ctx, K, beta):
    """A baseline ~100 noise sigmas tall, where marginalising it matters most.
    The bins sum the residuals of the curve's baseline fit, so the FP32 sums
    never carry the drift itself; the absolute floor is 1e-9 sum w x^2 (about
    1e-5 of the noise chi^2 here), far below what FP32 sums of w x would
    reach."""
    w = drifting(400 + K, [700, 1200, 90], 600, K)
    idx, Sk, Sd, st = run_drift(G, ctx, w, 16, K, beta, 3)
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, 16, K, beta)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, 16) <= 1e-9
        assert_S_close(Sd[c], S_or, bound, absf=1e-9, mask=~near, what=f"K={K} drifting curve {c}")
        o_idx, o_S = oracle.topk(S_or, 7)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-9 * bound, o_dense=S_or, what=f"K={K} drifting curve {c}")


@pytest.mark.parametrize("K,T,R", [(2, 64, 2), (3, 128, 2), (4, 32, 2), (3, 32, 1), (0, 128, 1), (1, 64, 2)])
def test_drift_block_shapes(G, ctx, K, T, R):
    """Every (threads, frequencies per thread) shape the drift call accepts,
    against the dense oracle; a frequency count that leaves a partial tile."""
    w = L.ragged(320 + K, [260, 33, 700], 611, M=14, k=4)
    p = G.fpw_params_default(threads=T, freqs_per_thread=R, inv_alpha2=0.2)
    idx, Sk, Sd, st = run_drift(G, ctx, w, 14, K, 0.8, 4, params=p)
    assert st == 0
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        S_or = oracle.fpw_drift(t, x, s, w.freqs, 14, K, 0.8, 0.2)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, 14) <= 1e-9
        assert_S_close(Sd[c], S_or, bound, mask=~near, what=f"K={K} T={T} R={R} curve {c}")
        o_idx, o_S = oracle.topk(S_or, 8)
        check_topk(idx[c], Sk[c], o_idx, o_S, abs_tol=1e-7 * bound, o_dense=S_or, what=f"K={K} T={T} R={R} curve {c}")


def test_drift_rejects_unsupported_shapes(G, ctx):
    """Valid parameters the drift kernel has no shape for give FPW_ENOTSUP;
    invalid ones (48 threads) FPW_EINVAL, as for every call."""
    w = L.ragged(330, [50], 64, M=8, k=2)
    for kw, code in (({"threads": 256}, G.FPW_ENOTSUP), ({"freqs_per_thread": 4}, G.FPW_ENOTSUP),
                     ({"threads": 48}, G.FPW_EINVAL)):
        with pytest.raises(G.FPWError) as ei:
            run_drift(G, ctx, w, 8, 2, 1.0, 2, params=G.fpw_params_default(**kw))
        assert ei.value.code == code, kw
