"""Pins for the FP64 oracle, each against something other than the oracle's own
formula: a hand-worked example, the dense matrix forms of Appendix A, the
least-squares (piecewise-constant fit) form, exact rational bin assignment,
closed forms, invariants, the null distribution and signal recovery.

Runs on CPU only (no GPU, no CUDA library)."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import lightcurves as L
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def exact_bins(t, f, M):
    """Appendix A.1 bins in exact rational arithmetic, plus the exact distance
    (cycles) of t*f to the nearest bin edge."""
    out, dist = [], []
    for ti in t:
        p = Fraction(float(ti)) * Fraction(float(f))
        fr = p - math.floor(p)
        y = fr * M
        out.append(int(math.floor(y)))
        r = y - round(y)
        dist.append(abs(float(r)) / M)
    return np.array(out), np.array(dist)


def one_hot(bins, M):
    P = np.zeros((len(bins), M))
    P[np.arange(len(bins)), bins] = 1.0
    return P


def dense_chi2_difference(x, sigma, bins, M, alpha):
    """Appendix A.3: S = X^T C^-1 X - X^T (C + C_P)^-1 X with C = diag(sigma^2) and
    C_P = P P^T, P = alpha * one-hot bin matrix (solved densely)."""
    C = np.diag(sigma ** 2)
    P = alpha * one_hot(bins, M)
    return float(x @ np.linalg.solve(C, x) - x @ np.linalg.solve(C + P @ P.T, x))


def dense_woodbury(x, sigma, bins, M, alpha):
    """Appendix A.3 after Sherman-Morrison: X^T C^-1 P (I + P^T C^-1 P)^-1 P^T C^-1 X."""
    Ci = np.diag(1.0 / sigma ** 2)
    P = alpha * one_hot(bins, M)
    u = P.T @ Ci @ x
    return float(u @ np.linalg.solve(np.eye(M) + P.T @ Ci @ P, u))


def least_squares_reduction(x, sigma, bins, M):
    """Appendix B basis (alpha -> infinity): chi^2 of the zero model minus chi^2 of
    the best piecewise-constant (per-bin weighted mean) model."""
    w = 1.0 / sigma ** 2
    chi0 = float(np.sum(w * x * x))
    chi1 = 0.0
    for m in range(M):
        sel = bins == m
        if not np.any(sel):
            continue
        mean = np.sum(w[sel] * x[sel]) / np.sum(w[sel])
        chi1 += float(np.sum(w[sel] * (x[sel] - mean) ** 2))
    return chi0 - chi1


def tiny_case(rng, n, negative_t=False):
    lo = -40.0 if negative_t else 0.0
    t = rng.uniform(lo, 40.0, n)
    x = rng.normal(0, 1, n)
    sigma = rng.uniform(0.3, 2.0, n)
    return t, x, sigma


# ---------------------------------------------------------------- hand example
def test_hand_worked_example():
    t = np.array([0, 0.1, 0.35, 0.6, 0.85, 1.2])
    x = np.array([1, 2, -1, 0.5, -3, 1.0])
    sigma = np.array([1, 0.5, 1, 2, 1, 0.5])
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "hand_example.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 4
    for f, c, num, den in rows:
        S = oracle.fpw(t, x, sigma, [float(f)], 4, float(c))[0]
        assert S == pytest.approx(int(num) / int(den), rel=1e-14), (f, c)


# ---------------------------------------------------------------- dense forms
@pytest.mark.parametrize("seed", range(12))
def test_dense_appendix_forms(seed):
    rng = np.random.default_rng([7, seed])
    n = int(rng.integers(1, 13))
    M = int(rng.choice([2, 3, 5]))
    t, x, sigma = tiny_case(rng, n, negative_t=(seed % 3 == 0))
    freqs = rng.uniform(0.05, 3.0, 4)
    for alpha in (0.5, 1.0, 3.0):
        S = oracle.fpw(t, x, sigma, freqs, M, 1.0 / alpha ** 2)
        for q, f in enumerate(freqs):
            b, _ = exact_bins(t, f, M)
            s1 = dense_chi2_difference(x, sigma, b, M, alpha)
            s2 = dense_woodbury(x, sigma, b, M, alpha)
            assert s1 == pytest.approx(s2, rel=1e-9, abs=1e-12)
            assert S[q] == pytest.approx(s1, rel=1e-9, abs=1e-12), (seed, alpha, f)


@pytest.mark.parametrize("seed", range(12))
def test_least_squares_form(seed):
    rng = np.random.default_rng([8, seed])
    n = int(rng.integers(1, 13))
    M = int(rng.choice([1, 2, 4, 5]))
    t, x, sigma = tiny_case(rng, n, negative_t=(seed % 2 == 0))
    freqs = rng.uniform(0.05, 3.0, 5)
    S = oracle.fpw(t, x, sigma, freqs, M, 0.0)
    for q, f in enumerate(freqs):
        b, _ = exact_bins(t, f, M)
        assert S[q] == pytest.approx(least_squares_reduction(x, sigma, b, M), rel=1e-9, abs=1e-10)


# ---------------------------------------------------------------- bins
@pytest.mark.parametrize("seed", range(6))
def test_bins_match_exact_rationals(seed):
    rng = np.random.default_rng([9, seed])
    t = np.concatenate([rng.uniform(0, 2000, 40), rng.uniform(-50, 0, 5)])
    freqs = np.concatenate([rng.uniform(0.01, 500, 6), [0.0]])
    M = int(rng.choice([3, 10, 20, 50]))
    b, e = oracle.bins(t, freqs, M)
    for q, f in enumerate(freqs):
        eb, ed = exact_bins(t, f, M)
        np.testing.assert_allclose(e[q], ed, rtol=0, atol=1e-15)
        far = ed > 1e-12
        np.testing.assert_array_equal(b[q][far], eb[far])
        assert np.all((b[q] >= 0) & (b[q] < M))


def test_bins_edges_half_open_and_clamp():
    # phase exactly on an edge belongs to the upper bin; phase just below 1 stays in bin M-1
    t = np.array([0.25, 0.5, 0.0, 1.0 - 2.0 ** -53, 3.0])
    b, e = oracle.bins(t, [1.0], 4)
    assert list(b[0]) == [1, 2, 0, 3, 0]
    assert e[0][0] == 0.0 and e[0][1] == 0.0 and e[0][2] == 0.0
    assert e[0][3] == pytest.approx(2.0 ** -53, rel=1e-12)


# ---------------------------------------------------------------- closed forms
def _curve(seed=0, n=300):
    w = L.ragged(seed, [n], 10)
    return w.curve(0)


def test_M1_and_zero_frequency_closed_form():
    t, x, sigma = _curve(1)
    rng = np.random.default_rng(3)
    xs = x + rng.normal(0, 0.3)  # not mean-subtracted
    w = 1 / sigma ** 2
    for c in (0.0, 0.7):
        want = np.sum(w * xs) ** 2 / (np.sum(w) + c)
        S1 = oracle.fpw(t, xs, sigma, rng.uniform(0.01, 50, 20), 1, c)
        np.testing.assert_allclose(S1, want, rtol=1e-12)
        for M in (2, 7, 20):
            S0 = oracle.fpw(t, xs, sigma, [0.0], M, c)
            assert S0[0] == pytest.approx(want, rel=1e-12)


def test_weighted_mean_subtracted_gives_zero_at_M1():
    t, x, sigma = _curve(2)  # generator subtracts the inverse-variance weighted mean
    S = oracle.fpw(t, x, sigma, np.linspace(0.01, 10, 50), 1, 0.0)
    scale = np.sum(x * x / sigma ** 2)
    assert np.max(np.abs(S)) < 1e-20 * max(scale, 1.0) + 1e-18


# ---------------------------------------------------------------- invariants
def test_permutation_invariance():
    t, x, sigma = _curve(3, 500)
    freqs = np.linspace(0.01, 20, 400)
    S = oracle.fpw(t, x, sigma, freqs, 20, 0.0)
    p = np.random.default_rng(4).permutation(t.shape[0])
    Sp = oracle.fpw(t[p], x[p], sigma[p], freqs, 20, 0.0)
    np.testing.assert_allclose(Sp, S, rtol=1e-11, atol=1e-12)


def test_sign_and_scale_invariance():
    t, x, sigma = _curve(5, 400)
    freqs = np.linspace(0.01, 20, 300)
    S = oracle.fpw(t, x, sigma, freqs, 10, 0.25)
    np.testing.assert_array_equal(oracle.fpw(t, -x, sigma, freqs, 10, 0.25), S)
    lam = 3.7
    Sl = oracle.fpw(t, lam * x, lam * sigma, freqs, 10, 0.25 / lam ** 2)
    np.testing.assert_allclose(Sl, S, rtol=1e-12)


def test_bounds():
    t, x, sigma = _curve(6, 700)
    freqs = np.linspace(0.01, 40, 2000)
    ub = np.sum(x * x / sigma ** 2)
    for c in (0.0, 1.0):
        S = oracle.fpw(t, x, sigma, freqs, 20, c)
        assert np.all(S >= 0.0)
        assert np.all(S <= ub * (1 + 1e-12))


def test_integer_time_alias_exact():
    rng = np.random.default_rng(7)
    t = np.sort(rng.integers(0, 1000, 300)).astype(np.float64)
    x = rng.normal(0, 1, 300)
    sigma = rng.uniform(0.5, 2, 300)
    f = np.arange(1, 200) / 1024.0 + 1.0 / 4096.0  # dyadic: every t*f is exact
    S = oracle.fpw(t, x, sigma, f, 10, 0.0)
    S1 = oracle.fpw(t, x, sigma, f + 1.0, 10, 0.0)
    S3 = oracle.fpw(t, x, sigma, f + 3.0, 10, 0.0)
    np.testing.assert_array_equal(S1, S)
    np.testing.assert_array_equal(S3, S)


def test_negative_frequency_mirrors_bins():
    rng = np.random.default_rng(8)
    t = np.sort(rng.uniform(0, 500, 250))
    x = rng.normal(0, 1, 250)
    sigma = rng.uniform(0.5, 2, 250)
    freqs = rng.uniform(0.1, 10, 100)
    _, e = oracle.bins(t, freqs, 10)
    keep = np.all(e > 1e-9, axis=1)  # off-edge frequencies: bin m -> M-1-m exactly
    assert keep.sum() > 50
    np.testing.assert_allclose(oracle.fpw(t, x, sigma, -freqs[keep], 10, 0.0),
                               oracle.fpw(t, x, sigma, freqs[keep], 10, 0.0), rtol=1e-13)
    b, _ = oracle.bins(t, freqs[keep], 10)
    bn, _ = oracle.bins(t, -freqs[keep], 10)
    np.testing.assert_array_equal(bn, 9 - b)


# ---------------------------------------------------------------- statistics
def test_null_distribution_is_chi2_M_minus_1():
    """Pure Gaussian noise with the true sigma, weighted-mean subtracted, 1/alpha^2 = 0:
    S ~ chi^2 with M-1 degrees of freedom (Section 3.2 / Appendix B DOF), so the
    mean is M-1 and the variance 2(M-1)."""
    M, n, C = 5, 120, 3000
    rng = np.random.default_rng(11)
    vals = []
    for c in range(C):
        t = rng.uniform(0, 300, n)
        sigma = rng.uniform(0.2, 3.0, n)
        x = rng.normal(0, 1, n) * sigma
        w = 1 / sigma ** 2
        x = x - np.sum(w * x) / np.sum(w)
        vals.append(oracle.fpw(t, x, sigma, [rng.uniform(0.5, 5.0)], M, 0.0)[0])
    vals = np.array(vals)
    se = math.sqrt(2 * (M - 1) / C)
    assert abs(vals.mean() - (M - 1)) < 5 * se
    assert abs(vals.var() - 2 * (M - 1)) < 0.15 * 2 * (M - 1)


# ---------------------------------------------------------------- recovery
def test_sinusoid_recovered_on_dense_local_grid():
    w = L.make("single_plain")
    t, x, sigma = w.curve(0)
    f0 = 1 / 0.37
    T = t.max() - t.min()
    grid = f0 + np.linspace(-20 / T, 20 / T, 801)  # 0.05/T spacing
    S = oracle.fpw(t, x, sigma, grid, 10, 0.0)
    assert abs(grid[np.argmax(S)] - f0) < 1 / T
    # and the wide-band maximum sits near f0 as well
    wide = np.linspace(0.05, 10, 40001)
    Sw = oracle.fpw(t, x, sigma, wide, 10, 0.0)
    assert abs(wide[np.argmax(Sw)] - f0) < 2 / T


def test_eclipse_recovered_at_fundamental_or_subharmonic():
    w = L.make("single_ztf")
    t, x, sigma = w.curve(0)
    f0 = 1 / 0.8123
    T = t.max() - t.min()
    grid = np.linspace(0.2, 3.0, 120001)
    S = oracle.fpw(t, x, sigma, grid, 20, 0.0)
    idx, _ = oracle.topk(S, 5)
    best = grid[idx[0]]
    ok = [abs(best - f0 / h) < 2 / T for h in range(1, 11)]
    assert any(ok), best


# ---------------------------------------------------------------- top-k
def test_topk_peaks_golden():
    S = np.array([1.0, 3.0, 2.0, 5.0, 5.0, 4.0, 6.0])
    idx, val = oracle.topk(S, 3)
    assert list(idx) == [6, 3, 1] and list(val) == [6.0, 5.0, 3.0]
    # raw mode ranks every entry, ties to the lower index
    idx, val = oracle.topk(S, 4, raw=True)
    assert list(idx) == [6, 3, 4, 5]
    # grid ends are one-sided; a plateau's first element is the peak
    idx, _ = oracle.topk(np.array([4.0, 4.0, 1.0, 2.0, 2.0]), 5)
    assert list(idx) == [0, 3, -1, -1, -1]
    # more requested than peaks: -1 / NaN
    idx, val = oracle.topk(np.array([1.0, 2.0, 3.0]), 3)
    assert list(idx) == [2, -1, -1] and np.isnan(val[1:]).all()
    idx, val = oracle.topk(np.array([7.0]), 2)
    assert list(idx) == [0, -1]
    # equal peaks: lower index first
    idx, _ = oracle.topk(np.array([0.0, 2.0, 0.0, 2.0, 0.0, 2.0]), 3)
    assert list(idx) == [1, 3, 5]


def test_topk_matches_sorting_brute_force():
    rng = np.random.default_rng(12)
    for _ in range(50):
        F = int(rng.integers(1, 60))
        S = np.round(rng.uniform(0, 5, F), 1)  # many ties
        k = int(rng.integers(1, 8))
        peaks = [q for q in range(F)
                 if (F == 1) or (q == 0 and S[0] >= S[1]) or (q == F - 1 and S[q] > S[q - 1])
                 or (0 < q < F - 1 and S[q] > S[q - 1] and S[q] >= S[q + 1])]
        want = sorted(peaks, key=lambda q: (-S[q], q))[:k]
        idx, _ = oracle.topk(S, k)
        assert list(idx[:len(want)]) == want and all(i == -1 for i in idx[len(want):])


# ---------------------------------------------------------------- batch & errors
def test_batch_matches_single_curve_calls():
    w = L.ragged(21, [0, 1, 5, 64, 200, 33], 700)
    S, idx, val = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 10, 0.5, nthreads=3, k=4)
    for c in range(w.ncurves):
        t, x, sigma = w.curve(c)
        Sc = oracle.fpw(t, x, sigma, w.freqs, 10, 0.5)
        np.testing.assert_array_equal(S[c], Sc)
        i2, v2 = oracle.topk(Sc, 4)
        np.testing.assert_array_equal(idx[c], i2)
        np.testing.assert_array_equal(val[c], v2)
    assert np.all(S[0] == 0.0)
    _, idx2, _ = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 10, 0.5, nthreads=2, dense=False, k=4)
    np.testing.assert_array_equal(idx2, idx)


def test_invalid_inputs_rejected():
    t = np.array([0.0, 1.0, 2.0])
    x = np.array([1.0, -1.0, 0.0])
    with pytest.raises(oracle.OracleError):
        oracle.fpw(t, x, np.array([1.0, 0.0, 1.0]), [1.0], 4)
    with pytest.raises(oracle.OracleError):
        oracle.fpw(t, x, np.array([1.0, -1.0, 1.0]), [1.0], 4)
    with pytest.raises(oracle.OracleError):
        oracle.fpw(np.array([0.0, np.nan, 1.0]), x, np.ones(3), [1.0], 4)
    with pytest.raises(oracle.OracleError):
        oracle.fpw(t, x, np.ones(3), [1.0], 0)
    assert oracle.fpw(np.zeros(0), np.zeros(0), np.zeros(0), [1.0, 2.0], 4).tolist() == [0.0, 0.0]


# ---------------------------------------------------------------- several M from one M_max pass (Section 3.4)
def exact_phase(t, f):
    p = Fraction(float(t)) * Fraction(float(f))
    return p - math.floor(p)


@pytest.mark.parametrize("seed", range(6))
def test_multi_m_offsets_match_shifted_bins_least_squares(seed):
    """Offset o of M = M_max/g is the plain statistic with bin edges shifted by
    o/M_max cycles: bins floor(M * frac(phase - o/M_max)) from exact rationals,
    S from the least-squares form."""
    rng = np.random.default_rng([23, seed])
    n = int(rng.integers(3, 14))
    M_max, g = [(12, 3), (12, 4), (20, 5), (20, 2), (6, 6), (8, 1)][seed]
    t, x, sigma = tiny_case(rng, n, negative_t=(seed % 2 == 1))
    freqs = rng.uniform(0.05, 3.0, 3)
    S = oracle.fpw_multi(t, x, sigma, freqs, M_max, g)
    M = M_max // g
    for q, f in enumerate(freqs):
        for o in range(g):
            bins = []
            for ti in t:
                ph = exact_phase(ti, f) - Fraction(o, M_max)
                ph -= math.floor(ph)
                bins.append(int(math.floor(ph * M)))
            assert S[o, q] == pytest.approx(least_squares_reduction(x, sigma, np.array(bins), M), rel=1e-9, abs=1e-10)


def test_multi_m_reduces_to_plain_statistic():
    t, x, sigma = _curve(8, 400)
    freqs = np.linspace(0.01, 20, 500)
    _, e = oracle.bins(t, freqs, 20)
    keep = np.all(e > 1e-12, axis=1)
    np.testing.assert_array_equal(oracle.fpw_multi(t, x, sigma, freqs, 20, 1)[0], oracle.fpw(t, x, sigma, freqs, 20))
    # offset 0 of M = 20/4 = 5 is the plain 5-bin statistic (away from rounding at the edges)
    np.testing.assert_allclose(oracle.fpw_multi(t, x, sigma, freqs, 20, 4)[0][keep],
                               oracle.fpw(t, x, sigma, freqs, 5)[keep], rtol=1e-12)
    # with the prior term as well
    np.testing.assert_allclose(oracle.fpw_multi(t, x, sigma, freqs, 20, 2, 0.4)[0][keep],
                               oracle.fpw(t, x, sigma, freqs, 10, 0.4)[keep], rtol=1e-12)


# ---------------------------------------------------------------- phase entropy (Appendix C)
def hutcheson(M, N):
    """Appendix C: expectation and variance of the phase entropy for equal bin
    probabilities, to the orders the paper gives."""
    E = math.log(M) - (M - 1) / (2 * N) - (M - 1) * (M + 1) / (12 * N * N)
    V = (M - 1) / (2 * N * N) + (M * M - 1) / (6 * N ** 3)
    return E, V


def test_phase_entropy_closed_forms():
    M, per = 8, 5
    N = M * per
    # phases i/N at f = 1: exactly `per` observations per bin -> H = log M
    t = np.arange(N) / N
    assert oracle.phase_entropy(t, [1.0], M)[0] == pytest.approx(math.log(M), rel=1e-15)
    # every observation in one bin -> H = 0 (f = 0, or integer times at integer f)
    assert oracle.phase_entropy(t, [0.0], M)[0] == 0.0
    assert oracle.phase_entropy(np.arange(30.0), [3.0], M)[0] == 0.0
    # two equally filled bins -> log 2; a 1:3 split -> -(1/4 log 1/4 + 3/4 log 3/4)
    assert oracle.phase_entropy(np.array([0.0, 0.5]), [1.0], 2)[0] == pytest.approx(math.log(2))
    h = oracle.phase_entropy(np.array([0.1, 0.6, 0.7, 0.8]), [1.0], 2)[0]
    assert h == pytest.approx(-(0.25 * math.log(0.25) + 0.75 * math.log(0.75)))
    assert oracle.phase_entropy(np.zeros(0), [1.0], M)[0] == 0.0


def test_phase_entropy_matches_hutcheson_for_random_times():
    M, N, C = 10, 200, 400
    rng = np.random.default_rng(31)
    vals = [oracle.phase_entropy(rng.uniform(0, 1000, N), [rng.uniform(1.0, 5.0)], M)[0] for _ in range(C)]
    E, V = hutcheson(M, N)
    vals = np.array(vals)
    assert abs(vals.mean() - E) < 5 * math.sqrt(V / C)
    assert abs(vals.var() / V - 1.0) < 0.3


def test_phase_entropy_ignores_order_and_fluxes():
    t, x, sigma = _curve(9, 300)
    f = np.linspace(0.05, 5, 200)
    H = oracle.phase_entropy(t, f, 20)
    np.testing.assert_allclose(oracle.phase_entropy(t[::-1].copy(), f, 20), H, rtol=1e-13)
    assert np.all(H >= 0) and np.all(H <= math.log(20) + 1e-12)


# ---------------------------------------------------------------- shared-timestamp batch (Section 4, Appendix D)
@pytest.mark.parametrize("seed", range(6))
def test_shared_batch_dense_form_with_one_bin_matrix(seed):
    """All curves use one exact bin matrix per frequency: the dense Appendix A.3
    form per curve with that shared matrix."""
    rng = np.random.default_rng([31, seed])
    n, C, M, alpha = int(rng.integers(1, 11)), 3, int(rng.choice([2, 3, 4])), 1.5
    t = rng.uniform(-20.0 if seed % 2 else 0.0, 20.0, n)
    x = rng.normal(0, 1, (C, n))
    sigma = rng.uniform(0.3, 2.0, (C, n))
    freqs = rng.uniform(0.05, 3.0, 3)
    S = oracle.fpw_shared(t, x, sigma, freqs, M, 1.0 / alpha ** 2)
    for q, f in enumerate(freqs):
        b, _ = exact_bins(t, f, M)
        for c in range(C):
            assert S[c, q] == pytest.approx(dense_chi2_difference(x[c], sigma[c], b, M, alpha), rel=1e-9, abs=1e-12)


def test_shared_batch_equals_single_curve_oracle_and_permutes_rows():
    w = L.make("single_ztf", nfreq=3000)
    t = w.t
    rng = np.random.default_rng(5)
    C = 5
    x = np.stack([w.x] + [rng.normal(0, 0.1, t.size) for _ in range(C - 1)])
    sigma = np.stack([w.sigma] + [rng.uniform(0.02, 0.2, t.size) for _ in range(C - 1)])
    S = oracle.fpw_shared(t, x, sigma, w.freqs, 20)
    for c in range(C):  # same arithmetic in the same order per curve: bitwise equal
        np.testing.assert_array_equal(S[c], oracle.fpw(t, x[c], sigma[c], w.freqs, 20))
    perm = rng.permutation(C)
    np.testing.assert_array_equal(oracle.fpw_shared(t, x[perm], sigma[perm], w.freqs, 20), S[perm])
    # a curve with invalid data gives a NaN row and leaves the others unchanged
    sigma_bad = sigma.copy()
    sigma_bad[2, 7] = 0.0
    S_bad = oracle.fpw_shared(t, x, sigma_bad, w.freqs, 20)
    assert np.isnan(S_bad[2]).all()
    np.testing.assert_array_equal(S_bad[[0, 1, 3, 4]], S[[0, 1, 3, 4]])
    with pytest.raises(oracle.OracleError):
        oracle.fpw_shared(np.array([0.0, np.inf]), np.zeros((1, 2)), np.ones((1, 2)), w.freqs[:3], 4)


# ---------------------------------------------------------------- baseline drift marginalised (Appendix A.1-A.2)
def test_drift_chebyshev_basis_is_cos_k_theta():
    theta = np.linspace(0.1, 3.0, 9)
    t = np.cos(theta)  # tau = t after the span map when the span is exactly [-1, 1]
    t = np.concatenate([[-1.0], t, [1.0]])
    Bm = oracle.chebyshev_basis(t, 5, 2.0)
    tau = 2.0 * (t + 1.0) / 2.0 - 1.0
    for k in range(5):
        np.testing.assert_allclose(Bm[:, k], 2.0 * np.cos(k * np.arccos(tau)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_drift_sherman_morrison_equals_chi2_difference(seed):
    """The dense A.2 form against the A.1 definition (difference of two quadratic
    forms with full covariance matrices), for finite alpha."""
    rng = np.random.default_rng([41, seed])
    n, M, K = int(rng.integers(4, 25)), int(rng.choice([2, 3, 5])), int(rng.integers(1, 4))
    t = np.sort(rng.uniform(0.0, 200.0, n))
    sigma = rng.uniform(0.2, 1.0, n)
    x = rng.normal(0, 1, n)
    alpha, beta = float(rng.uniform(0.5, 3.0)), float(rng.uniform(0.3, 5.0))
    freqs = rng.uniform(0.05, 2.0, 3)
    S = oracle.fpw_drift(t, x, sigma, freqs, M, K, beta, 1.0 / alpha ** 2)
    for q, f in enumerate(freqs):
        assert S[q] == pytest.approx(oracle.fpw_drift_chi2_difference(t, x, sigma, f, M, K, beta, alpha),
                                     rel=1e-9, abs=1e-12)


def test_drift_reduces_to_eq1_without_baseline_and_as_beta_vanishes():
    w = L.make("single_plain", nfreq=400)
    t, x, s = w.curve(0)
    S1 = oracle.fpw(t, x, s, w.freqs, 10)
    np.testing.assert_allclose(oracle.fpw_drift(t, x, s, w.freqs, 10, 0, 1.0), S1, rtol=1e-10)
    np.testing.assert_allclose(oracle.fpw_drift(t, x, s, w.freqs, 10, 3, 1e-7), S1, rtol=1e-8)
    S1a = oracle.fpw(t, x, s, w.freqs, 10, 0.3)
    np.testing.assert_allclose(oracle.fpw_drift(t, x, s, w.freqs, 10, 2, 1e-7, 0.3), S1a, rtol=1e-8)


def test_drift_absorbs_a_polynomial_baseline_as_beta_grows():
    """With a nearly flat prior on the baseline coefficients, adding a polynomial
    of degree < K (in the mapped time) to the fluxes leaves S unchanged."""
    rng = np.random.default_rng(44)
    n = 60
    t = np.sort(rng.uniform(0.0, 500.0, n))
    sigma = rng.uniform(0.1, 0.3, n)
    x = 0.4 * np.sin(2 * np.pi * t / 0.731) + rng.normal(0, 1, n) * sigma
    tau = 2.0 * (t - t.min()) / (t.max() - t.min()) - 1.0
    drift = 3.0 + 2.0 * tau - 1.5 * (2 * tau ** 2 - 1)
    freqs = np.linspace(0.5, 3.0, 40)
    for K in (1, 2, 3):
        d = np.polynomial.chebyshev.chebval(tau, [3.0, 2.0, -1.5][:K])
        S0 = oracle.fpw_drift(t, x, sigma, freqs, 8, K, 1e5, 1.0)
        Sd = oracle.fpw_drift(t, x + d, sigma, freqs, 8, K, 1e5, 1.0)
        np.testing.assert_allclose(Sd, S0, rtol=1e-6)
    # without the baseline term the same trend changes S a lot
    assert np.max(np.abs(oracle.fpw(t, x + drift, sigma, freqs, 8, 1.0) - oracle.fpw(t, x, sigma, freqs, 8, 1.0))) > 1.0


def test_drift_ignores_observation_order():
    rng = np.random.default_rng(45)
    n = 30
    t = rng.uniform(0.0, 100.0, n)
    sigma = rng.uniform(0.2, 0.6, n)
    x = rng.normal(0, 1, n)
    f = np.linspace(0.1, 1.0, 20)
    p = rng.permutation(n)
    np.testing.assert_allclose(oracle.fpw_drift(t[p], x[p], sigma[p], f, 6, 3, 2.0),
                               oracle.fpw_drift(t, x, sigma, f, 6, 3, 2.0), rtol=1e-10)
