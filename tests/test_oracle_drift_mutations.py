"""Mutation check of the baseline-drift oracle's pins: plant one plausible
mistake at a time in a copy of `oracle/drift.py` (a dropped prior, an unscaled
or wrong basis, the drift left out of the covariance, unweighted projections,
stale bins), load the copy, and require that the pin battery below rejects
every mutant while accepting the original.

The battery holds the mutant against references that share no code with it:
the Appendix A.1 definition (a difference of two quadratic forms with full
covariance matrices) with the basis written as beta cos(k arccos tau) and the
bins of the C oracle; the Eq. 1 C oracle for K = 0 (empty bins included); the
basis itself; and the absorption of a polynomial baseline under a nearly flat
coefficient prior. CPU only."""
from __future__ import annotations

import os
import types

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "drift.py")

MUTATIONS = {
    "basis_not_scaled_by_beta": ("    return beta * Bm", "    return Bm"),
    "wrong_recurrence": ("Tkm1, Tk = Tk, 2.0 * tau * Tk - Tkm1", "Tkm1, Tk = Tk, tau * Tk - Tkm1"),
    "time_mapped_to_unit_interval": ("2.0 * (t - lo) / (hi - lo) - 1.0", "(t - lo) / (hi - lo)"),
    "drift_left_out_of_covariance": ("C = np.diag(sigma ** 2) + Bm @ Bm.T", "C = np.diag(sigma ** 2)"),
    "sigma_not_squared": ("C = np.diag(sigma ** 2) + Bm @ Bm.T", "C = np.diag(sigma) + Bm @ Bm.T"),
    "prior_term_dropped": ("T = inv_alpha2 * np.eye(E.shape[1]) + E.T @ W @ E", "T = E.T @ W @ E"),
    "alpha_squared_for_inverse": ("T = inv_alpha2 * np.eye(E.shape[1]) + E.T @ W @ E",
                                  "T = (1.0 / inv_alpha2 if inv_alpha2 else 0.0) * np.eye(E.shape[1]) + E.T @ W @ E"),
    "unweighted_projection": ("u = E.T @ Wx", "u = E.T @ x"),
    "bins_of_first_frequency": ("E[np.arange(n), b[q]] = 1.0", "E[np.arange(n), b[0]] = 1.0"),
    "empty_bins_kept": ("        if inv_alpha2 == 0.0:\n            E = E[:, E.sum(axis=0) > 0]\n", ""),
}


def load_drift(src: str):
    """The drift oracle module built from `src` (package `oracle`, so its
    relative import of the C bins resolves)."""
    mod = types.ModuleType("oracle._drift_under_test")
    mod.__package__ = "oracle"
    exec(compile(src, SRC, "exec"), mod.__dict__)
    return mod


def cos_basis(t, K, beta):
    t = np.asarray(t, dtype=np.float64)
    lo, hi = t.min(), t.max()
    tau = np.clip(2.0 * (t - lo) / (hi - lo) - 1.0, -1.0, 1.0)
    return beta * np.stack([np.cos(k * np.arccos(tau)) for k in range(K)], 1)


def a1_definition(t, x, sigma, f, M, K, beta, alpha):
    """Appendix A.1 before any identity: X^T (C_B + C_s)^-1 X - X^T (C_B + C_P + C_s)^-1 X."""
    n = t.size
    B = cos_basis(t, K, beta)
    b, _ = oracle.bins(t, [f], M, want_edge=False)
    P = np.zeros((n, M))
    P[np.arange(n), b[0]] = alpha
    C = np.diag(sigma ** 2) + B @ B.T
    return float(x @ np.linalg.solve(C, x) - x @ np.linalg.solve(C + P @ P.T, x))


def battery(mod) -> list[str]:
    """Names of the pins the module fails (an exception counts as a failure)."""
    failed = []
    rng = np.random.default_rng(2024)
    n = 36
    t = np.sort(rng.uniform(0.0, 300.0, n))
    sigma = np.exp(rng.uniform(np.log(0.05), np.log(0.3), n))
    x = 0.4 * np.sin(2 * np.pi * t / 3.7) + rng.normal(0, 1, n) * sigma
    freqs = np.array([0.0913, 0.27027, 0.5531, 1.3])

    def pin(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:  # a mutant that cannot even evaluate fails
            failed.append(name)

    # the A.1 definition, finite alpha of 0.8 and 2.0 (1/alpha^2 != 1)
    def a1():
        for K, beta, alpha in ((2, 1.3, 0.8), (3, 0.7, 2.0)):
            S = mod.fpw_drift(t, x, sigma, freqs, 6, K, beta, 1.0 / alpha ** 2)
            ref = [a1_definition(t, x, sigma, f, 6, K, beta, alpha) for f in freqs]
            if not np.allclose(S, ref, rtol=1e-8, atol=1e-10):
                return False
        return True
    pin("appendix_a1", a1)

    # K = 0 is Eq. 1 (the C oracle), with empty bins at M = 40 and 1/alpha^2 = 0
    def eq1():
        for M, ia2 in ((40, 0.0), (6, 0.5)):
            if not np.allclose(mod.fpw_drift(t, x, sigma, freqs, M, 0, 1.0, ia2), oracle.fpw(t, x, sigma, freqs, M, ia2),
                               rtol=1e-9, atol=1e-12):
                return False
        return True
    pin("eq1_without_basis", eq1)

    # the basis: beta T_k(tau) = beta cos(k arccos tau)
    pin("basis", lambda: np.allclose(mod.chebyshev_basis(t, 4, 1.7), cos_basis(t, 4, 1.7), atol=1e-12))

    # a polynomial baseline of degree < K is absorbed under a nearly flat prior
    def absorbed():
        tau = 2.0 * (t - t.min()) / np.ptp(t) - 1.0
        xd = x + 5.0 * tau - 3.0 * tau ** 2
        S0 = mod.fpw_drift(t, x, sigma, freqs, 6, 3, 1e4)
        S1 = mod.fpw_drift(t, xd, sigma, freqs, 6, 3, 1e4)
        return np.allclose(S0, S1, rtol=1e-4, atol=1e-6)
    pin("baseline_absorbed", absorbed)
    return failed


def test_battery_accepts_the_oracle():
    with open(SRC) as fh:
        src = fh.read()
    assert battery(load_drift(src)) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_battery_rejects_mutant(name):
    old, new = MUTATIONS[name]
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    failed = battery(load_drift(src.replace(old, new)))
    assert failed, f"mutant {name} passes every pin"
