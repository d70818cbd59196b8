"""FPW with the baseline drift marginalised (Appendix A.1-A.2): a plain, slow,
dense binary64 implementation. TEST INFRASTRUCTURE ONLY (see the package
docstring): nothing in the product path may import it.

Model (Appendix A.1): x = B c + y_m(i,f) + noise, with
  * C_sigma = diag(sigma_i^2),
  * C_B = B B^T, B[i, k] = beta * T_k(tau_i), k = 0..K-1, Chebyshev polynomials
    of the first kind (the appendix names a Chebyshev basis) in the time mapped
    to [-1, 1] over the curve's span, tau_i = 2 (t_i - t_min) / (t_max - t_min) - 1
    (tau = 0 when all times are equal); beta is the prior standard deviation of
    each coefficient;
  * C_P = P P^T, P = alpha * E, E the one-hot bin matrix (Appendix A.1 bins).

Statistic (Appendix A.2, Sherman-Morrison form; reported with the sign that
makes it the Eq. 1 statistic when C_B = 0):

    S = X^T W P (I + P^T W P)^-1 P^T W X,   W = (C_B + C_sigma)^-1
      = u^T (I / alpha^2 + E^T W E)^-1 u,   u = E^T W X.

With 1/alpha^2 = 0 the bins that hold no observation are dropped (their rows
and columns of E^T W E vanish; the limit alpha -> infinity of the expression).
Everything is formed densely (N x N inverse once per curve, an M x M solve per
frequency), in the order the appendix states it.
"""
from __future__ import annotations

import numpy as np

from . import bins as _bins


def chebyshev_basis(t, K: int, beta: float) -> np.ndarray:
    """B[i, k] = beta * T_k(tau_i), k < K (Appendix A.1's polynomial baseline)."""
    t = np.asarray(t, dtype=np.float64)
    n = t.shape[0]
    Bm = np.zeros((n, K))
    if n == 0 or K == 0:
        return Bm
    lo, hi = float(t.min()), float(t.max())
    tau = np.zeros(n) if hi == lo else 2.0 * (t - lo) / (hi - lo) - 1.0
    Tkm1, Tk = np.ones(n), tau
    for k in range(K):
        if k == 0:
            Bm[:, 0] = 1.0
        elif k == 1:
            Bm[:, 1] = tau
        else:
            Tkm1, Tk = Tk, 2.0 * tau * Tk - Tkm1
            Bm[:, k] = Tk
    return beta * Bm


def fpw_drift(t, x, sigma, freqs, M: int, K: int, beta: float, inv_alpha2: float = 0.0) -> np.ndarray:
    """S at every trial frequency for one curve (dense Appendix A.2 form)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    freqs = np.asarray(freqs, dtype=np.float64)
    n = t.shape[0]
    S = np.zeros(freqs.shape[0])
    if n == 0:
        return S
    Bm = chebyshev_basis(t, K, beta)
    C = np.diag(sigma ** 2) + Bm @ Bm.T          # C_B + C_sigma
    W = np.linalg.inv(C)
    Wx = W @ x
    b, _ = _bins(t, freqs, M, want_edge=False)   # [F, n], Appendix A.1 bins (binary64 fl(t f))
    for q in range(freqs.shape[0]):
        E = np.zeros((n, M))
        E[np.arange(n), b[q]] = 1.0
        if inv_alpha2 == 0.0:
            E = E[:, E.sum(axis=0) > 0]
        u = E.T @ Wx
        T = inv_alpha2 * np.eye(E.shape[1]) + E.T @ W @ E
        S[q] = float(u @ np.linalg.solve(T, u))
    return S


def fpw_drift_chi2_difference(t, x, sigma, f: float, M: int, K: int, beta: float, alpha: float) -> float:
    """The Appendix A.1 definition before any identity is applied:
    X^T (C_B + C_sigma)^-1 X - X^T (C_B + C_P + C_sigma)^-1 X, for one frequency."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = t.shape[0]
    Bm = chebyshev_basis(t, K, beta)
    b, _ = _bins(t, [f], M, want_edge=False)
    P = np.zeros((n, M))
    P[np.arange(n), b[0]] = alpha
    Cb = np.diag(np.asarray(sigma, dtype=np.float64) ** 2) + Bm @ Bm.T
    return float(x @ np.linalg.solve(Cb, x) - x @ np.linalg.solve(Cb + P @ P.T, x))
