"""FPW oracle: plain FP64 CPU implementation of Eq. 1 (Section 2) of
Finkbeiner, Prince & Whitebook, "A Fast Periodicity Detection Algorithm
Sensitive to Arbitrary Waveforms" (arXiv:2502.00243).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package. It shares
no code with the CUDA library under ``paper_2502_00243_gb300/`` and never
imports it.

The arithmetic lives in ``fpw_oracle.c`` (binary64, built with
``-ffp-contract=off`` so every operation rounds exactly as written on x86 and
Arm alike). This module only compiles it with the system C compiler and
marshals numpy arrays through ctypes.

Functions and the passages they follow:

* :func:`fpw` -- Eq. 1 for one light curve at every trial frequency, bins from
  Appendix A.1 (m = floor(M * frac(t f)), t_ref = 0), sums from Appendix A.4.
* :func:`fpw_batch` -- the same for a ragged batch (CSR offsets), threads over
  curves, optional dense S and per-curve top-k peaks (Section 3.5
  post-processing).
* :func:`fpw_multi` -- Section 3.4: S for M = M_max / g from the M_max-bin sums,
  for each of the g bin offsets.
* :func:`phase_entropy` -- Appendix C, phase entropy of the times per frequency.
* :func:`topk` -- the k highest local maxima of a periodogram (Section 3.5).
* :func:`bins` -- bin of every (frequency, observation) pair and the exact
  distance from t*f to the nearest bin edge, for bin-mismatch accounting.
* :func:`fpw_shared` -- Section 4 / Appendix D batch routine: curves sharing
  their times, bins computed once per frequency.
* :func:`fpw_drift` (``drift.py``, numpy) -- Appendix A.1-A.2: the statistic with
  a polynomial baseline drift marginalised, formed densely.

``sanitize_driver.c`` calls every C entry point on seeded inputs and edge cases;
the tests build it with the C source under AddressSanitizer and
UndefinedBehaviorSanitizer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fpw.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "invalid data", 3: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``fpw_oracle.c`` into ``liboracle_fpw.so`` next to it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, c_int = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            vp = ctypes.c_void_p
            lib.oracle_fpw.argtypes = [vp, vp, vp, i64, vp, i64, c_int, d, vp]
            lib.oracle_fpw.restype = c_int
            lib.oracle_fpw_batch.argtypes = [vp, i64, vp, vp, vp, vp, i64, c_int, d, c_int, vp, c_int, c_int, vp, vp]
            lib.oracle_fpw_batch.restype = c_int
            lib.oracle_topk.argtypes = [vp, i64, c_int, c_int, vp, vp]
            lib.oracle_topk.restype = c_int
            lib.oracle_bins.argtypes = [vp, i64, vp, i64, c_int, vp, vp]
            lib.oracle_bins.restype = c_int
            lib.oracle_fpw_multi.argtypes = [vp, vp, vp, i64, vp, i64, c_int, c_int, d, vp]
            lib.oracle_fpw_multi.restype = c_int
            lib.oracle_fpw_shared.argtypes = [vp, i64, i64, vp, vp, vp, i64, c_int, d, vp]
            lib.oracle_fpw_shared.restype = c_int
            lib.oracle_phase_entropy.argtypes = [vp, i64, vp, i64, c_int, vp]
            lib.oracle_phase_entropy.restype = c_int
            lib.oracle_min_edge.argtypes = [vp, i64, vp, i64, c_int, vp]
            lib.oracle_min_edge.restype = c_int
            lib.oracle_version.restype = c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc: int) -> None:
    if rc != 0:
        raise OracleError(f"oracle status {rc}: {STATUS.get(rc, 'unknown')}")


def fpw(t, x, sigma, freqs, M: int, inv_alpha2: float = 0.0) -> np.ndarray:
    """S_FPW (Eq. 1) of one curve at every frequency in ``freqs`` (float64)."""
    lib = _load()
    t, x, sigma, freqs = _f64(t), _f64(x), _f64(sigma), _f64(freqs)
    n = t.shape[0]
    if x.shape[0] != n or sigma.shape[0] != n:
        raise ValueError("t, x, sigma must have equal length")
    S = np.empty(freqs.shape[0], dtype=np.float64)
    _check(lib.oracle_fpw(_ptr(t), _ptr(x), _ptr(sigma), n, _ptr(freqs), freqs.shape[0], int(M), float(inv_alpha2),
                          _ptr(S)))
    return S


def fpw_multi(t, x, sigma, freqs, M_max: int, g: int, inv_alpha2: float = 0.0) -> np.ndarray:
    """Section 3.4: S for M = M_max / g bins, combined from the M_max-bin sums,
    for each of the g bin offsets: array ``[g, F]``."""
    lib = _load()
    t, x, sigma, freqs = _f64(t), _f64(x), _f64(sigma), _f64(freqs)
    S = np.empty((int(g), freqs.shape[0]), dtype=np.float64)
    _check(lib.oracle_fpw_multi(_ptr(t), _ptr(x), _ptr(sigma), t.shape[0], _ptr(freqs), freqs.shape[0], int(M_max),
                                int(g), float(inv_alpha2), _ptr(S)))
    return S


def fpw_shared(t, x, sigma, freqs, M: int, inv_alpha2: float = 0.0) -> np.ndarray:
    """Section 4 / Appendix D batch routine: curves sharing the times ``t``
    (``x`` and ``sigma`` of shape ``[C, n]``), bins computed once per
    frequency: array ``[C, F]``; NaN rows for curves with invalid data."""
    lib = _load()
    t, freqs = _f64(t), _f64(freqs)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, t.shape[0]))
    sigma = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(x.shape))
    S = np.empty((x.shape[0], freqs.shape[0]), dtype=np.float64)
    _check(lib.oracle_fpw_shared(_ptr(t), t.shape[0], x.shape[0], _ptr(x), _ptr(sigma), _ptr(freqs), freqs.shape[0],
                                 int(M), float(inv_alpha2), _ptr(S)))
    return S


def phase_entropy(t, freqs, M: int) -> np.ndarray:
    """Appendix C: phase entropy of the times at each frequency (natural log)."""
    lib = _load()
    t, freqs = _f64(t), _f64(freqs)
    H = np.empty(freqs.shape[0], dtype=np.float64)
    _check(lib.oracle_phase_entropy(_ptr(t), t.shape[0], _ptr(freqs), freqs.shape[0], int(M), _ptr(H)))
    return H


def fpw_batch(offsets, t, x, sigma, freqs, M: int, inv_alpha2: float = 0.0, *, nthreads: int | None = None,
              dense: bool = True, k: int = 0, raw: bool = False):
    """Ragged batch. Returns ``(S, topk_idx, topk_S)``; ``S`` is ``[C, F]`` or None."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    t, x, sigma, freqs = _f64(t), _f64(x), _f64(sigma), _f64(freqs)
    C = offsets.shape[0] - 1
    F = freqs.shape[0]
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    S = np.empty((C, F), dtype=np.float64) if dense else None
    idx = np.empty((C, max(k, 0)), dtype=np.int32)
    val = np.empty((C, max(k, 0)), dtype=np.float64)
    _check(lib.oracle_fpw_batch(_ptr(offsets), C, _ptr(t), _ptr(x), _ptr(sigma), _ptr(freqs), F, int(M),
                                float(inv_alpha2), int(nthreads), _ptr(S), int(k), int(bool(raw)),
                                _ptr(idx) if k > 0 else None, _ptr(val) if k > 0 else None))
    return S, idx, val


def topk(S, k: int, raw: bool = False):
    """Top-k peaks (or raw top-k) of one periodogram: ``(idx int32[k], S float64[k])``."""
    lib = _load()
    S = _f64(S)
    idx = np.empty(k, dtype=np.int32)
    val = np.empty(k, dtype=np.float64)
    _check(lib.oracle_topk(_ptr(S), S.shape[0], int(k), int(bool(raw)), _ptr(idx), _ptr(val)))
    return idx, val


def bins(t, freqs, M: int, *, want_bins: bool = True, want_edge: bool = True):
    """Bins ``int32[F, n]`` and exact edge distances ``float64[F, n]`` (cycles)."""
    lib = _load()
    t, freqs = _f64(t), _f64(freqs)
    n, F = t.shape[0], freqs.shape[0]
    b = np.empty((F, n), dtype=np.int32) if want_bins else None
    e = np.empty((F, n), dtype=np.float64) if want_edge else None
    _check(lib.oracle_bins(_ptr(t), n, _ptr(freqs), F, int(M), _ptr(b), _ptr(e)))
    return b, e


def min_edge(t, freqs, M: int) -> np.ndarray:
    """Per frequency, the smallest exact distance (cycles) from t_i * f to a bin edge."""
    lib = _load()
    t, freqs = _f64(t), _f64(freqs)
    out = np.empty(freqs.shape[0], dtype=np.float64)
    _check(lib.oracle_min_edge(_ptr(t), t.shape[0], _ptr(freqs), freqs.shape[0], int(M), _ptr(out)))
    return out


def _split_freqs(fn, freqs, nthreads, *args):
    import concurrent.futures as cf
    freqs = _f64(freqs)
    nthreads = max(1, int(nthreads or (os.cpu_count() or 1)))
    parts = np.array_split(np.arange(freqs.shape[0]), nthreads)
    out = np.empty(freqs.shape[0], dtype=np.float64)

    def one(ix):
        if ix.size:
            out[ix[0]:ix[-1] + 1] = fn(*args, freqs[ix[0]:ix[-1] + 1])
    with cf.ThreadPoolExecutor(max_workers=nthreads) as ex:  # ctypes calls release the GIL
        list(ex.map(one, parts))
    return out


def fpw_parallel(t, x, sigma, freqs, M: int, inv_alpha2: float = 0.0, nthreads: int | None = None) -> np.ndarray:
    """:func:`fpw` with the frequency grid split across threads (same arithmetic per frequency)."""
    return _split_freqs(lambda t_, x_, s_, f_: fpw(t_, x_, s_, f_, M, inv_alpha2), freqs, nthreads, t, x, sigma)


def min_edge_parallel(t, freqs, M: int, nthreads: int | None = None) -> np.ndarray:
    return _split_freqs(lambda t_, f_: min_edge(t_, f_, M), freqs, nthreads, t)


def version() -> int:
    return int(_load().oracle_version())


from .drift import chebyshev_basis, fpw_drift, fpw_drift_chi2_difference  # noqa: E402  (uses bins above)
