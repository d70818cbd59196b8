"""Seeded synthetic ZTF-shaped light curves for the FPW periodogram.

This module holds input generators only: it computes none of the FPW
statistic (no phases, bins, sums or peaks). Both the oracle-side tests and the
GPU side draw their inputs from here.

Workloads (the paper's ZTF light curves are not available, so seeded synthetic
curves with ZTF-like cadence and noise stand in for them):

* ``single_plain``  -- 200 times uniform over 0-1000 d, 0.3-amplitude sinusoid
  at P = 0.37 d, sigma log-uniform [0.01, 0.1], M = 10, 1e4 linear frequencies
  0.01-50 1/d.
* ``single_ztf``    -- one N = 1000 curve with ZTF-like cadence, a detached
  eclipse (8%-of-phase box dip of 0.5 mag) at P = 0.8123 d, sigma log-uniform
  [0.02, 0.2], M = 20, 1e6 frequencies 0.01-100 1/d.
* ``ragged_10k``    -- 10,000 curves, N uniform 50..2000, waveforms 25% each of
  sinusoid / box eclipse / sawtooth / pure noise, P log-uniform 0.05-50 d,
  amplitude/noise ratio log-uniform 0.2-5, sigma log-uniform [0.01, 0.3],
  M = 20, 2e5 frequencies 0.02-50 1/d, top-5 peaks.
* ``precision``     -- 100 curves, N = 1500 over a 2000-day baseline,
  sinusoid + eclipse at P log-uniform 0.05-0.5 d, 2e6 frequencies up to
  500 1/d (t*f up to 1e6 cycles), M = 20.
* ``sweep_100k``    -- 1e5 curves, N log-uniform 100-3000, mixed waveforms as
  ``ragged_10k``, M in {10, 20, 50}, 5e5 frequencies 0.01-50 1/d, top-5.
* ``shared_4096``   -- 4096 curves of one field observed in the same exposures:
  one ZTF-like cadence of N = 1000 times shared by all, per-curve waveforms,
  amplitudes and sigma as ``ragged_10k``, M = 20, 5e5 frequencies 0.01-50 1/d,
  top-5 (the shared-timestamp batch).

Cadence model: seasons of 240 days starting every 365 days; nights about 3 days
apart (3 +- 0.5 d); each night holds visit pairs 30 min apart starting
0.1-0.4 d past the integer day; one pair per night while N <= 2 * nights, else
ceil(N / (2 * nights)) pairs per night 1 h apart; exactly N of those slots are
drawn without replacement; times are shifted to start at 0. Every curve has its
flux shifted by its inverse-variance-weighted mean (the paper's input is
mean-subtracted; the library itself never subtracts anything).

Seeding: curve ``c`` of workload id ``w`` draws from
``numpy.random.default_rng([w, c])``, so any subset of a workload can be
regenerated on its own.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PAIR_GAP_DAYS = 30.0 / 1440.0
WAVEFORMS = ("sinusoid", "eclipse", "sawtooth", "noise")


@dataclasses.dataclass
class Workload:
    name: str
    offsets: np.ndarray  # int64 [C+1]
    t: np.ndarray  # float64 [sum n]
    x: np.ndarray  # float64
    sigma: np.ndarray  # float64
    freqs: np.ndarray  # float64 [F]
    M: int
    k: int
    curve_ids: np.ndarray  # int64 [C], index of each curve within the full workload
    periods: np.ndarray  # float64 [C], injected period (nan for noise)
    kinds: list  # waveform kind per curve

    @property
    def ncurves(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nfreq(self) -> int:
        return int(self.freqs.shape[0])

    @property
    def nobs(self) -> int:
        return int(self.offsets[-1])

    def evals(self) -> int:
        return self.nobs * self.nfreq

    def curve(self, c: int):
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        return self.t[a:b], self.x[a:b], self.sigma[a:b]

    def subset(self, cs) -> "Workload":
        """The curves at positions ``cs`` of this workload (same grid, M and k)."""
        curves = [(*self.curve(int(c)), self.periods[int(c)], self.kinds[int(c)]) for c in cs]
        return _assemble(self.name, [int(self.curve_ids[int(c)]) for c in cs], curves, self.freqs, self.M, self.k)


SPECS = {
    "single_plain": dict(wid=1, ncurves=1, M=10, k=5, f=(0.01, 50.0, 10_000)),
    "single_ztf": dict(wid=2, ncurves=1, M=20, k=5, f=(0.01, 100.0, 1_000_000)),
    "ragged_10k": dict(wid=3, ncurves=10_000, M=20, k=5, f=(0.02, 50.0, 200_000)),
    "precision": dict(wid=4, ncurves=100, M=20, k=5, f=(0.01, 500.0, 2_000_000)),
    "sweep_100k": dict(wid=5, ncurves=100_000, M=20, k=5, f=(0.01, 50.0, 500_000)),
    "shared_4096": dict(wid=6, ncurves=4096, M=20, k=5, f=(0.01, 50.0, 500_000)),
}

SHARED_N = 1000


def shared_times() -> np.ndarray:
    """The observation times every ``shared_4096`` curve shares."""
    return ztf_cadence(np.random.default_rng([SPECS["shared_4096"]["wid"]]), SHARED_N)


def freq_grid(name: str) -> np.ndarray:
    lo, hi, n = SPECS[name]["f"]
    return np.linspace(lo, hi, n, dtype=np.float64)


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def ztf_cadence(rng, n: int, seasons: int = 3, season_days: float = 240.0, baseline_days: float | None = None):
    """Sorted observation times (days, starting at 0) for one ZTF-like curve."""
    nights = []
    for y in range(seasons):
        start = 365.0 * y
        steps = 3.0 + rng.uniform(-0.5, 0.5, size=int(season_days / 2.5) + 2)
        d = start + rng.uniform(0.0, 3.0) + np.concatenate(([0.0], np.cumsum(steps[1:])))
        nights.append(np.floor(d[d < start + season_days]))
    nights = np.concatenate(nights)
    if baseline_days is not None:
        nights = nights[nights < baseline_days - 1.0]
    nn = nights.shape[0]
    pairs = max(1, -(-n // (2 * nn)))
    first = nights + rng.uniform(0.1, 0.4, size=nn)
    slots = (first[:, None, None] + (np.arange(pairs) / 24.0)[None, :, None]
             + np.array([0.0, PAIR_GAP_DAYS])[None, None, :]).ravel()
    if slots.shape[0] < n:
        raise ValueError("cadence model has fewer slots than requested observations")
    t = np.sort(slots[rng.choice(slots.shape[0], size=n, replace=False)])
    return t - t[0]


def waveform(kind: str, t, period: float, phase0: float, amp: float):
    """Noise-free signal of one kind at times t."""
    ph = np.mod(t / period + phase0, 1.0)
    if kind == "sinusoid":
        return amp * np.sin(2.0 * np.pi * ph)
    if kind == "eclipse":
        return np.where(ph < 0.08, amp, 0.0)
    if kind == "sawtooth":
        return amp * (ph - 0.5)
    if kind == "noise":
        return np.zeros_like(t)
    raise ValueError(kind)


def _finish(rng, t, signal, sigma):
    x = signal + rng.normal(0.0, 1.0, size=t.shape[0]) * sigma
    w = 1.0 / (sigma * sigma)
    x = x - np.sum(w * x) / np.sum(w)
    return x


def _curve(name: str, c: int):
    spec = SPECS[name]
    rng = np.random.default_rng([spec["wid"], c])
    if name == "single_plain":
        n = 200
        t = np.sort(rng.uniform(0.0, 1000.0, size=n))
        sigma = _loguniform(rng, 0.01, 0.1, n)
        phase0 = rng.uniform(0.0, 1.0)
        x = _finish(rng, t, waveform("sinusoid", t, 0.37, phase0, 0.3), sigma)
        return t, x, sigma, 0.37, "sinusoid"
    if name == "single_ztf":
        n = 1000
        t = ztf_cadence(rng, n)
        sigma = _loguniform(rng, 0.02, 0.2, n)
        phase0 = rng.uniform(0.0, 1.0)
        x = _finish(rng, t, waveform("eclipse", t, 0.8123, phase0, 0.5), sigma)
        return t, x, sigma, 0.8123, "eclipse"
    if name in ("ragged_10k", "sweep_100k"):
        if name == "ragged_10k":
            n = int(rng.integers(50, 2001))
        else:
            n = int(round(float(_loguniform(rng, 100.0, 3000.0))))
        t = ztf_cadence(rng, n)
        sigma = _loguniform(rng, 0.01, 0.3, n)
        kind = WAVEFORMS[int(rng.integers(0, 4))]
        period = float(_loguniform(rng, 0.05, 50.0))
        amp = float(_loguniform(rng, 0.2, 5.0)) * float(np.median(sigma))
        x = _finish(rng, t, waveform(kind, t, period, rng.uniform(0.0, 1.0), amp), sigma)
        return t, x, sigma, (period if kind != "noise" else float("nan")), kind
    if name == "shared_4096":
        t = shared_times()
        sigma = _loguniform(rng, 0.01, 0.3, t.shape[0])
        kind = WAVEFORMS[int(rng.integers(0, 4))]
        period = float(_loguniform(rng, 0.05, 50.0))
        amp = float(_loguniform(rng, 0.2, 5.0)) * float(np.median(sigma))
        x = _finish(rng, t, waveform(kind, t, period, rng.uniform(0.0, 1.0), amp), sigma)
        return t, x, sigma, (period if kind != "noise" else float("nan")), kind
    if name == "precision":
        n = 1500
        t = ztf_cadence(rng, n, seasons=6, baseline_days=2000.0)
        sigma = _loguniform(rng, 0.01, 0.3, n)
        period = float(_loguniform(rng, 0.05, 0.5))
        med = float(np.median(sigma))
        a_sin = float(_loguniform(rng, 0.2, 5.0)) * med
        a_ecl = float(_loguniform(rng, 0.2, 5.0)) * med
        ph0 = rng.uniform(0.0, 1.0)
        s = waveform("sinusoid", t, period, ph0, a_sin) + waveform("eclipse", t, period, ph0, a_ecl)
        x = _finish(rng, t, s, sigma)
        return t, x, sigma, period, "sinusoid+eclipse"
    raise KeyError(name)


def _assemble(name, ids, curves, freqs, M, k):
    ns = np.array([c[0].shape[0] for c in curves], dtype=np.int64)
    offsets = np.zeros(len(curves) + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    cat = (lambda j: np.concatenate([c[j] for c in curves]) if curves else np.zeros(0))
    return Workload(name=name, offsets=offsets, t=cat(0), x=cat(1), sigma=cat(2), freqs=freqs, M=M, k=k,
                    curve_ids=np.asarray(ids, dtype=np.int64),
                    periods=np.array([c[3] for c in curves], dtype=np.float64), kinds=[c[4] for c in curves])


def make(name: str, curves=None, *, M: int | None = None, nfreq: int | None = None) -> Workload:
    """Build a workload (or the subset ``curves`` of its curve indices).

    ``nfreq`` optionally replaces the grid by a linear grid over the same range
    with fewer points (for bounded oracle runs); ``M`` overrides the bin count.
    """
    spec = SPECS[name]
    ids = range(spec["ncurves"]) if curves is None else [int(c) for c in curves]
    lo, hi, n = spec["f"]
    freqs = np.linspace(lo, hi, n if nfreq is None else nfreq, dtype=np.float64)
    return _assemble(name, list(ids), [_curve(name, c) for c in ids], freqs, spec["M"] if M is None else M, spec["k"])


def ragged(seed: int, ns, nfreq: int, *, fmax: float = 50.0, M: int = 20, k: int = 5) -> Workload:
    """Small ragged batch with explicit sizes ``ns`` (zero allowed) for parity tests."""
    rng = np.random.default_rng([99, seed])
    curves = []
    for n in ns:
        n = int(n)
        if n == 0:
            curves.append((np.zeros(0), np.zeros(0), np.zeros(0), float("nan"), "empty"))
            continue
        t = np.sort(rng.uniform(0.0, 1000.0, size=n)) if n < 60 else ztf_cadence(rng, n)
        sigma = _loguniform(rng, 0.01, 0.3, n)
        kind = WAVEFORMS[int(rng.integers(0, 4))]
        period = float(_loguniform(rng, 0.05, 20.0))
        amp = float(_loguniform(rng, 0.5, 5.0)) * float(np.median(sigma))
        x = _finish(rng, t, waveform(kind, t, period, rng.uniform(0.0, 1.0), amp), sigma)
        curves.append((t, x, sigma, period, kind))
    freqs = np.linspace(0.01, fmax, nfreq, dtype=np.float64)
    return _assemble(f"ragged_seed{seed}", list(range(len(ns))), curves, freqs, M, k)
