"""The synthetic stand-ins for ZTF light curves against the recipes they follow:
sizes, grids, noise ranges, the cadence model (three 240-day seasons a year,
nights about 3 days apart, visit pairs 30 minutes apart), the waveform mix,
weighted-mean-subtracted fluxes, shared times for the field workload, and
determinism. CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L


def _wmean(x, s):
    w = 1.0 / (s * s)
    return float(np.sum(w * x) / np.sum(w))


def test_single_curves_follow_their_recipes():
    w = L.make("single_plain")
    t, x, s = w.curve(0)
    assert t.size == 200 and w.M == 10 and w.nfreq == 10_000
    assert np.all(np.diff(t) >= 0) and 0.0 <= t.min() and t.max() <= 1000.0
    assert 0.01 <= s.min() and s.max() <= 0.1
    assert w.freqs[0] == 0.01 and w.freqs[-1] == 50.0
    assert abs(_wmean(x, s)) < 1e-12 * np.abs(x).max()
    z = L.make("single_ztf")
    t, x, s = z.curve(0)
    assert t.size == 1000 and z.M == 20 and z.nfreq == 1_000_000 and z.freqs[-1] == 100.0
    assert 0.02 <= s.min() and s.max() <= 0.2
    assert z.kinds[0] == "eclipse" and z.periods[0] == 0.8123


def test_cadence_model():
    rng = np.random.default_rng(5)
    t = L.ztf_cadence(rng, 1000)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    # three seasons of at most 240 days, one per 365-day year
    gaps = np.diff(np.unique(np.floor(t)))
    assert np.sum(gaps > 100) == 2                     # two between-season gaps
    # nights about 3 days apart within a season; visits in pairs 30 min apart
    within = gaps[gaps < 100]
    assert 2.0 <= np.median(within) <= 4.0
    d = np.diff(t)
    assert np.any(np.isclose(d, 30.0 / 1440.0, atol=1e-9))
    assert t.max() < 3 * 365.0


def test_ragged_and_sweep_curves():
    r = L.make("ragged_10k", range(400))
    n = np.diff(r.offsets)
    assert n.min() >= 50 and n.max() <= 2000 and r.nfreq == 200_000
    kinds = {k: r.kinds.count(k) for k in set(r.kinds)}
    assert set(kinds) == {"sinusoid", "eclipse", "sawtooth", "noise"}
    assert all(60 <= v <= 140 for v in kinds.values())  # 25 % each of 400
    assert 0.01 <= r.sigma.min() and r.sigma.max() <= 0.3
    per = r.periods[~np.isnan(r.periods)]
    assert 0.05 <= per.min() and per.max() <= 50.0
    s = L.make("sweep_100k", range(300))
    n = np.diff(s.offsets)
    assert n.min() >= 100 and n.max() <= 3000 and s.nfreq == 500_000
    assert 350 <= np.median(n) <= 850                  # log-uniform 100-3000: median ~ 550
    for c in (0, 7, 123):
        t, x, sg = s.curve(c)
        assert abs(_wmean(x, sg)) < 1e-11 * np.abs(x).max()


def test_precision_and_shared_workloads():
    p = L.make("precision", range(3))
    assert np.all(np.diff(p.offsets) == 1500) and p.nfreq == 2_000_000 and p.freqs[-1] == 500.0
    assert p.t.max() < 2000.0 and np.all((0.05 <= p.periods) & (p.periods <= 0.5))
    f = L.make("shared_4096", range(5))
    t0 = f.curve(0)[0]
    assert t0.size == L.SHARED_N
    assert all(np.array_equal(f.curve(c)[0], t0) for c in range(5))
    assert not np.array_equal(f.curve(0)[1], f.curve(1)[1])


@pytest.mark.parametrize("name", ["ragged_10k", "sweep_100k", "shared_4096"])
def test_workloads_are_deterministic_and_subsets_agree(name):
    a = L.make(name, [3, 11])
    b = L.make(name, [11])
    assert np.array_equal(a.curve(1)[0], b.curve(0)[0]) and np.array_equal(a.curve(1)[1], b.curve(0)[1])
    sub = a.subset([1])
    assert np.array_equal(sub.x, b.x) and sub.curve_ids.tolist() == [11]
