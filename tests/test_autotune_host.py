"""Host-side pieces of the autotuner (no GPU)."""
from paper_2502_00243_gb300 import autotune


def test_m_ranges_partition_the_bin_counts():
    r = autotune.m_ranges([20, 10, 50])
    assert [m for m, _, _ in r] == [10, 20, 50]
    assert r[0][1] == 1 and r[-1][2] >= 1 << 20
    for (m0, lo0, hi0), (m1, lo1, hi1) in zip(r, r[1:]):
        assert hi0 + 1 == lo1 and lo0 <= m0 <= hi0 and lo1 <= m1 <= hi1


def test_typical_n_and_synthetic_curves():
    assert autotune.typical_n(0, 300) == 122 and autotune.typical_n(1000, 1 << 40) == 1732
    off, t, x, s = autotune.synthetic_curves(50, 3, seed=1)
    assert list(off) == [0, 50, 100, 150] and t.shape == x.shape == s.shape == (150,)
    assert (s > 0).all() and all((t[i * 50:(i + 1) * 50][1:] >= t[i * 50:(i + 1) * 50][:-1]).all() for i in range(3))


def test_table_round_trip(tmp_path):
    e = [{"M_lo": 1, "M_hi": 15, "n_lo": 0, "n_hi": 300, "threads": 128, "freqs_per_thread": 8, "obs_chunk": 0}]
    p = tmp_path / "t.json"
    autotune.save(e, str(p))
    assert autotune.load(str(p)) == e


def test_n_typical_matches_the_library_key():
    import numpy as np
    off = np.array([0, 100, 100, 400, 1400], dtype=np.int64)
    n = np.array([100, 0, 300, 1000], dtype=np.float64)
    assert autotune.n_typical(off) == int((n * n).sum() / n.sum())
    assert autotune.n_typical(np.array([0], dtype=np.int64)) == 0


def test_stratified_sample_keeps_whole_curves_across_sizes():
    import numpy as np
    rng = np.random.default_rng(3)
    sizes = rng.integers(1, 50, 40)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    t = np.arange(off[-1], dtype=np.float64)
    x, s = -t, t + 0.5
    so, st, sx, ss = autotune.stratified_sample(off, t, x, s, 9)
    picked = np.diff(so)
    assert 1 <= picked.size <= 9 and picked.min() == sizes.min() and picked.max() == sizes.max()
    # every sampled curve is one of the batch's curves, whole and in order
    starts = {int(t[o]): int(n) for o, n in zip(off[:-1], sizes)}
    for a, b in zip(so[:-1], so[1:]):
        seg = st[a:b]
        assert starts[int(seg[0])] == b - a and np.all(np.diff(seg) == 1)
        assert np.array_equal(sx[a:b], -seg) and np.array_equal(ss[a:b], seg + 0.5)
    # a request for more curves than the batch holds returns every curve once
    so, st, _, _ = autotune.stratified_sample(off, t, x, s, 100)
    assert so[-1] == off[-1] and np.array_equal(np.sort(np.diff(so)), np.sort(sizes))
