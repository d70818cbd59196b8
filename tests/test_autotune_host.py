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
