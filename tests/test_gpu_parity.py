"""GPU parity: the sm_103a kernels (through the C ABI) against the FP64 oracle on
the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, bin_mismatches, check_topk, run_batch, run_bins, run_single, s_bound, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = None


@pytest.fixture(scope="module")
def ctx():
    global G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    G = G_
    c = G.Context(0)
    yield c
    c.close()


def P(**kw):
    return G.fpw_params_default(**kw)


# ------------------------------------------------------------------ single curve, plain sinusoid (10^4 freqs)
def test_single_plain_dense_default(ctx):
    w = L.make("single_plain")
    t, x, s = w.curve(0)
    S_or = oracle.fpw(t, x, s, w.freqs, w.M)
    S_g, st = run_single(ctx, t, x, s, w.freqs, w.M)
    assert st == 0
    assert_S_close(S_g, S_or, s_bound(x, s), what="single_plain fixed64/fp32")


def test_single_plain_fp64_plain_form_matches_bitwise(ctx):
    w = L.make("single_plain")
    t, x, s = w.curve(0)
    for c in (0.0, 1.0):
        S_or = oracle.fpw(t, x, s, w.freqs, w.M, c)
        S_g, st = run_single(ctx, t, x, s, w.freqs, w.M, P(phase_mode=G.FPW_PHASE_FP64, inv_alpha2=c))
        assert st == 0
        # same binary64 operations in the same order: identical bins and sums
        np.testing.assert_array_equal(S_g, S_or)


def test_single_plain_fixed64_fp64_sums(ctx):
    w = L.make("single_plain")
    t, x, s = w.curve(0)
    S_or = oracle.fpw(t, x, s, w.freqs, w.M, 0.3)
    S_g, st = run_single(ctx, t, x, s, w.freqs, w.M, P(accum=G.FPW_ACCUM_FP64, inv_alpha2=0.3))
    assert st == 0
    assert_S_close(S_g, S_or, s_bound(x, s), rel=1e-6, absf=1e-9, what="fixed64/fp64 sums")


# ------------------------------------------------------------------ single ZTF-like curve, 10^6 freqs
def test_single_ztf_full_grid(ctx):
    w = L.make("single_ztf")
    t, x, s = w.curve(0)
    S_or = oracle.fpw_parallel(t, x, s, w.freqs, w.M)
    near = oracle.min_edge_parallel(t, w.freqs, w.M) <= 1e-9
    S_g, st = run_single(ctx, t, x, s, w.freqs, w.M)
    assert st == 0
    assert_S_close(S_g, S_or, s_bound(x, s), mask=~near, what="single_ztf dense")
    # top-5 through the batch path on the same curve
    idx, Sk, _, st = run_batch(ctx, w)
    assert st == 0
    o_idx, o_S = oracle.topk(S_or, 12)
    check_topk(idx[0], Sk[0], o_idx, o_S, o_dense=S_or, abs_tol=1e-7 * s_bound(x, s), what="single_ztf topk")


# ------------------------------------------------------------------ ragged batches, edge sizes
RAGGED = [
    # (ns, nfreq, M, k, params)
    ([0, 1, 2, 31, 32, 33, 127, 500], 1021, 20, 5, {}),
    ([3000, 1, 1025, 64], 3001, 10, 8, {"obs_chunk": 256}),
    ([700, 0, 250], 1, 5, 3, {}),
    ([700, 250, 40], 2, 5, 3, {}),
    ([400, 900], 509, 50, 64, {}),
    ([400, 900], 510, 50, 5, {"freqs_per_thread": 8, "threads": 64}),
    ([333, 1200], 2048, 1, 4, {}),
    ([333, 1200, 77], 4097, 3, 6, {"freqs_per_thread": 2, "threads": 256}),
    ([1500, 10, 800], 2500, 20, 5, {"accum": 1}),
    ([1500, 10, 800, 63, 2], 2500, 20, 5, {"accum": 2}),
    ([400, 900], 509, 50, 6, {"accum": 2, "inv_alpha2": 0.7}),
    ([1500, 10, 800], 2500, 20, 5, {"peak_mode": 1}),
    ([600, 2100], 1999, 64, 7, {"inv_alpha2": 0.5}),
    ([50, 1700, 333], 2111, 55, 5, {}),
    ([900, 2600, 31, 450], 3001, 30, 5, {"freqs_per_thread": 3}),
    ([900, 2600, 31, 450], 2999, 16, 5, {"freqs_per_thread": 6, "threads": 96}),
    ([900, 2600, 31, 450], 3001, 19, 5, {"freqs_per_thread": 5, "threads": 128, "obs_chunk": 128}),
]


@pytest.mark.parametrize("case", range(len(RAGGED)))
def test_ragged_batches_dense_and_topk(ctx, case):
    ns, F, M, k, kw = RAGGED[case]
    w = L.ragged(case, ns, F, M=M, k=k)
    p = P(**kw)
    c = kw.get("inv_alpha2", 0.0)
    raw = kw.get("peak_mode", 0) == 1
    idx, Sk, Sd, st = run_batch(ctx, w, params=p, dense=True)
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, M, c, k=k + 4, raw=raw)
    wide = kw.get("accum", 0) in (1, 2)  # binary64 or compensated FP32 sums
    rel = 1e-6 if wide else 1e-4
    for ci in range(w.ncurves):
        t, x, s = w.curve(ci)
        near = oracle.min_edge(t, w.freqs, M) <= 1e-9 if t.size else np.zeros(F, bool)
        bound = s_bound(x, s)
        assert_S_close(Sd[ci], S_or[ci], bound, rel=rel, absf=1e-9 if wide else 1e-7, mask=~near,
                       what=f"case {case} curve {ci} dense")
        check_topk(idx[ci], Sk[ci], o_idx[ci], o_S[ci], rel=rel, abs_tol=1e-7 * bound, o_dense=S_or[ci], raw=raw,
                   what=f"case {case} curve {ci}")


def test_empty_curve_peaks(ctx):
    w = L.ragged(50, [0, 10], 100, M=4, k=3)
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == 0
    assert np.all(Sd[0] == 0.0)
    # a flat zero periodogram has exactly one peak, at frequency 0
    assert list(idx[0]) == [0, -1, -1] and Sk[0][0] == 0.0 and np.isnan(Sk[0][1:]).all()


# ------------------------------------------------------------------ bins of the periodogram kernel itself
# fpw_periodogram_batch_bins runs the kernels of the batched call (same shape,
# tiles, anchors and stepping) and writes the bin it gave every observation.
def _bins_case(ctx, mode, K=256, accum=0, nwin=3000, f_start=499.0):
    """One 1500-observation curve of the 2000-day workload on its full 2e6-point
    grid to 500 1/d (t f up to 1e6 cycles); bins of nwin frequencies near f_start."""
    w = L.make("precision", [0])
    k0 = int(np.searchsorted(w.freqs, f_start))
    g, _, st = run_bins(ctx, w, k0, k0 + nwin, params=P(phase_mode=mode, K=K, accum=accum))
    assert st == 0
    return bin_mismatches(g, w, k0, k0 + nwin, w.M, oracle.bins)


@pytest.mark.parametrize("accum", [0, 1, 2])
def test_bins_fixed64_identical_off_edge(ctx, accum):
    pairs, mism, far, worst = _bins_case(ctx, G.FPW_PHASE_FIXED64, accum=accum)
    assert pairs == 3000 * 1500
    assert far == 0, f"{far} mismatches beyond 1e-9 cycles (worst edge distance {worst})"


def test_bins_fp64_plain_identical(ctx):
    pairs, mism, far, worst = _bins_case(ctx, G.FPW_PHASE_FP64)
    assert pairs == 3000 * 1500 and mism == 0


@pytest.mark.parametrize("K", [64, 256, 1024])
def test_bins_fp32_phase_mismatch_within_analytic_margin(ctx, K):
    pairs, mism, far, worst = _bins_case(ctx, G.FPW_PHASE_FP32, K=K)
    margin = (2 * K + 4) * 2.0 ** -24
    assert worst <= margin, f"K={K}: mismatch at edge distance {worst} > {margin}"
    print(f"fp32 phase K={K}: mismatch rate {mism / pairs:.3e}")


# tile widths W = T R of 1024 (M = 10), 512 (M = 20), 256 (M = 50; and 16-byte
# bins at M = 20); curves split into several work items; chunk tails of every
# size mod 32; the first window contains the tile that starts one step before
# frequency 0, the second the grid's end
BIN_SHAPES = [(10, {}), (20, {}), (50, {}), (20, {"accum": 1}), (20, {"accum": 2}),
              (20, {"obs_chunk": 96}), (20, {"threads": 64, "freqs_per_thread": 8}),
              (12, {"threads": 96, "freqs_per_thread": 1}), (16, {}), (30, {})]


@pytest.mark.parametrize("case", range(len(BIN_SHAPES)))
def test_bins_every_tile_width_and_segment(ctx, case):
    M, kw = BIN_SHAPES[case]
    w = L.ragged(40 + case, [2500, 37, 1000, 64, 65, 999, 0, 31], 30_000, M=M)
    d = to_dev(w)
    for k0, k1 in ((0, 1500), (w.nfreq - 4000, w.nfreq)):
        g, _, st = run_bins(ctx, w, k0, k1, params=P(**kw), d=d)
        assert st == 0
        pairs, mism, far, worst = bin_mismatches(g, w, k0, k1, M, oracle.bins)
        assert pairs == (k1 - k0) * w.nobs
        assert far == 0, f"M={M} {kw} window {k0}: {far} mismatches beyond 1e-9 cycles"
    T, R, NC, grid = ctx.last_shape()
    if "threads" in kw:
        assert (T, R) == (kw["threads"], kw["freqs_per_thread"])
    if not kw:
        assert R == {10: 8, 20: 5, 50: 2, 16: 6, 30: 3}[M]  # the default frequencies per thread


def test_three_five_and_six_frequencies_per_thread_only_where_instantiated(ctx):
    """R = 3, 5 and 6 exist for FP32 sums of one M: asked for elsewhere they are
    refused; a tuned table entry with them gives the other calls R = 2 or 4."""
    w = L.ragged(81, [700, 1500, 40], 3000, M=30, k=4)
    d = to_dev(w)
    for kw in ({"freqs_per_thread": 3, "accum": 2}, {"freqs_per_thread": 5, "accum": 2},
               {"freqs_per_thread": 6, "accum": 1}):
        with pytest.raises(G.FPWError) as ei:
            run_batch(ctx, w, d=d, params=P(**kw))
        assert ei.value.code == G.FPW_ENOTSUP
    C, k = w.ncurves, 4
    mi = torch.empty(C * k, dtype=torch.int32, device="cuda")
    mo, ms_ = torch.empty_like(mi), torch.empty(C * k, dtype=torch.float32, device="cuda")
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram_batch_multi(ctx, None, P(freqs_per_thread=3), d["offsets"], w.offsets, d["t"], d["x"],
                                      d["sigma"], d["freqs"], 30, (3,), k, mi, mo, ms_)
    assert ei.value.code == G.FPW_ENOTSUP
    ref = run_batch(ctx, w, d=d, params=P(accum=2))
    ctx.set_shape(1, 100, 0, 1 << 40, 128, 3, 0, 0)
    try:
        got = run_batch(ctx, w, d=d, params=P(accum=2))  # compensated sums: R = 2
        assert ctx.last_shape()[1] == 2
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        G.fpw_periodogram_batch_multi(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"],
                                      d["freqs"], 30, (3,), k, mi, mo, ms_)
        torch.cuda.synchronize()
        assert ctx.last_shape()[1] == 2 and ctx.status() == 0
        run_batch(ctx, w, d=d)  # FP32 sums of one M: the entry's R = 3
        assert ctx.last_shape()[:2] == (128, 3)
    finally:
        ctx.clear_shapes()


def test_bins_nonlinear_grid_direct_anchors(ctx):
    w = L.ragged(78, [900, 300, 33], 10, M=12)
    rng = np.random.default_rng(2)
    w.freqs = np.sort(rng.uniform(0.01, 30.0, 1500))
    g, _, st = run_bins(ctx, w, 0, w.nfreq)
    assert st == 0
    pairs, mism, far, worst = bin_mismatches(g, w, 0, w.nfreq, 12, oracle.bins)
    assert pairs == w.nfreq * w.nobs and far == 0


def test_bins_call_writes_the_same_S_as_the_batched_call(ctx):
    w = L.ragged(79, [700, 1500, 40], 6000, M=20)
    d = to_dev(w)
    _, _, Sd, st = run_batch(ctx, w, d=d, dense=True, k=0)
    assert st == 0
    g, Sb, st = run_bins(ctx, w, 100, 300, d=d, dense=True)
    assert st == 0
    np.testing.assert_array_equal(Sb, Sd)


# ------------------------------------------------------------------ non-linear grid
def test_nonlinear_grid_uses_direct_anchor(ctx):
    w = L.ragged(77, [900, 300], 10)
    rng = np.random.default_rng(1)
    freqs = np.sort(rng.uniform(0.01, 30.0, 1500))
    t, x, s = w.curve(0)
    S_or = oracle.fpw(t, x, s, freqs, 12)
    S_g, st = run_single(ctx, t, x, s, freqs, 12)
    assert st == 0
    near = oracle.min_edge(t, freqs, 12) <= 1e-9
    assert_S_close(S_g, S_or, s_bound(x, s), mask=~near, what="non-linear grid")


# ------------------------------------------------------------------ errors
def test_invalid_data_reported_per_curve(ctx):
    w = L.ragged(9, [100, 200, 300], 500, M=10, k=3)
    sig = w.sigma.copy()
    sig[150] = 0.0  # curve 1
    w.sigma = sig
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True)
    assert st == G.FPW_EDATA
    assert np.all(idx[1] == -1) and np.isnan(Sk[1]).all() and np.isnan(Sd[1]).all()
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets[:2], w.t, w.x, w.sigma, w.freqs, 10, k=6)
    check_topk(idx[0], Sk[0], o_idx[0], o_S[0], o_dense=S_or[0], what="valid curve next to a bad one")
    assert ctx.status() == 0  # cleared by the previous read


def test_invalid_frequency_and_sync_entry_points(ctx):
    w = L.ragged(10, [50], 64, M=4, k=2)
    d = to_dev(w)
    d["freqs"][3] = float("nan")
    S = torch.empty(64, dtype=torch.float64, device="cuda")
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram(d["t"], d["x"], d["sigma"], d["freqs"], 4, S)
    assert ei.value.code == G.FPW_EDATA
    d["freqs"][3] = 1.0
    sig = d["sigma"].clone()
    sig[0] = -1.0
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram(d["t"], d["x"], sig, d["freqs"], 4, S)
    assert ei.value.code == G.FPW_EDATA
    G.fpw_periodogram(d["t"], d["x"], d["sigma"], d["freqs"], 4, S)  # recovers


def test_invalid_arguments_rejected_before_launch(ctx):
    w = L.ragged(11, [20, 30], 16, M=4, k=2)
    d = to_dev(w)
    idx = torch.empty(4, dtype=torch.int32, device="cuda")
    S = torch.empty(4, dtype=torch.float32, device="cuda")
    for M, k in ((0, 2), (4, -1), (4, G.FPW_MAX_TOPK + 1)):
        with pytest.raises(G.FPWError) as ei:
            G.fpw_periodogram_batch_ex(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"],
                                       d["freqs"], M, k, idx, S)
        assert ei.value.code == G.FPW_EINVAL
    bad_off = np.array([0, 30, 20], dtype=np.int64)
    with pytest.raises(G.FPWError) as ei:
        G.fpw_periodogram_batch_ex(ctx, None, None, d["offsets"], bad_off, d["t"], d["x"], d["sigma"], d["freqs"], 4,
                                   2, idx, S)
    assert ei.value.code == G.FPW_EINVAL
    for bad in (P(K=0), P(threads=48), P(freqs_per_thread=7), P(inv_alpha2=-1.0), P(phase_mode=9)):
        with pytest.raises(G.FPWError) as ei:
            G.fpw_periodogram_batch_ex(ctx, None, bad, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"],
                                       d["freqs"], 4, 2, idx, S)
        assert ei.value.code == G.FPW_EINVAL


# ------------------------------------------------------------------ graphs, host entry point, plain batch
def test_graph_replay_matches_direct(ctx):
    w = L.ragged(12, [300, 1000, 20, 2000], 5000, M=20, k=5)
    d = to_dev(w)
    a = run_batch(ctx, w, d=d)
    g1 = run_batch(ctx, w, d=d, params=P(use_graph=1))
    g2 = run_batch(ctx, w, d=d, params=P(use_graph=1))
    for r in (g1, g2):
        np.testing.assert_array_equal(r[0], a[0])
        np.testing.assert_array_equal(r[1], a[1])


def test_host_entry_point_matches_device_call(ctx):
    w = L.ragged(13, [300, 1000, 20], 3000, M=10, k=4)
    a = run_batch(ctx, w)
    idx = np.empty(w.ncurves * 4, dtype=np.int32)
    S = np.empty(w.ncurves * 4, dtype=np.float32)
    G.fpw_periodogram_batch_host(ctx, None, w.offsets, w.t, w.x, w.sigma, w.freqs, 10, 4, idx, S)
    np.testing.assert_array_equal(idx.reshape(-1, 4), a[0])
    np.testing.assert_array_equal(S.reshape(-1, 4), a[1])


def test_plain_fp64_batch_form(ctx):
    w = L.ragged(14, [300, 0, 800, 50], 2000, M=20, k=5)
    idx, Sk, Sd, st = run_batch(ctx, w, dense=True, params=P(phase_mode=G.FPW_PHASE_FP64))
    assert st == 0
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 20, k=5)
    np.testing.assert_array_equal(Sd, S_or)
    for ci in range(w.ncurves):
        np.testing.assert_array_equal(idx[ci], o_idx[ci])
        np.testing.assert_array_equal(Sk[ci], o_S[ci].astype(np.float32))


# ------------------------------------------------------------------ schedule: work items per resident block
def test_work_item_split_leaves_every_value_unchanged(ctx):
    """Tile anchors sit at q (W - 2) - 1 whatever the item boundaries, so the
    segment size of the persistent schedule changes no S value and no peak."""
    w = L.ragged(80, [2900, 35, 1200, 64, 700, 0, 2100], 20_000, M=20, k=6)
    d = to_dev(w)
    ref = run_batch(ctx, w, d=d, dense=True)
    assert ref[3] == 0
    for items in (1, 3, 64):
        got = run_batch(ctx, w, d=d, dense=True, params=P(items_per_slot=items))
        assert got[3] == 0
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
    with pytest.raises(G.FPWError) as ei:
        run_batch(ctx, w, d=d, params=P(items_per_slot=-1))
    assert ei.value.code == G.FPW_EINVAL
