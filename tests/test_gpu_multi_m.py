"""Several bin counts from one M_max pass (Section 3.4) on the GPU against the
oracle: per curve and group g, S_g(f) = max over the g bin offsets of the
statistic with M = M_max / g bins, its peaks and their offsets."""
from __future__ import annotations

import numpy as np
import pytest

import lightcurves as L
import oracle
from gpu_util import assert_S_close, check_topk, s_bound, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_00243_gb300 as G_
    return G_


def run_multi(G, ctx, w, M_max, groups, k, params=None):
    d = to_dev(w)
    C, F, ng = w.ncurves, w.nfreq, len(groups)
    idx = torch.empty(C * ng * k, dtype=torch.int32, device="cuda")
    off = torch.empty(C * ng * k, dtype=torch.int32, device="cuda")
    S = torch.empty(C * ng * k, dtype=torch.float32, device="cuda")
    Sd = torch.empty(C * ng * F, dtype=torch.float64, device="cuda")
    G.fpw_periodogram_batch_multi(ctx, None, params, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"],
                                  M_max, groups, k, idx, off, S, Sd)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return (idx.cpu().numpy().reshape(C, ng, k), off.cpu().numpy().reshape(C, ng, k),
            S.cpu().numpy().reshape(C, ng, k), Sd.cpu().numpy().reshape(C, ng, F))


@pytest.mark.parametrize("M_max,groups,ns,F", [
    (20, [1, 2, 4, 5, 10], [0, 50, 700, 1500, 3100], 3000),
    (60, [3, 6, 15], [400, 1200], 2048),
    (12, [12, 1, 3], [90, 333], 1021),
    (40, [2, 4, 10], [700, 64, 1500], 1500),
])
def test_multi_m_dense_topk_and_offsets(G, M_max, groups, ns, F):
    w = L.ragged(60 + M_max, ns, F, M=M_max, k=5)
    ctx = G.Context(0)
    k = 5
    idx, off, S, Sd = run_multi(G, ctx, w, M_max, groups, k)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, M_max) <= 1e-9 if t.size else np.zeros(F, bool)
        for q, g in enumerate(groups):
            So = oracle.fpw_multi(t, x, s, w.freqs, M_max, g)  # [g, F]
            Sg = So.max(axis=0)
            # FP32 prefix sums of the fine bins: S within 1e-4 relative, floor 1e-6 of sum w x^2
            assert_S_close(Sd[c, q], Sg, bound, rel=1e-4, absf=1e-6, mask=~near,
                           what=f"M_max={M_max} g={g} curve {c}")
            o_idx, o_S = oracle.topk(Sg, k + 4)
            check_topk(idx[c, q], S[c, q], o_idx, o_S, abs_tol=1e-6 * bound, o_dense=Sg,
                       what=f"M_max={M_max} g={g} curve {c} peaks")
            for j in range(k):
                fi = idx[c, q, j]
                if fi < 0:
                    assert off[c, q, j] == -1
                    continue
                o = off[c, q, j]
                assert 0 <= o < g
                tol = 2 * (1e-4 * abs(Sg[fi]) + 1e-6 * bound)
                assert So[o, fi] >= Sg[fi] - tol, (g, fi, o, So[:, fi])
    ctx.close()


def test_multi_m_group_one_equals_single_m_path(G):
    w = L.ragged(70, [800, 120, 2000], 2500, M=20, k=5)
    ctx = G.Context(0)
    idx, off, S, Sd = run_multi(G, ctx, w, 20, [1], 5)
    d = to_dev(w)
    Sd1 = torch.empty(w.ncurves * w.nfreq, dtype=torch.float64, device="cuda")
    i1 = torch.empty(w.ncurves * 5, dtype=torch.int32, device="cuda")
    s1 = torch.empty(w.ncurves * 5, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_ex(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"], 20, 5,
                               i1, s1, Sd1)
    torch.cuda.synchronize()
    Sd1 = Sd1.cpu().numpy().reshape(w.ncurves, w.nfreq)
    # same bins; the prefix-sum window differs from the direct bin sum only by FP32 rounding
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        assert_S_close(Sd[c, 0], Sd1[c], s_bound(x, s), rel=1e-4, absf=1e-6, what=f"g=1 curve {c}")
    assert np.all(off[idx >= 0] == 0)
    ctx.close()


def test_multi_m_rejects_bad_groups(G):
    w = L.ragged(71, [100], 64, M=20, k=2)
    ctx = G.Context(0)
    for M_max, groups in ((20, [3]), (20, []), (20, [1, 2, 4, 5, 10, 20, 1, 2, 4])):
        with pytest.raises(G.FPWError) as ei:
            run_multi(G, ctx, w, M_max, groups, 2)
        assert ei.value.code == G.FPW_EINVAL
    with pytest.raises(G.FPWError) as ei:
        run_multi(G, ctx, w, 20, [2], 2, params=G.fpw_params_default(accum=1))
    assert ei.value.code == G.FPW_ENOTSUP
    ctx.close()


def test_multi_m_thread_bound(G):
    """The several-M kernel takes at most 256 threads per block: explicit wider
    blocks are refused, and a wider shape-table entry is capped, with results
    equal to the default shape's within rounding of the summation order."""
    w = L.ragged(77, [600, 1300, 50], 2500, M=20, k=5)
    ctx = G.Context(0)
    with pytest.raises(G.FPWError) as ei:
        run_multi(G, ctx, w, 20, [1, 2], 5, params=G.fpw_params_default(threads=512))
    assert ei.value.code == G.FPW_ENOTSUP
    ref = run_multi(G, ctx, w, 20, [1, 2], 5)
    ctx.set_shape(1, 1000, 0, 1 << 40, 512, 1)
    got = run_multi(G, ctx, w, 20, [1, 2], 5)
    assert ctx.last_shape()[0] == 256
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        bound = s_bound(x, s)
        near = oracle.min_edge(t, w.freqs, 20) <= 1e-9  # other tiles, other anchors: edge pairs may move
        for q in range(2):
            assert_S_close(got[3][c, q], ref[3][c, q], bound, rel=1e-5, absf=1e-7, mask=~near,
                           what=f"capped shape curve {c}")
    ctx.clear_shapes()
    ctx.close()


def test_long_curve_peaks_merged_by_a_block(G):
    """A curve whose grid splits into hundreds of work items (its candidate rows
    are merged by a whole block instead of one warp), next to short ones, in the
    single-M call and in the several-M call (peaks with their offsets)."""
    w = L.ragged(78, [1500, 40, 600], 200_000, M=12, k=7)
    ctx = G.Context(0)
    d = to_dev(w)
    idx = torch.empty(w.ncurves * 7, dtype=torch.int32, device="cuda")
    S = torch.empty(w.ncurves * 7, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_ex(ctx, None, None, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"], 12,
                               7, idx, S)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    idx, S = idx.cpu().numpy().reshape(-1, 7), S.cpu().numpy().reshape(-1, 7)
    S_or, o_idx, o_S = oracle.fpw_batch(w.offsets, w.t, w.x, w.sigma, w.freqs, 12, k=11)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        check_topk(idx[c], S[c], o_idx[c], o_S[c], o_dense=S_or[c], abs_tol=1e-7 * s_bound(x, s),
                   what=f"long-grid curve {c}")
    mi, mo, ms_, Sd = run_multi(G, ctx, w, 12, [1, 3], 5)
    for c in range(w.ncurves):
        t, x, s = w.curve(c)
        bound = s_bound(x, s)
        for q, g in enumerate((1, 3)):
            So = oracle.fpw_multi(t, x, s, w.freqs, 12, g)
            Sg = So.max(axis=0)
            o_i, o_s = oracle.topk(Sg, 9)
            check_topk(mi[c, q], ms_[c, q], o_i, o_s, o_dense=Sg, abs_tol=1e-6 * bound, what=f"multi g={g} curve {c}")
            for j in range(5):
                if mi[c, q, j] >= 0:  # the reported offset is the best one at that frequency
                    col = So[:, mi[c, q, j]]
                    assert abs(col[mo[c, q, j]] - col.max()) <= 1e-4 * abs(col.max()) + 1e-6 * bound
    ctx.close()


@pytest.mark.parametrize("M_max,groups,ns,F", [
    (60, [3, 6, 15], [1300, 45, 2600, 700], 3001),
    (40, [2, 4, 10], [900, 2000, 77], 2500),
    (20, [1, 2, 4], [1500, 300, 2900], 4099),
])
def test_compiled_combination_equals_generic_bitwise(G, M_max, groups, ns, F):
    """(M_max, groups) = (60; 3, 6, 15), (40; 2, 4, 10) and (20; 1, 2, 4), in that
    order, run a combination compiled for them (one pass over the bins with
    the prefix sums in registers); the same groups in reverse order run the
    generic one. Same windows, terms and order of additions: the dense S, the
    peaks and their offsets must agree bit for bit, with and without a
    nonzero 1/alpha^2."""
    w = L.ragged(90 + M_max, ns, F, M=M_max, k=5)
    ctx = G.Context(0)
    for inv_a2 in (0.0, 0.7):
        p = G.fpw_params_default(inv_alpha2=inv_a2)
        i1, o1, s1, d1 = run_multi(G, ctx, w, M_max, groups, 5, params=p)
        i2, o2, s2, d2 = run_multi(G, ctx, w, M_max, groups[::-1], 5, params=p)
        assert np.array_equal(d1, d2[:, ::-1], equal_nan=True)
        assert np.array_equal(i1, i2[:, ::-1]) and np.array_equal(o1, o2[:, ::-1])
        assert np.array_equal(s1, s2[:, ::-1], equal_nan=True)
        assert np.isfinite(d1).all() and (i1[:, :, 0] >= 0).all()
    ctx.close()
