"""Helpers shared by the GPU parity tests: move seeded workloads to the device,
call the library through its C ABI, and compare against the oracle with the
tolerances of the parity contract:

* bins identical for every observation more than 1e-9 cycles from a bin edge;
* S within 1e-4 relative (FP32 bin sums) or 1e-6 relative (binary64 sums), with
  an absolute floor of 1e-7 * sum_i w_i x_i^2 for S near 0 (S is bounded by
  that sum, so the floor is relative to the curve's largest possible S);
* top-k indices identical wherever the oracle's neighbouring ranked peaks are
  separated by more than the S tolerance; near-tied peaks may swap ranks."""
from __future__ import annotations

import numpy as np
import torch

import paper_2502_00243_gb300 as G


def to_dev(w):
    return dict(offsets=torch.from_numpy(w.offsets).cuda(), t=torch.from_numpy(w.t).cuda(),
                x=torch.from_numpy(w.x).cuda(), sigma=torch.from_numpy(w.sigma).cuda(),
                freqs=torch.from_numpy(w.freqs).cuda())


def run_batch(ctx, w, *, M=None, k=None, params=None, dense=False, d=None):
    d = d or to_dev(w)
    M = w.M if M is None else M
    k = w.k if k is None else k
    C, F = w.ncurves, w.nfreq
    idx = torch.empty(C * k, dtype=torch.int32, device="cuda")
    S = torch.empty(C * k, dtype=torch.float32, device="cuda")
    Sd = torch.empty(C * F, dtype=torch.float64, device="cuda") if dense else None
    G.fpw_periodogram_batch_ex(ctx, None, params, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"],
                               M, k, idx if k else None, S if k else None, Sd)
    torch.cuda.synchronize()
    st = ctx.status()
    return (idx.cpu().numpy().reshape(C, k), S.cpu().numpy().reshape(C, k),
            Sd.cpu().numpy().reshape(C, F) if dense else None, st)


def run_bins(ctx, w, k0, k1, *, M=None, params=None, d=None, dense=False):
    """Bins that the periodogram kernel itself gave every observation of the
    batch at frequencies k0 <= k < k1 (fpw_periodogram_batch_bins; the same
    launch as the batched call): int32 ``[k1 - k0, nobs]``, -1 where nothing was
    written; with ``dense`` also S ``[C, F]``."""
    d = d or to_dev(w)
    M = w.M if M is None else M
    nobs = int(w.offsets[-1])
    out = torch.full(((k1 - k0) * nobs,), -1, dtype=torch.int32, device="cuda")
    Sd = torch.empty(w.ncurves * w.nfreq, dtype=torch.float64, device="cuda") if dense else None
    G.fpw_periodogram_batch_bins(ctx, None, params, d["offsets"], w.offsets, d["t"], d["x"], d["sigma"], d["freqs"],
                                 M, k0, k1, out, Sd)
    torch.cuda.synchronize()
    st = ctx.status()
    return (out.cpu().numpy().reshape(k1 - k0, nobs), Sd.cpu().numpy().reshape(w.ncurves, w.nfreq) if dense else None,
            st)


def bin_mismatches(g_bins, w, k0, k1, M, oracle_bins, curves=None):
    """Compare kernel bins ``[k1 - k0, nobs]`` of the batch ``w`` with the oracle's,
    curve by curve: (pairs, mismatches, mismatches farther than 1e-9 cycles
    from a bin edge, largest edge distance of a mismatch). Every pair must have
    been written."""
    pairs = mism = far = 0
    worst = 0.0
    fr = w.freqs[k0:k1]
    for c in (range(w.ncurves) if curves is None else curves):
        o0, o1 = int(w.offsets[c]), int(w.offsets[c + 1])
        if o1 == o0:
            continue
        g = g_bins[:, o0:o1]
        assert (g >= 0).all() and (g < M).all(), f"curve {c}: unwritten or out-of-range bins"
        b, e = oracle_bins(w.t[o0:o1], fr, M)
        mm = g != b
        pairs += mm.size
        mism += int(mm.sum())
        far += int((mm & (e > 1e-9)).sum())
        if mm.any():
            worst = max(worst, float(e[mm].max()))
    return pairs, mism, far, worst


def run_single(ctx, t, x, sigma, freqs, M, params=None):
    tt = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in (t, x, sigma, freqs)]
    S = torch.empty(tt[3].numel(), dtype=torch.float64, device="cuda")
    G.fpw_periodogram_ex(ctx, None, params, tt[0], tt[1], tt[2], tt[3], M, S)
    torch.cuda.synchronize()
    return S.cpu().numpy(), ctx.status()


def s_bound(x, sigma):
    return float(np.sum(x * x / (sigma * sigma)))


def assert_S_close(S_gpu, S_or, bound, *, rel=1e-4, absf=1e-7, mask=None, what=""):
    err = np.abs(S_gpu - S_or)
    tol = rel * np.abs(S_or) + absf * max(bound, 1e-300)
    # a NaN on one side only is a mismatch; NaN on both sides agrees
    bad = ~(err <= tol) & ~(np.isnan(S_gpu) & np.isnan(S_or))
    if mask is not None:
        bad &= mask
    if bad.any():
        i = int(np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0)))
        raise AssertionError(f"{what}: {int(bad.sum())} S values out of tolerance; worst at {i}: gpu {S_gpu[i]!r} "
                             f"oracle {S_or[i]!r} tol {tol[i]:.3g}")


def check_topk(g_idx, g_S, o_idx, o_S, *, rel=1e-4, abs_tol=0.0, o_dense=None, raw=False, what=""):
    """Compare one curve's GPU top-k with the oracle's extended top list
    (o_idx/o_S at least as long as k, sorted, -1/NaN padded).

    Unique parts must match: the ranked S values (within tolerance). Indices
    must equal the oracle's, unless the choice is a tie: with the oracle's dense
    periodogram, a GPU index is valid when its oracle S is within tolerance of
    the rank's value and it is a local maximum up to the tolerance (a swap among
    near-equal peaks, or a flat top whose maximum moved by one index under
    rounding); without it, the index must be within one frequency of an oracle
    peak of near-equal S."""
    k = len(g_idx)
    gv = [int(g) for g in g_idx if g >= 0]
    assert len(set(gv)) == len(gv), f"{what}: repeated indices {g_idx}"
    ov = np.where(o_idx >= 0, o_S, -np.inf)
    for j in range(k):
        oi = int(o_idx[j]) if j < len(o_idx) else -1
        g = int(g_idx[j])
        if oi < 0:
            if g >= 0:
                assert o_dense is not None and _locally_maximal(o_dense, g, rel, abs_tol, raw), \
                    f"{what}: rank {j}: gpu peak {g} where the oracle has none"
            continue
        s = ov[j]
        tol = 2 * (rel * abs(s) + abs_tol)
        assert g >= 0, f"{what}: rank {j}: gpu has no peak, oracle has {oi} (S {s})"
        assert abs(g_S[j] - s) <= tol, f"{what}: rank {j}: gpu S {g_S[j]} vs oracle S {s}"
        if g == oi:
            continue
        if o_dense is not None:
            ok = abs(o_dense[g] - s) <= tol and _locally_maximal(o_dense, g, rel, abs_tol, raw)
        else:
            ok = _near_tie_member(g, g_S[j], o_idx, ov, rel, abs_tol, target=s)
        assert ok, (f"{what}: rank {j}: gpu idx {g} (S {g_S[j]}) vs oracle idx {oi} (S {s}); "
                    f"oracle list {list(zip(o_idx.tolist(), o_S.tolist()))}")


def _locally_maximal(S, g, rel, abs_tol, raw):
    if raw:
        return True
    tol = 2 * (rel * abs(S[g]) + abs_tol)
    left = S[g - 1] if g > 0 else -np.inf
    right = S[g + 1] if g + 1 < len(S) else -np.inf
    return S[g] >= left - tol and S[g] >= right - tol


def _near_tie_member(gi, gs, o_idx, ov, rel, abs_tol, target=None):
    """gi is acceptable if an oracle peak within one frequency of it has an S
    within tolerance of the rank's S."""
    if gi < 0:
        return False
    ref = target if target is not None else gs
    for q in range(len(o_idx)):
        if o_idx[q] < 0:
            continue
        if abs(int(o_idx[q]) - int(gi)) <= 1 and abs(ov[q] - ref) <= 2 * (rel * abs(ref) + abs_tol):
            return True
    return False
