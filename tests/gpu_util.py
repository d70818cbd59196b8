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
    bad = err > tol
    if mask is not None:
        bad &= mask
    if bad.any():
        i = int(np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0)))
        raise AssertionError(f"{what}: {int(bad.sum())} S values out of tolerance; worst at {i}: gpu {S_gpu[i]!r} "
                             f"oracle {S_or[i]!r} tol {tol[i]:.3g}")


def check_topk(g_idx, g_S, o_idx, o_S, *, rel=1e-4, abs_tol=0.0, o_dense=None, what=""):
    """Compare one curve's GPU top-k with the oracle's extended top list
    (o_idx/o_S longer than k, sorted, -1/NaN padded)."""
    k = len(g_idx)
    valid = o_idx >= 0
    ov = np.where(valid, o_S, -np.inf)
    for j in range(k):
        oi = int(o_idx[j]) if j < len(o_idx) else -1
        if oi < 0:
            assert g_idx[j] == -1 or _near_tie_member(g_idx[j], g_S[j], o_idx, ov, rel, abs_tol, o_dense), \
                f"{what}: rank {j}: gpu has peak {g_idx[j]} where the oracle has none"
            continue
        s = ov[j]
        tol = rel * abs(s) + abs_tol
        sep_prev = j == 0 or ov[j - 1] - s > tol
        sep_next = (j + 1 >= len(ov)) or (s - ov[j + 1] > tol)
        if sep_prev and sep_next and g_idx[j] == oi:
            pass
        elif not _near_tie_member(g_idx[j], g_S[j], o_idx, ov, rel, abs_tol, o_dense, target=s):
            raise AssertionError(f"{what}: rank {j}: gpu idx {g_idx[j]} (S {g_S[j]}) vs oracle idx {oi} (S {s}); "
                                 f"oracle list {list(zip(o_idx.tolist(), o_S.tolist()))}")
        if g_idx[j] >= 0 and o_dense is not None:
            sg = o_dense[g_idx[j]]
            assert abs(g_S[j] - sg) <= rel * abs(sg) + abs_tol, f"{what}: S at {g_idx[j]}: gpu {g_S[j]} oracle {sg}"


def _near_tie_member(gi, gs, o_idx, ov, rel, abs_tol, o_dense, target=None):
    """gi is acceptable if an oracle peak within one frequency of it has an S
    within tolerance of the rank's S (a swap among near-ties, or a flat top
    whose maximum moved by one index under rounding)."""
    if gi < 0:
        return False
    ref = target if target is not None else gs
    for q in range(len(o_idx)):
        if o_idx[q] < 0:
            continue
        if abs(int(o_idx[q]) - int(gi)) <= 1 and abs(ov[q] - ref) <= 2 * (rel * abs(ref) + abs_tol):
            return True
    return False
