"""Autotuner for the FPW tile kernel's shape.

For each (bin count M, curve-size bucket) it times candidate shapes on
synthetic light curves through the C ABI (the library's own timing hook: CUDA
events around the tile kernel on its stream) and installs the fastest in a
context's shape table (``fpw_ctx_set_shape``), in two stages: threads per block
x frequencies per thread, then, for the best of those, the observations staged
per pass (which set the blocks per SM) x the work items per resident block
(the segment size of the persistent schedule's curve-to-block mapping).
``tune`` measures synthetic curves of one size per bucket; ``tune_batch``
measures a size-stratified sample of a workload's own curves. The table can
be saved to / loaded from JSON.

Shapes matter because the kernel is bound by the shared-memory pipe: every
(thread, frequency) slot holds M (A, B) bin pairs, so M and the frequencies
per thread R decide how many warps fit per SM (latency hiding) and how many
per-observation broadcast loads are amortised (R).
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import Context, FPWError, fpw_params_default, fpw_periodogram_batch_ex

CANDIDATES = ((128, 8), (128, 6), (128, 5), (128, 4), (128, 3), (128, 2), (128, 1), (256, 4), (256, 2), (256, 1),
              (64, 8), (64, 4), (192, 2))
SCHEDULES = ((0, 8), (0, 4), (0, 16), (128, 8), (256, 8), (512, 8))  # (observations per pass, items per resident block)
DEFAULT_MS = (10, 20, 50)
DEFAULT_BUCKETS = ((0, 300), (300, 1000), (1000, 1 << 40))


def m_ranges(Ms):
    """Split [1, inf) into one M range per tuned M (boundaries at midpoints)."""
    Ms = sorted(set(int(m) for m in Ms))
    out = []
    for i, m in enumerate(Ms):
        lo = 1 if i == 0 else (Ms[i - 1] + m) // 2 + 1
        hi = (1 << 30) if i == len(Ms) - 1 else (m + Ms[i + 1]) // 2
        out.append((m, lo, hi))
    return out


def typical_n(lo, hi):
    hi = min(hi, 3000)
    lo = max(lo, 50)
    return int(round(math.sqrt(lo * hi))) if hi > lo else lo


def synthetic_curves(n, ncurves, seed=0):
    """Random light curves of n observations each (times over 1000 d)."""
    rng = np.random.default_rng(seed)
    offsets = np.arange(ncurves + 1, dtype=np.int64) * n
    t = np.sort(rng.uniform(0.0, 1000.0, (ncurves, n)), axis=1).ravel()
    sigma = np.exp(rng.uniform(np.log(0.01), np.log(0.3), ncurves * n))
    x = rng.normal(0.0, 1.0, ncurves * n) * sigma
    return offsets, t, x, sigma


def measure(ctx, dev, offsets_h, freqs, M, k, T, R, reps=2, NC=0, items=0):
    """Mean tile-kernel milliseconds for one shape, or None if it does not fit."""
    import torch
    C = offsets_h.shape[0] - 1
    idx = torch.empty(C * k, dtype=torch.int32, device="cuda")
    S = torch.empty(C * k, dtype=torch.float32, device="cuda")
    p = fpw_params_default(threads=T, freqs_per_thread=R, obs_chunk=NC, items_per_slot=items)
    try:
        fpw_periodogram_batch_ex(ctx, None, p, dev[0], offsets_h, dev[1], dev[2], dev[3], freqs, M, k, idx, S)
        torch.cuda.synchronize()
        ctx.set_timing(True)
        ctx.kernel_time()
        for _ in range(reps):
            fpw_periodogram_batch_ex(ctx, None, p, dev[0], offsets_h, dev[1], dev[2], dev[3], freqs, M, k, idx, S)
        torch.cuda.synchronize()
        ms, n = ctx.kernel_time()
    except FPWError:
        return None
    finally:
        ctx.set_timing(False)
    return ms / max(n, 1)


def tune(ctx: Context, Ms=DEFAULT_MS, buckets=DEFAULT_BUCKETS, *, nfreq=50_000, evals_per_case=1.5e10, k=5,
         candidates=CANDIDATES, schedules=SCHEDULES, apply=True, log=None):
    """Measure every candidate shape per (M, bucket); returns the table entries
    (and installs them in ``ctx`` when ``apply``)."""
    import torch
    freqs = torch.linspace(0.01, 50.0, nfreq, dtype=torch.float64, device="cuda")
    entries = []
    for M, m_lo, m_hi in m_ranges(Ms):
        for b_lo, b_hi in buckets:
            n = typical_n(b_lo, b_hi)
            ncurves = max(8, int(evals_per_case / (n * nfreq)))
            off, t, x, s = synthetic_curves(n, ncurves, seed=M * 7919 + n)
            dev = [torch.from_numpy(a).cuda() for a in (off, t, x, s)]
            evals = float(off[-1]) * nfreq
            best = None
            for T, R in candidates:
                ms = measure(ctx, dev, off, freqs, M, k, T, R)
                if ms is None:
                    continue
                rate = evals / (ms / 1e3)
                if log:
                    log(f"M={M} n={n} T={T} R={R}: {rate / 1e9:.1f} Geval/s")
                if best is None or rate > best[2]:
                    best = (T, R, rate)
            if best is None:
                continue
            sched = (0, 0, best[2])
            for NC, items in schedules:
                ms = measure(ctx, dev, off, freqs, M, k, best[0], best[1], NC=NC, items=items)
                if ms is None:
                    continue
                rate = evals / (ms / 1e3)
                if log:
                    log(f"M={M} n={n} T={best[0]} R={best[1]} NC={NC} items={items}: {rate / 1e9:.1f} Geval/s")
                if rate > sched[2]:
                    sched = (NC, items, rate)
            e = {"M_lo": m_lo, "M_hi": m_hi, "n_lo": int(b_lo), "n_hi": int(min(b_hi, 1 << 40)), "threads": best[0],
                 "freqs_per_thread": best[1], "obs_chunk": sched[0], "items_per_slot": sched[1],
                 "geval_s": sched[2] / 1e9, "M": M, "n": n}
            entries.append(e)
    if apply:
        install(ctx, entries)
    return entries


def n_typical(offsets_h) -> int:
    """The observation-weighted mean curve size sum(n^2) / sum(n) of a batch:
    the curve-size key under which the library looks a batch up in the shape
    table."""
    n = np.diff(np.asarray(offsets_h, dtype=np.int64)).astype(np.float64)
    s = float(n.sum())
    return int(float((n * n).sum()) / s) if s > 0 else 0


def stratified_sample(offsets_h, t, x, sigma, ncurves):
    """Up to ``ncurves`` curves of a host batch taken evenly through its curves
    sorted by size (so the sample keeps the batch's size mix), as a new host
    batch (offsets, t, x, sigma)."""
    off = np.asarray(offsets_h, dtype=np.int64)
    C = off.shape[0] - 1
    order = np.argsort(np.diff(off), kind="stable")
    pick = order[np.linspace(0, C - 1, min(ncurves, C)).round().astype(np.int64)] if C > 0 else order
    pick = np.unique(pick)
    sizes = off[pick + 1] - off[pick]
    sub_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rows = np.concatenate([np.arange(off[c], off[c + 1]) for c in pick]) if pick.size else np.zeros(0, np.int64)
    return sub_off, np.asarray(t)[rows], np.asarray(x)[rows], np.asarray(sigma)[rows]


def tune_batch(ctx: Context, offsets_h, t, x, sigma, f_lo: float, f_hi: float, Ms, *, k=5, sample_curves=4000,
               nfreq=20_000, candidates=CANDIDATES, schedules=SCHEDULES, apply=True, log=None):
    """Tune the shape on a workload's own curves rather than on curves of one
    size: a batch whose sizes are spread (e.g. 100 to 3000 observations) can
    favour another shape than uniform curves of its typical size. Times every
    candidate (then every schedule for the best) on a size-stratified sample
    of the host batch over ``nfreq`` linear frequencies in [f_lo, f_hi], for
    each bin count in ``Ms``, and installs one entry per M covering curve sizes
    within a factor of two of the batch's typical size (later entries take
    precedence, so these override a generic table for such batches)."""
    import torch
    nt = n_typical(offsets_h)
    off, ts, xs, ss = stratified_sample(offsets_h, t, x, sigma, sample_curves)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (off, ts, xs, ss)]
    freqs = torch.linspace(float(f_lo), float(f_hi), nfreq, dtype=torch.float64, device="cuda")
    evals = float(off[-1]) * nfreq
    entries = []
    for M in sorted(set(int(m) for m in Ms)):
        best = None
        for T, R in candidates:
            ms = measure(ctx, dev, off, freqs, M, k, T, R)
            if ms is None:
                continue
            rate = evals / (ms / 1e3)
            if log:
                log(f"batch M={M} T={T} R={R}: {rate / 1e9:.1f} Geval/s")
            if best is None or rate > best[2]:
                best = (T, R, rate)
        if best is None:
            continue
        sched = (0, 0, best[2])
        for NC, items in schedules:
            ms = measure(ctx, dev, off, freqs, M, k, best[0], best[1], NC=NC, items=items)
            if ms is None:
                continue
            rate = evals / (ms / 1e3)
            if rate > sched[2]:
                sched = (NC, items, rate)
        entries.append({"M_lo": M, "M_hi": M, "n_lo": nt // 2, "n_hi": 2 * nt + 1, "threads": best[0],
                        "freqs_per_thread": best[1], "obs_chunk": sched[0], "items_per_slot": sched[1],
                        "geval_s": sched[2] / 1e9, "M": M, "n": nt, "sample_curves": int(off.shape[0] - 1)})
    if apply:
        install(ctx, entries)
    return entries


def install(ctx: Context, entries) -> None:
    for e in entries:
        ctx.set_shape(e["M_lo"], e["M_hi"], e["n_lo"], e["n_hi"], e["threads"], e["freqs_per_thread"],
                      e.get("obs_chunk", 0), e.get("items_per_slot", 0))


def save(entries, path: str) -> None:
    with open(path, "w") as fh:
        json.dump({"version": 1, "entries": entries}, fh, indent=1)


def load(path: str):
    with open(path) as fh:
        data = json.load(fh)
    return data["entries"]
