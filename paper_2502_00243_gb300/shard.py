"""Host-side sharding of the batched periodogram over several GPUs, one process
per GPU (torch.distributed ranks).

Curves are independent, so a ragged batch splits over ranks with no exchange
on the data path: rank r takes a set of whole curves chosen by the longest-
processing-time rule on the cost n_c * F (each curve, largest first, goes to
the rank with the least work so far), runs them on its own GPU, and the
per-curve top-k lists (k index + S pairs per curve) are gathered to rank 0 and
put back in curve order. One long curve splits over its frequency grid instead:
part p owns a contiguous range [lo, hi) and is evaluated on [lo - 1, hi + 1),
so every owned frequency has both neighbours for the local-maximum test of the
peak finder; each part reports its k best owned peaks, and the parts' lists
merge by S descending, ties to the lower frequency index (Section 3.5's
peaks, with the library's ranking).

Long runs can be checkpointed: `run_chunked` processes a batch chunk by chunk,
saves each finished chunk's top-k and, rerun after an interruption, skips the
chunks already saved.

The compute step is a callable so that the partition and merge logic can be
exercised without a GPU; by default it is the library's batched call.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(offsets, nfreq: int, nparts: int) -> list[np.ndarray]:
    """Curve indices per part: longest-processing-time assignment of the cost
    (n_c + 32) * nfreq (the 32 stands for a curve's fixed per-tile work), each
    part's indices in increasing order."""
    offsets = np.asarray(offsets, dtype=np.int64)
    n = offsets[1:] - offsets[:-1]
    cost = (n + 32).astype(np.float64) * float(max(nfreq, 1))
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, p) for p in range(nparts)]
    parts: list[list[int]] = [[] for _ in range(nparts)]
    for c in order:
        load, p = heapq.heappop(heap)
        parts[p].append(int(c))
        heapq.heappush(heap, (load + float(cost[c]), p))
    return [np.sort(np.asarray(q, dtype=np.int64)) for q in parts]


def subset(offsets, t, x, sigma, ids):
    """CSR arrays of the curves ``ids`` (in that order)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    spans = [(int(offsets[c]), int(offsets[c + 1])) for c in ids]
    o = np.zeros(len(spans) + 1, dtype=np.int64)
    o[1:] = np.cumsum([b - a for a, b in spans])
    cat = (lambda arr: np.concatenate([arr[a:b] for a, b in spans]) if spans else np.zeros(0, dtype=np.float64))
    return o, cat(t), cat(x), cat(sigma)


def frequency_parts(nfreq: int, nparts: int) -> list[tuple[int, int, int, int]]:
    """(lo, hi, a, b) per part: owned frequencies [lo, hi), evaluated on [a, b)
    = [lo - 1, hi + 1) clipped to the grid."""
    out = []
    for p in range(nparts):
        lo, hi = nfreq * p // nparts, nfreq * (p + 1) // nparts
        if hi > lo:
            out.append((lo, hi, max(lo - 1, 0), min(hi + 1, nfreq)))
    return out


def owned_topk(idx, S, a: int, lo: int, hi: int, k: int):
    """A part's peaks (indices local to its evaluated range starting at a)
    restricted to its owned range, as global indices; at most k kept."""
    keep = [(int(i) + a, float(s)) for i, s in zip(idx, S) if i >= 0 and lo <= int(i) + a < hi]
    return keep[:k]


def merge_topk(lists, k: int):
    """Merge (index, S) candidate lists: S descending, ties to the lower index;
    -1 / NaN padded to k."""
    pool = sorted((c for lst in lists for c in lst), key=lambda c: (-c[1], c[0]))[:k]
    idx = np.full(k, -1, dtype=np.int32)
    S = np.full(k, np.nan, dtype=np.float32)
    for j, (i, s) in enumerate(pool):
        idx[j], S[j] = i, s
    return idx, S


def library_compute(ctx, M: int, params=None):
    """Compute step on this rank's GPU: the batched call on host arrays (the
    host-buffer entry point copies them to the device), top-k back on the host."""
    import paper_2502_00243_gb300 as G

    def run(offsets, t, x, sigma, freqs, k):
        C = len(offsets) - 1
        idx = np.empty(C * k, dtype=np.int32)
        S = np.empty(C * k, dtype=np.float32)
        if C > 0:
            G.fpw_periodogram_batch_host(ctx, params, np.ascontiguousarray(offsets, dtype=np.int64),
                                         np.ascontiguousarray(t), np.ascontiguousarray(x),
                                         np.ascontiguousarray(sigma), np.ascontiguousarray(freqs), M, k, idx, S)
        return idx.reshape(C, k), S.reshape(C, k)
    return run


def _gather(dist, obj, world: int):
    if dist is None or world == 1:
        return [obj]
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out


def batch_topk_sharded(compute, offsets, t, x, sigma, freqs, k: int, rank: int = 0, world: int = 1, dist=None):
    """Per-curve top-k of a ragged batch split over `world` ranks (LPT on cost);
    every rank returns the full ``(idx [C, k], S [C, k])`` in curve order."""
    offsets = np.asarray(offsets, dtype=np.int64)
    C = len(offsets) - 1
    parts = lpt_partition(offsets, len(freqs), world)
    ids = parts[rank]
    o, tt, xx, ss = subset(offsets, t, x, sigma, ids)
    idx, S = compute(o, tt, xx, ss, freqs, k)
    got = _gather(dist, (ids, np.asarray(idx), np.asarray(S)), world)
    out_i = np.full((C, k), -1, dtype=np.int32)
    out_s = np.full((C, k), np.nan, dtype=np.float32)
    for q_ids, q_i, q_s in got:
        out_i[q_ids] = q_i
        out_s[q_ids] = q_s
    return out_i, out_s


def curve_topk_split(compute, t, x, sigma, freqs, k: int, rank: int = 0, world: int = 1, dist=None):
    """Top-k of one curve whose frequency grid is split over `world` ranks (one
    part per rank, one-frequency halo on each side); every rank returns the
    merged ``(idx [k], S [k])``."""
    freqs = np.asarray(freqs, dtype=np.float64)
    parts = frequency_parts(len(freqs), world)
    mine = []
    if rank < len(parts):
        lo, hi, a, b = parts[rank]
        o = np.array([0, len(t)], dtype=np.int64)
        idx, S = compute(o, t, x, sigma, freqs[a:b], k + 2)  # at most two halo peaks to drop
        mine = owned_topk(np.asarray(idx)[0], np.asarray(S)[0], a, lo, hi, k)
    got = _gather(dist, mine, world)
    return merge_topk(got, k)


def run_chunked(compute, offsets, t, x, sigma, freqs, k: int, chunk_curves: int, state_dir=None):
    """Per-curve top-k of a batch processed in chunks of `chunk_curves` curves.

    With `state_dir`, each finished chunk's top-k is saved there
    (``chunk_<first curve>_<count>.npz``, written to a temporary name and
    renamed, so a file is either complete or absent), and a rerun loads the
    chunks already saved instead of recomputing them: a long run interrupted
    at any point resumes where it stopped. Returns ``(idx [C, k], S [C, k])``
    in curve order."""
    import os

    offsets = np.asarray(offsets, dtype=np.int64)
    C = len(offsets) - 1
    out_i = np.full((C, k), -1, dtype=np.int32)
    out_s = np.full((C, k), np.nan, dtype=np.float32)
    if state_dir is not None:
        os.makedirs(state_dir, exist_ok=True)
    for c0 in range(0, C, max(1, int(chunk_curves))):
        ids = np.arange(c0, min(C, c0 + int(chunk_curves)), dtype=np.int64)
        path = None if state_dir is None else os.path.join(state_dir, f"chunk_{c0}_{len(ids)}.npz")
        if path is not None and os.path.exists(path):
            with np.load(path) as z:
                out_i[ids], out_s[ids] = z["idx"], z["S"]
            continue
        o, tt, xx, ss = subset(offsets, t, x, sigma, ids)
        idx, S = compute(o, tt, xx, ss, freqs, k)
        out_i[ids], out_s[ids] = idx, S
        if path is not None:
            tmp = path + ".tmp.npz"
            np.savez(tmp, idx=np.asarray(idx, dtype=np.int32), S=np.asarray(S, dtype=np.float32))
            os.replace(tmp, path)
    return out_i, out_s
