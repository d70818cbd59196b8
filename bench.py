#!/usr/bin/env python3
"""Throughput benchmark of the GB300 FPW periodogram.

Workload (one "step" = one pass of the whole hot path over one batch): the
10^5-curve sweep -- curves with N log-uniform in [100, 3000] and ZTF-like
cadence, mixed waveforms, M phase bins (default 20), 5*10^5 linear trial
frequencies 0.01-50 1/d, per-curve top-5 peaks -- split into ten batches of
10^4 curves; step s processes batch (s * world + rank) mod 10, so the default
ten timed steps on one GPU cover the whole sweep once. Inputs are synthetic
(seeded) and larger than L2 per batch.

Reported: evaluations (observation x frequency pairs) per second for the whole
job, the tile kernel's roofline fraction, an end-to-end number through the
host-buffer C entry point, the FP64 CPU oracle on a bounded sample
(cpu_baseline), the plain binary64 one-curve-per-launch GPU form and the
batched call on the same stratified curve sample (their ratio is the speed-up),
and, in `per_M`, the same sweep at the other bin counts of the throughput
sweep (M = 10 and 50), each over one pass of the 1e5 curves.

--impl reference times the FP64 CPU oracle instead (each step a bounded sample
of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "obs×freq FPW evals/s on 1 GB300 (batched split-prec vs plain FP64), % roofline"
UNIT = "evals/s"
WORKLOAD = "sweep_100k"
NSM_NOMINAL = 152
SM_MAX_MHZ_NOMINAL = 2070.0
SMEM_EVALS_PER_CLK_SM = 8  # 16 B (A, B) read-modify-write per evaluation at 128 B/clk/SM
KERNELS_PER_STEP = 5  # prep, tile_dev, tile, merge, latch
SWEEP_MS = (10, 20, 50)  # bin counts of the throughput sweep
ENTROPY_INST_PER_EVAL = 9.86  # thread instructions per evaluation of the dense phase-entropy kernel (ncu, M = 20)


def entropy_R(M: int) -> int:
    """Frequencies per thread of the dense phase-entropy kernel at M bins (the
    library's launch rule)."""
    return 8 if M <= 12 else (4 if M <= 24 else (2 if M <= 96 else 1))
# DRAM bytes (read + write) of one tile-kernel launch at M = 20, from an ncu capture of a 1e4-curve sweep
# batch over 2e4 frequencies (dram__bytes_read.sum + dram__bytes_write.sum). The kernel reads each curve
# from DRAM once per launch (t and the staged weights, about 16.7 B per observation; per-tile re-reads
# hit L2), so a full launch adds only the larger grid (8 B per extra frequency). Valid only for the
# kernel source it was measured on (sha256 prefix of the tile-kernel sources, tile_source_hash).
TILE_TRAFFIC = {"source_sha256_16": "ce9276e3f4830ec5", "bytes": 142.63e6, "nfreq": 20_000}


# ---------------------------------------------------------------- workload generation (spawned workers)
def _gen_chunk(args):
    lo, hi, M = args
    import lightcurves as L
    w = L.make(WORKLOAD, range(lo, hi), M=M, nfreq=2)
    return lo, w.offsets, w.t, w.x, w.sigma


def make_batches(batch_ids, batch_curves, M, workers):
    """Host arrays for each batch id: dict b -> (offsets, t, x, sigma)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    chunk = 500
    tasks = []
    for b in batch_ids:
        for lo in range(b * batch_curves, (b + 1) * batch_curves, chunk):
            tasks.append((lo, min(lo + chunk, (b + 1) * batch_curves), M))
    parts = {}
    if workers > 1:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            for lo, off, t, x, s in ex.map(_gen_chunk, tasks):
                parts[lo] = (off, t, x, s)
    else:
        for tsk in tasks:
            lo, off, t, x, s = _gen_chunk(tsk)
            parts[lo] = (off, t, x, s)
    out = {}
    for b in batch_ids:
        los = list(range(b * batch_curves, (b + 1) * batch_curves, chunk))
        offs, ts, xs, ss, base = [np.zeros(1, dtype=np.int64)], [], [], [], 0
        for lo in los:
            off, t, x, s = parts[lo]
            offs.append(off[1:] + base)
            base += int(off[-1])
            ts.append(t)
            xs.append(x)
            ss.append(s)
        out[b] = (np.concatenate(offs), np.concatenate(ts), np.concatenate(xs), np.concatenate(ss))
    return out


def stratified(offsets, count):
    """Curve indices spread evenly over the batch sorted by size."""
    import numpy as np
    n = offsets[1:] - offsets[:-1]
    order = np.argsort(n, kind="stable")
    pick = np.linspace(0, len(order) - 1, min(count, len(order))).round().astype(int)
    return np.sort(order[pick])


def subset(batch, ids):
    import numpy as np
    off, t, x, s = batch
    parts = [(off[i], off[i + 1]) for i in ids]
    o = np.zeros(len(ids) + 1, dtype=np.int64)
    o[1:] = np.cumsum([b - a for a, b in parts])
    cat = lambda arr: np.concatenate([arr[a:b] for a, b in parts]) if parts else np.zeros(0)
    return o, cat(t), cat(x), cat(s)


# ---------------------------------------------------------------- multi-GPU: curves shard across ranks
def shard_batches(steps, world, rank, nbatches):
    """Batch processed by this rank at each step: (step * world + rank) mod nbatches.
    Ranks take disjoint batches within a step (weak scaling: per-rank work is fixed)."""
    return [(s * world + rank) % nbatches for s in range(steps)]


def reduce_timing(dist, device, elapsed_ms, evals):
    """Across ranks: the max elapsed time and the summed evaluations (no data-path collective)."""
    import torch
    if dist is None:
        return elapsed_ms, evals
    tt = torch.tensor([elapsed_ms, evals], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- helpers
def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peak_bf16_tflops():
    """Measured dense bf16 burst peak (fp16 runs at the same nominal rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0  # earlier GB300 measurement


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh).get("sm_max_mhz", SM_MAX_MHZ_NOMINAL))
    except (OSError, ValueError):
        return SM_MAX_MHZ_NOMINAL


def tile_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("fpw_tile.cuh", "fpw_tile.cu", "fpw_tile_f32.cu", "fpw_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2502_00243_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def tile_traffic(nfreq):
    """DRAM bytes per tile-kernel launch of the timed workload, or None when the
    kernel source changed since the counters were taken."""
    if TILE_TRAFFIC["bytes"] is None or tile_source_hash() != TILE_TRAFFIC["source_sha256_16"]:
        return None
    return TILE_TRAFFIC["bytes"] + 8.0 * (nfreq - TILE_TRAFFIC["nfreq"])


def grid(args):
    import numpy as np
    return np.linspace(0.01, 50.0, args.nfreq, dtype=np.float64)


def config_block(args, nbatches, batch_evals_mean):
    return {"workload": f"{WORKLOAD}: 1e5 ZTF-like curves, N log-uniform 100-3000, mixed waveforms, M={args.M}, "
                        f"{args.nfreq:.0e} linear freqs 0.01-50 1/d, top-{args.k}; one step = one batch of {args.batch_curves} "
                        f"curves ({nbatches} batches)",
            "curves_per_step": args.batch_curves, "nfreq": args.nfreq, "M": args.M, "k": args.k,
            "phase": "fixed64 (exact integer anchor + 64-bit stepping)", "bin_sums": "f32",
            "evals_per_step_mean": batch_evals_mean,
            "l2": (f"inputs larger than L2: {batch_evals_mean / args.nfreq * 24 / 1e6:.0f} MB of float64 t, x, sigma "
                   f"per batch against 129 MB of L2, a distinct batch each step" if batch_evals_mean
                   else "host run (no device caches)")}


def oracle_rate(batch, ids, F_grid, M, k, nthreads):
    import numpy as np

    import oracle
    o, t, x, s = subset(batch, ids)
    t0 = time.perf_counter()
    oracle.fpw_batch(o, t, x, s, F_grid, M, dense=False, k=k, nthreads=nthreads)
    dt = time.perf_counter() - t0
    ev = float(o[-1]) * F_grid.shape[0]
    return ev, dt


def oracle_sample(batch, F_grid, M, k, target_s, cores):
    """A bounded oracle sample of about target_s seconds: curves stratified by
    N, a multiple of the core count (threads take whole curves), and the full
    frequency grid; or, where `cores` curves over the full grid already take
    longer, those curves over a central slice of the grid."""
    import math
    ids = stratified(batch[0], cores)
    o = subset(batch, ids)[0]
    probe_ids = stratified(batch[0], 4 * cores)  # several curves per thread: balanced like the sample
    probe_F = F_grid[: max(1000, F_grid.shape[0] // 200)]
    oracle_rate(batch, probe_ids, probe_F[:100], M, k, cores)  # first call: library load, thread start-up
    ev, dt = oracle_rate(batch, probe_ids, probe_F, M, k, cores)
    rate = ev / max(dt, 1e-6)
    full_s = float(o[-1]) * F_grid.shape[0] / rate
    if full_s < target_s:
        ncurves = len(batch[0]) - 1
        per_curve = float(batch[0][-1]) / max(ncurves, 1) * F_grid.shape[0]  # mean evaluations per curve
        q = max(1, min(ncurves // cores, math.ceil(target_s * rate / max(per_curve, 1.0) / cores)))
        return stratified(batch[0], cores * q), F_grid
    nf = int(max(1000, min(F_grid.shape[0], target_s * rate / max(float(o[-1]), 1.0))))
    start = (F_grid.shape[0] - nf) // 2
    return ids, F_grid[start:start + nf]


# ---------------------------------------------------------------- reference arm: the CPU oracle
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import numpy as np

    import lightcurves as L
    cores = os.cpu_count() or 1
    nb = args.curves_total // args.batch_curves
    steps = args.warmup + args.steps
    ids = sorted({s % nb for s in range(steps)})
    batches = make_batches(ids, args.batch_curves, args.M, workers=min(cores, 16))
    F_grid = grid(args)
    pick0, F_s = oracle_sample(batches[ids[0]], F_grid, args.M, args.k, args.ref_step_seconds, cores)
    n_pick = len(pick0)
    total_ev, total_t = 0.0, 0.0
    for s in range(steps):
        b = batches[s % nb]
        pick = stratified(b[0], n_pick)
        ev, dt = oracle_rate(b, pick, F_s, args.M, args.k, cores)
        if s >= args.warmup:
            total_ev += ev
            total_t += dt
    value = total_ev / total_t
    sample = (f"{n_pick} curves per step, stratified by N from the step's {args.batch_curves}-curve batch, x "
              f"{F_s.shape[0]} of the {F_grid.shape[0]} grid frequencies, M={args.M}, top-{args.k}, {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_block(args, nb, None), phase="binary64 fl(t f)", bin_sums="f64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def shape_label(ctx, M):
    T, R, NC, grid = ctx.last_shape()
    return f"tile_kernel<R={R}, fixed64, f32 sums> T={T} obs_chunk={NC} grid={grid} (M={M})"


def run_gb300(args):
    import numpy as np
    import torch

    rank, world, local_rank = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(local_rank)
    import paper_2502_00243_gb300 as G
    G.lib()  # fail loudly if the library is missing

    cores = os.cpu_count() or 1
    nb = args.curves_total // args.batch_curves
    steps = args.warmup + args.steps
    batch_of = shard_batches(steps, world, rank, nb)
    other_Ms = [m for m in SWEEP_MS if m != args.M] if not args.no_per_m else []
    pm_steps, pm_warm = min(args.steps, nb), min(args.warmup, 2)
    pm_batch_of = shard_batches(pm_warm + pm_steps, world, rank, nb)
    ids = sorted(set(batch_of) | (set(pm_batch_of) if other_Ms else set()))
    workers = max(1, min(16, cores // max(1, min(world, cores))))
    t_gen = time.perf_counter()
    host = make_batches(ids, args.batch_curves, args.M, workers=workers)
    t_gen = time.perf_counter() - t_gen
    F_grid = grid(args)
    F = F_grid.shape[0]
    dev = {b: dict(offsets=torch.from_numpy(h[0]).cuda(), t=torch.from_numpy(h[1]).cuda(),
                   x=torch.from_numpy(h[2]).cuda(), sigma=torch.from_numpy(h[3]).cuda()) for b, h in host.items()}
    freqs = torch.from_numpy(F_grid).cuda()
    C, k = args.batch_curves, args.k
    idx = torch.empty(C * k, dtype=torch.int32, device="cuda")
    Sk = torch.empty(C * k, dtype=torch.float32, device="cuda")
    ctx = G.Context(local_rank)
    tuned = None
    if not args.no_autotune:  # a few seconds: shapes and schedules for the bin counts timed below
        from paper_2502_00243_gb300 import autotune
        t_tune = time.perf_counter()
        h0 = host[batch_of[0]]  # a size-stratified sample of the workload's own curves
        tuned = {"entries": autotune.tune_batch(ctx, h0[0], h0[1], h0[2], h0[3], float(F_grid[0]),
                                                float(F_grid[-1]), (args.M, *other_Ms), k=k),
                 "on": f"a size-stratified sample of batch {batch_of[0]}'s curves over 2e4 linear frequencies "
                       f"spanning the grid"}
        tuned["seconds"] = round(time.perf_counter() - t_tune, 1)
    params = G.fpw_params_default()
    stream = torch.cuda.current_stream()
    nsm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak = nsm * sm_max_mhz() * 1e6 * SMEM_EVALS_PER_CLK_SM / 1e9

    def step(b, M):
        d = dev[b]
        G.fpw_periodogram_batch_ex(ctx, stream, params, d["offsets"], host[b][0], d["t"], d["x"], d["sigma"], freqs,
                                   M, k, idx, Sk)
        return float(host[b][0][-1]) * F

    def timed_steps(M, order, warm):
        """Warm-up, then the timed steps bracketed by barriers and device
        syncs; CUDA events on the launching stream for the whole region and
        (library hook) around each tile-kernel launch; clocks sampled during it."""
        for b in order[:warm]:
            step(b, M)
        torch.cuda.synchronize()
        if ctx.status() != 0:
            raise RuntimeError("device status error during warm-up")
        ctx.set_timing(True)
        ctx.kernel_time()
        clocks = ClockSampler(local_rank) if rank == 0 else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        evals = 0.0
        for b in order[warm:]:
            evals += step(b, M)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        kern_ms, launches = ctx.kernel_time()
        ctx.set_timing(False)
        status = ctx.status()
        if status != 0:
            raise RuntimeError(f"device status {status} in the timed region")
        ms_max, evals_all = reduce_timing(dist, "cuda", ms, evals)
        return dict(ms=ms_max, evals_all=evals_all, evals=evals, kern_ms=kern_ms, launches=launches, clk=clk,
                    label=shape_label(ctx, M))

    head = timed_steps(args.M, batch_of, args.warmup)
    value = head["evals_all"] / (head["ms"] / 1e3)
    kern_ms, launches = head["kern_ms"], head["launches"]

    # ---- end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        pinned = {}
        for b in sorted(set(batch_of)):
            arrs = []
            for a in host[b]:
                p = torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, pin_memory=True)
                p.numpy()[...] = a
                arrs.append(p)
            pinned[b] = arrs
        fp = torch.empty(F, dtype=torch.float64, pin_memory=True)
        fp.numpy()[...] = F_grid
        oi = torch.empty(C * k, dtype=torch.int32, pin_memory=True)
        os_ = torch.empty(C * k, dtype=torch.float32, pin_memory=True)

        def hstep(s):
            b = batch_of[s]
            o, t, x, sg = (p.numpy() for p in pinned[b])
            G.fpw_periodogram_batch_host(ctx, params, o, t, x, sg, fp.numpy(), args.M, k, oi.numpy(), os_.numpy())
            return float(o[-1]) * F, 8 * (o.size + 3 * t.size + F), 8 * C * k

        for s in range(min(args.warmup, 2)):
            hstep(s)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ev_h, h2d, d2h = 0.0, 0, 0
        for s in range(args.warmup, steps):
            e_, hb, db = hstep(s)
            ev_h += e_
            h2d += hb
            d2h += db
        dt = time.perf_counter() - t0
        dt, ev_h = reduce_timing(dist, "cuda", dt, ev_h)
        e2e = {"value": ev_h / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
               "d2h_bytes_per_step": int(d2h // args.steps), "api": "fpw_periodogram_batch_host"}

    # ---- the plain binary64 one-curve-per-launch GPU form and the batched call on the same curve sample
    def plain_vs_batched(M):
        b0 = batch_of[0]
        pick = stratified(host[b0][0], args.plain_curves)
        o, t, x, sg = subset(host[b0], pick)
        dp = [torch.from_numpy(a).cuda() for a in (o, t, x, sg)]
        pi = torch.empty(len(pick) * k, dtype=torch.int32, device="cuda")
        ps = torch.empty(len(pick) * k, dtype=torch.float32, device="cuda")

        def rate(pp, reps):
            G.fpw_periodogram_batch_ex(ctx, stream, pp, dp[0], o, dp[1], dp[2], dp[3], freqs, M, k, pi, ps)
            torch.cuda.synchronize()
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(reps):
                G.fpw_periodogram_batch_ex(ctx, stream, pp, dp[0], o, dp[1], dp[2], dp[3], freqs, M, k, pi, ps)
            q1.record(stream)
            torch.cuda.synchronize()
            return reps * float(o[-1]) * F / (q0.elapsed_time(q1) / 1e3)

        pval = rate(G.fpw_params_default(phase_mode=G.FPW_PHASE_FP64), 1)
        bval = rate(params, 5)
        return {"value": pval, "unit": UNIT, "sample": f"{len(pick)} curves stratified by N from batch {b0}, "
                f"full grid, M={M}, one launch per curve (+1 top-k launch)", "batched_same_sample": bval,
                "speedup_of_batched_split": bval / pval,
                "speedup_vs_sweep_value": None}

    plain = None
    if not args.no_plain:
        plain = plain_vs_batched(args.M)
        plain["speedup_vs_sweep_value"] = value / plain["value"]

    # ---- the other bin counts of the throughput sweep: one pass over the 1e5 curves each
    per_M = {}
    for M in other_Ms:
        r = timed_steps(M, pm_batch_of, pm_warm)
        v = r["evals_all"] / (r["ms"] / 1e3)
        ach = r["evals"] / (r["kern_ms"] / 1e3) / 1e9 if r["kern_ms"] > 0 else None
        ent = {"value": v, "unit": UNIT, "steps": pm_steps, "warmup": pm_warm,
               "ms_per_step": r["ms"] / pm_steps, "kernel_ms_avg": r["kern_ms"] / max(r["launches"], 1),
               "roofline_frac": (ach / peak) if ach else None, "achieved": ach, "peak": peak, "unit_roofline": "Geval/s",
               "kernel": r["label"], "clocks": r["clk"]}
        if not args.no_plain:
            pv = plain_vs_batched(M)
            ent["plain_fp64"] = pv["value"]
            ent["batched_same_sample"] = pv["batched_same_sample"]
            ent["speedup_of_batched_split"] = pv["speedup_of_batched_split"]
        per_M[str(M)] = ent

    # ---- CPU oracle on a bounded sample (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        b0 = batch_of[0]
        pick, F_s = oracle_sample(host[b0], F_grid, args.M, k, args.cpu_seconds, cores)
        ev, dt = oracle_rate(host[b0], pick, F_s, args.M, k, cores)
        # one core: the sample's median-N curve over the first 2e5 grid frequencies (about 1 s)
        o_b = host[b0][0]
        n_pick = o_b[np.asarray(pick) + 1] - o_b[np.asarray(pick)]
        one = [int(np.asarray(pick)[np.argsort(n_pick, kind="stable")[len(pick) // 2]])]
        ev1, dt1 = oracle_rate(host[b0], one, F_s[:200_000], args.M, k, 1)
        cpu = {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(pick)} curves stratified by N from batch {b0} x {F_s.shape[0]} of the {F} grid "
                         f"frequencies, M={args.M}, top-{k}, {cores} threads ({ev:.3g} evals in {dt:.1f} s)",
               "single_core_value": ev1 / dt1,
               "single_core_sample": f"curve {one[0]} of batch {b0} (the sample's median N) x the first "
                                     f"{min(200_000, F_s.shape[0])} of those frequencies, one thread"}

    if rank == 0:
        achieved = head["evals"] / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else None
        roof = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "Geval/s",
                "frac": (achieved / peak) if achieved else None, "traffic": tile_traffic(F),
                "kernel": head["label"], "launches": launches,
                "kernel_ms_avg": kern_ms / max(launches, 1),
                "peak_basis": f"shared-memory pipe: one 8 B load + one 8 B store of the (A,B) bin pair per "
                              f"evaluation at 128 B/clk/SM -> {SMEM_EVALS_PER_CLK_SM} evals/clk/SM x {nsm} SMs x "
                              f"{sm_max_mhz():.0f} MHz (recipe unit counts and max clock); the per-evaluation "
                              f"instruction issue bound is higher"}
        mean_ev = float(np.mean([float(host[b][0][-1]) * F for b in sorted(set(batch_of))]))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_block(args, nb, mean_ev), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": head["clk"], "plain_fp64": plain,
                "per_M": per_M or None, "gen_seconds": round(t_gen, 2), "autotuned": tuned}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- per-workload report
def timed_batch(ctx, w, M, k, params, reps=3):
    """Evaluations/s of the batched call (whole call and tile kernel) and its ms."""
    import torch

    import paper_2502_00243_gb300 as G
    d = [torch.from_numpy(a).cuda() for a in (w.offsets, w.t, w.x, w.sigma, w.freqs)]
    C = w.ncurves
    idx = torch.empty(max(C * k, 1), dtype=torch.int32, device="cuda")
    S = torch.empty(max(C * k, 1), dtype=torch.float32, device="cuda")
    call = lambda: G.fpw_periodogram_batch_ex(ctx, None, params, d[0], w.offsets, d[1], d[2], d[3], d[4], M, k,
                                              idx if k else None, S if k else None)
    call()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    kms, n = ctx.kernel_time()
    ctx.set_timing(False)
    ev = float(w.offsets[-1]) * w.nfreq
    kern = ev / (kms / n / 1e3) if n > 0 and kms > 0 else None
    return ev / (e0.elapsed_time(e1) / reps / 1e3), kern, e0.elapsed_time(e1) / reps


def run_configs(args):
    """One JSON line per workload: device-resident evaluations/s of the batched
    fixed64 path (tile-kernel time and whole-call time), and the plain binary64
    form where it is cheap enough to time."""
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    torch.cuda.set_device(0)
    ctx = G.Context(0)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = nsm * sm_max_mhz() * 1e6 * SMEM_EVALS_PER_CLK_SM

    timed = lambda w, M, k, params, reps=3: timed_batch(ctx, w, M, k, params, reps)

    want = lambda sec: args.configs in ("all", sec)
    cases = []
    if want("batch"):
        cases = [("single_plain", L.make("single_plain"), 10), ("single_ztf", L.make("single_ztf"), 20),
                 ("ragged_10k", L.make("ragged_10k"), 20), ("precision", L.make("precision", range(20)), 20)]
        for M in (10, 20, 50):
            cases.append((f"sweep_100k/M={M} (batch of 1e4 curves)", L.make("sweep_100k", range(10_000), M=M), M))
    for name, w, M in cases:
        call_rate, kern_rate, ms = timed(w, M, w.k, G.fpw_params_default())
        line = {"config": name, "curves": w.ncurves, "nobs": int(w.offsets[-1]), "nfreq": w.nfreq, "M": M,
                "evals": float(w.offsets[-1]) * w.nfreq, "ms_per_call": ms, "evals_per_s_call": call_rate,
                "evals_per_s_tile_kernel": kern_rate, "roofline_frac": (kern_rate / peak) if kern_rate else None}
        if w.evals() <= 2e10:
            pr, _, _ = timed(w, M, w.k, G.fpw_params_default(phase_mode=G.FPW_PHASE_FP64), reps=1)
            line["plain_fp64_evals_per_s"] = pr
        if w.evals() <= 1e11:  # small calls: launch overhead matters, so replay a captured CUDA graph
            gr, _, gms = timed(w, M, w.k, G.fpw_params_default(use_graph=1), reps=20)
            line["graph_ms_per_call"] = gms
            line["graph_evals_per_s_call"] = gr
        print(json.dumps(line), flush=True)

    if want("accum"):
        run_configs_accum(ctx, peak)
    if want("shared"):
        run_configs_shared(ctx, peak)
    if want("drift"):
        run_configs_drift(ctx, peak)
    if want("multi"):
        run_configs_multi(ctx, peak)
    if want("entropy"):
        run_configs_entropy(ctx, peak)
    ctx.close()
    return 0


def run_configs_accum(ctx, peak):
    """The bin-sum modes on one 1e4-curve batch of the sweep at M = 20: FP32
    sums, compensated FP32 sums (16-byte bins, two-sum per addition) and
    binary64 sums; tile-kernel rate and roofline fraction of each (the roof is
    the 8-byte bin pair's; 16-byte bins halve it)."""
    import lightcurves as L
    import paper_2502_00243_gb300 as G
    w = L.make("sweep_100k", range(10_000), M=20)
    for name, acc in (("f32", G.FPW_ACCUM_FP32), ("f32 compensated", G.FPW_ACCUM_FP32_COMP),
                      ("binary64", G.FPW_ACCUM_FP64)):
        call_rate, kern_rate, ms = timed_batch(ctx, w, 20, w.k, G.fpw_params_default(accum=acc))
        T, R, NC, grid = ctx.last_shape()
        print(json.dumps({"config": f"sweep_100k/M=20 (batch of 1e4 curves), {name} bin sums", "accum": name,
                          "shape": dict(threads=T, freqs_per_thread=R, obs_chunk=NC), "ms_per_call": ms,
                          "evals_per_s_call": call_rate, "evals_per_s_tile_kernel": kern_rate,
                          "roofline_frac": (kern_rate / peak) if kern_rate else None}), flush=True)


def run_configs_shared(ctx, peak):
    """Curves sharing their times: the tensor-core path against the batched path
    on the same curves."""
    import numpy as np
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    w = L.make("shared_4096")
    C, n = w.ncurves, L.SHARED_N
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
         for a in (w.t[:n], w.x.reshape(C, n), w.sigma.reshape(C, n), w.freqs)]
    idx = torch.empty(C * w.k, dtype=torch.int32, device="cuda")
    Sk = torch.empty(C * w.k, dtype=torch.float32, device="cuda")
    call = lambda: G.fpw_periodogram_shared(ctx, None, None, d[0], d[1], d[2], d[3], w.M, w.k, idx, Sk)
    call()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    kms, nl = ctx.kernel_time()
    ctx.set_timing(False)
    ev = float(C) * n * w.nfreq
    fpm = 256 // w.M
    n_mma = -(-fpm * w.M // 16) * 16
    npass = -(-w.nfreq // (2 * fpm))
    flops = 2.0 * 128 * 2 * n_mma * (-(-n // 32) * 64) * npass * (-(-C // 64))  # issued MMA flops per call
    kern_s = kms / nl / 1e3
    tile_rate, tile_kern, _ = timed_batch(ctx, w, w.M, w.k, G.fpw_params_default())
    line = {"config": "shared_4096 (4096 curves sharing N=1000 times, M=20, 5e5 freqs, top-5)", "curves": C,
            "nobs_shared": n, "nfreq": w.nfreq, "M": w.M, "evals": ev,
            "ms_per_call": e0.elapsed_time(e1) / reps, "evals_per_s_call": ev / (e0.elapsed_time(e1) / reps / 1e3),
            "evals_per_s_mma_kernel": ev / kern_s,
            "mma_tflops_issued": flops / kern_s / 1e12,
            "tensor_frac_of_measured_bf16_peak": flops / kern_s / 1e12 / peak_bf16_tflops(),
            "batched_path_same_curves_evals_per_s_call": tile_rate,
            "batched_path_same_curves_evals_per_s_tile_kernel": tile_kern}
    print(json.dumps(line), flush=True)


def run_configs_drift(ctx, peak):
    """Baseline drift marginalised (K = 3 Chebyshev terms, beta = 1) on the
    ragged batch."""
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    w = L.make("ragged_10k")
    d = [torch.from_numpy(a).cuda() for a in (w.offsets, w.t, w.x, w.sigma, w.freqs)]
    idx = torch.empty(w.ncurves * w.k, dtype=torch.int32, device="cuda")
    Sk = torch.empty(w.ncurves * w.k, dtype=torch.float32, device="cuda")
    call = lambda: G.fpw_periodogram_drift(ctx, None, None, d[0], d[1], d[2], d[3], d[4], w.M, 3, 1.0, w.k, idx, Sk)
    call()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    call()
    e1.record()
    torch.cuda.synchronize()
    kms, nl = ctx.kernel_time()
    ctx.set_timing(False)
    ev = float(w.offsets[-1]) * w.nfreq
    print(json.dumps({"config": "ragged_10k, baseline drift marginalised (K=3 Chebyshev terms, beta=1), M=20, top-5",
                      "evals": ev, "ms_per_call": e0.elapsed_time(e1), "evals_per_s_call": ev / (e0.elapsed_time(e1) / 1e3),
                      "evals_per_s_drift_kernel": ev / (kms / nl / 1e3),
                      "smem_roof_evals_per_s": peak * 16.0 / 32.0,
                      "roofline_frac": ev / (kms / nl / 1e3) / (peak * 16.0 / 32.0),
                      "note": "K=3: one (Y, Bw, Q_1, Q_2) float4 read-modify-write (2 x 16 B) per evaluation"}), flush=True)


def run_configs_multi(ctx, peak):
    """Several M from one M_max pass (Section 3.4) on one 1e4-curve batch of the
    sweep: M_max = 20 (M = 20, 10, 5), 40 and 60 (M = 20, 10, 4, with 2..15
    bin offsets each), against the single-M call at M = 20 on the same batch.
    An evaluation is one (observation, frequency) pair accumulated at M_max."""
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    w = L.make("sweep_100k", range(10_000), M=20)
    d = [torch.from_numpy(a).cuda() for a in (w.offsets, w.t, w.x, w.sigma, w.freqs)]
    ev = float(w.offsets[-1]) * w.nfreq
    for M_max, groups in ((20, (1, 2, 4)), (40, (2, 4, 10)), (60, (3, 6, 15))):
        ng, k = len(groups), w.k
        idx = torch.empty(w.ncurves * ng * k, dtype=torch.int32, device="cuda")
        off = torch.empty(w.ncurves * ng * k, dtype=torch.int32, device="cuda")
        Sk = torch.empty(w.ncurves * ng * k, dtype=torch.float32, device="cuda")
        call = lambda: G.fpw_periodogram_batch_multi(ctx, None, None, d[0], w.offsets, d[1], d[2], d[3], d[4],
                                                     M_max, groups, k, idx, off, Sk)
        call()
        torch.cuda.synchronize()
        ctx.set_timing(True)
        ctx.kernel_time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        kms, nl = ctx.kernel_time()
        ctx.set_timing(False)
        kern = ev / (kms / nl / 1e3)
        print(json.dumps({"config": f"sweep_100k batch of 1e4 curves, several M: M_max={M_max}, "
                                    f"M={[M_max // g for g in groups]} with every offset, top-{k} per M",
                          "evals": ev, "ms_per_call": e0.elapsed_time(e1),
                          "evals_per_s_call": ev / (e0.elapsed_time(e1) / 1e3), "evals_per_s_tile_kernel": kern,
                          "roofline_frac": kern / peak, "status": ctx.status(),
                          "note": "roof: the 16 B (A, B) read-modify-write per evaluation at M_max bins"}), flush=True)


def run_configs_entropy(ctx, peak):
    """Phase entropy (Appendix C): the dense H(f) of the N = 1000 ZTF-cadence
    times over 1e6 frequencies, and H with its z-score at the top-5 peaks of
    the 1e4 ragged curves."""
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    w = L.make("single_ztf")
    t, fr = torch.from_numpy(w.t).cuda(), torch.from_numpy(w.freqs).cuda()
    H = torch.empty(w.nfreq, dtype=torch.float32, device="cuda")
    reps = 20  # one call is ~0.4 ms: the mean of 20 back-to-back calls
    for M in (10, 20, 50):
        G.fpw_phase_entropy(ctx, None, t, fr, M, H)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            G.fpw_phase_entropy(ctx, None, t, fr, M, H)
        e1.record()
        torch.cuda.synchronize()
        ev = float(w.t.size) * w.nfreq
        rate = ev / (e0.elapsed_time(e1) / reps / 1e3)
        # shared-memory term: per observation and warp, R count loads and R
        # count stores of 4 B per lane (one wavefront each) plus the staged
        # 16-byte record read by every lane (two wavefronts), over 32 R
        # evaluations; the kernel's frequencies per thread R follow M
        R = entropy_R(M)
        smem_roof = peak / SMEM_EVALS_PER_CLK_SM * (32.0 * R / (2.0 * R + 2.0))
        issue_roof = peak / SMEM_EVALS_PER_CLK_SM * 128.0 / ENTROPY_INST_PER_EVAL
        terms = {"smem": smem_roof}
        if R == 4:  # the instruction mix was measured at R = 4 (M = 20)
            terms["issue"] = issue_roof
        binding = min(terms, key=terms.get)
        print(json.dumps({"config": f"single_ztf times (N={w.t.size}), dense phase entropy, M={M}, "
                                    f"{w.nfreq:.0e} freqs 0.01-100 1/d", "evals": ev,
                          "ms_per_call": e0.elapsed_time(e1) / reps, "evals_per_s_call": rate,
                          "roofline": {"smem_counts_and_record": smem_roof, "issue": terms.get("issue"),
                                       "binding": binding, "frac_binding": rate / terms[binding],
                                       "frac_smem": rate / smem_roof, "R": R},
                          "status": ctx.status(),
                          "note": f"roof terms: R count read-modify-writes (4 B per lane) and one 16 B broadcast "
                                  f"record per observation and warp, 2 R + 2 wavefronts per 32 R evaluations; "
                                  f"128 thread instructions/clk/SM over {ENTROPY_INST_PER_EVAL} instructions per "
                                  f"evaluation (ncu, M = 20, R = 4)"}),
              flush=True)
    r = L.make("ragged_10k")
    d = [torch.from_numpy(a).cuda() for a in (r.offsets, r.t, r.x, r.sigma, r.freqs)]
    k = r.k
    idx = torch.empty(r.ncurves * k, dtype=torch.int32, device="cuda")
    Sk = torch.empty(r.ncurves * k, dtype=torch.float32, device="cuda")
    G.fpw_periodogram_batch_ex(ctx, None, None, d[0], r.offsets, d[1], d[2], d[3], d[4], r.M, k, idx, Sk)
    Hp = torch.empty(r.ncurves * k, dtype=torch.float32, device="cuda")
    zp = torch.empty(r.ncurves * k, dtype=torch.float32, device="cuda")
    G.fpw_phase_entropy_peaks(ctx, None, d[0], d[1], d[4], r.M, k, idx, Hp, zp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    G.fpw_phase_entropy_peaks(ctx, None, d[0], d[1], d[4], r.M, k, idx, Hp, zp)
    e1.record()
    torch.cuda.synchronize()
    ev = float(r.offsets[-1]) * k
    print(json.dumps({"config": f"ragged_10k top-{k} peaks: H and Hutcheson z per peak, M={r.M}", "evals": ev,
                      "ms_per_call": e0.elapsed_time(e1), "evals_per_s_call": ev / (e0.elapsed_time(e1) / 1e3),
                      "status": ctx.status()}), flush=True)


def run_case(args):
    """One small call of the shared-timestamp, baseline-drift, several-M or
    phase-entropy path, for profiling: two untimed calls, then one call timed
    with the library's kernel-timing hook (CUDA events around the call for the
    entropy kernel, the call's only launch); prints one JSON line."""
    import numpy as np
    import torch

    import lightcurves as L
    import paper_2502_00243_gb300 as G
    torch.cuda.set_device(0)
    ctx = G.Context(0)
    C, F = args.case_curves, args.nfreq
    idx = torch.empty(C * 5, dtype=torch.int32, device="cuda")
    Sk = torch.empty(C * 5, dtype=torch.float32, device="cuda")
    if args.case == "shared":
        w = L.make("shared_4096", range(C))
        n = L.SHARED_N
        freqs = np.linspace(0.01, 50.0, F)
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
             for a in (w.t[:n], w.x.reshape(C, n), w.sigma.reshape(C, n), freqs)]
        call = lambda: G.fpw_periodogram_shared(ctx, None, None, d[0], d[1], d[2], d[3], 20, 5, idx, Sk)
        ev = float(C) * n * F
        what = f"shared_4096: {C} curves sharing N={n} times, M=20, {F} freqs 0.01-50 1/d, top-5"
    elif args.case == "drift":
        w = L.make("ragged_10k", range(C), nfreq=F)
        d = [torch.from_numpy(a).cuda() for a in (w.offsets, w.t, w.x, w.sigma, w.freqs)]
        call = lambda: G.fpw_periodogram_drift(ctx, None, None, d[0], d[1], d[2], d[3], d[4], 20, 3, 1.0, 5, idx, Sk)
        ev = float(w.offsets[-1]) * F
        what = f"ragged_10k: first {C} curves, baseline drift K=3 beta=1, M=20, {F} freqs 0.02-50 1/d, top-5"
    elif args.case == "multi":
        w = L.make("sweep_100k", range(C), M=20, nfreq=F)
        d = [torch.from_numpy(a).cuda() for a in (w.offsets, w.t, w.x, w.sigma, w.freqs)]
        groups = (3, 6, 15)
        mi = torch.empty(C * 5 * len(groups), dtype=torch.int32, device="cuda")
        mo = torch.empty_like(mi)
        ms = torch.empty(C * 5 * len(groups), dtype=torch.float32, device="cuda")
        call = lambda: G.fpw_periodogram_batch_multi(ctx, None, None, d[0], w.offsets, d[1], d[2], d[3], d[4], 60,
                                                     groups, 5, mi, mo, ms)
        ev = float(w.offsets[-1]) * F
        what = f"sweep_100k: first {C} curves, several M from M_max=60 (M=20, 10, 4), {F} freqs 0.01-50 1/d, top-5"
    else:
        w = L.make("single_ztf", nfreq=F)
        t, fr = torch.from_numpy(w.t).cuda(), torch.from_numpy(w.freqs).cuda()
        H = torch.empty(F, dtype=torch.float32, device="cuda")
        call = lambda: G.fpw_phase_entropy(ctx, None, t, fr, 20, H)
        ev = float(w.t.size) * F
        what = f"single_ztf times (N={w.t.size}), dense phase entropy, M=20, {F} freqs 0.01-100 1/d"
        call()
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ms_ = e0.elapsed_time(e1)
        st = ctx.status()
        print(json.dumps({"case": args.case, "config": what, "status": st, "call_ms": ms_, "evals": ev,
                          "evals_per_s_call": ev / (ms_ / 1e3)}), flush=True)
        ctx.close()
        return 0 if st == 0 else 1
    call()
    call()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_time()
    call()
    torch.cuda.synchronize()
    kms, nl = ctx.kernel_time()
    ctx.set_timing(False)
    st = ctx.status()
    print(json.dumps({"case": args.case, "config": what, "status": st, "kernel_ms": kms / max(nl, 1),
                      "evals": ev, "evals_per_s_kernel": ev / (kms / max(nl, 1) / 1e3)}), flush=True)
    ctx.close()
    return 0 if st == 0 else 1


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--M", type=int, default=20)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--batch-curves", type=int, default=10_000)
    ap.add_argument("--curves-total", type=int, default=100_000)
    ap.add_argument("--nfreq", type=int, default=500_000,
                    help="linear grid points over 0.01-50 1/d (the sweep uses 5e5; fewer for small profiling runs)")
    ap.add_argument("--plain-curves", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=3.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-m", action="store_true", help="skip the M = 10 / 50 lines of the sweep")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the built-in kernel shapes (default: measure and install tuned shapes first)")
    ap.add_argument("--configs", nargs="?", const="all", default=None,
                    choices=["all", "batch", "accum", "shared", "drift", "multi", "entropy"],
                    help="report every workload (one JSON line each) instead, or one section of them")
    ap.add_argument("--case", choices=["shared", "drift", "multi", "entropy"],
                    help="one small call of that path (profiling case)")
    ap.add_argument("--case-curves", type=int, default=256)
    args = ap.parse_args(argv)
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.configs:
        return run_configs(args)
    if args.case:
        return run_case(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
