#!/usr/bin/env python
"""X-drop seed-and-extend benchmark on one GB300 (or N replicas).

Workload: the 29x overlap-pair workload (uniform random 4.6 Mbp genome,
lognormal reads of mean 10 kb / sd 6 kb, 12 % errors, every true overlap of
at least 2 kb seeded by one exact 17-mer; about 314k pairs = 628k
extensions), X = 50, scores +1/-1/-1, synthetic and seeded.

One step = one pass of the whole alignment path over that batch through the
C ABI: device validation and task expansion, length binning, the persistent
band kernel, the wider fallback tiers and the result write (a CUDA graph).
`value` is cell updates per second (GCUPS, cells counted by the reading's
range rule) with the inputs already in HBM; `e2e` is the same metric through
the host-memory call, with host-to-device and device-to-host copies inside
the timed region.  The plain per-10,000-pair form is timed beside it.

--impl reference times the CPU oracle (the only other implementation of
the method here) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "X-drop GCUPS & pairs/s on 1 GB300 (bit-exact), batched vs plain; p99 @25 producers"
UNIT = "GCUPS"
# algorithmic int ops per DP cell: 1 substitution select, 3 adds (diagonal + s,
# up + gap, left + gap), 2 max, 1 threshold compare/select, 1 running max
INT_OPS_PER_CELL = 8
INT32_LANES_PER_SM = 128  # 4 sub-partitions x 32 lanes, one warp instruction each per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--x", type=int, default=50)
    ap.add_argument("--workload", default="genome29x",
                    choices=["genome29x", "uneven", "genome100x"],
                    help="genome29x (default, the headline), uneven (1M Pareto-length pairs), "
                         "genome100x (100x coverage)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--pairs", type=int, default=0,
                    help="use only the first N pairs (small cases for profiling)")
    ap.add_argument("--tile", default="", help="force the first tile, e.g. 8x8 (no autotune)")
    ap.add_argument("--serve", action="store_true",
                    help="serving sweep only: 4 launch policies x load 0.5/0.75/1.0")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--seeds", action="store_true",
                    help="seed discovery only: reliable 31-mers and candidate pairs at 29x")
    ap.add_argument("--seeds-genome", type=int, default=4_600_000,
                    help="genome length of the seed-discovery read set")
    ap.add_argument("--seeds-sort", action="store_true",
                    help="seed discovery with the sort-based product (default: row-wise)")
    ap.add_argument("--no-seeds", action="store_true",
                    help="skip the seed-discovery object of the default line")
    ap.add_argument("--seeds-cpu", action="store_true",
                    help="with --seeds: also time the oracle on a 20 kb-genome sample")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device):
    """Maximum of a per-rank float over all ranks (timing only; no data)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


WORKLOAD_NAME = {"genome29x": "genome-29x-overlaps", "uneven": "uneven-pareto-1M-pairs",
                 "genome100x": "genome-100x-overlaps"}


def workload(x, pairs=0, kind="genome29x"):
    import numpy as np
    from paper_2309_07270_gb300 import workloads as W
    if kind == "uneven":
        w = W.uneven_pairs(n_pairs=1_000_000, seed=3, x=x)
        w.meta.update(genome_len=None, coverage=None, mean_len=None, sd_len=None, seed=3)
    elif kind == "genome100x":
        w = W.genome_overlaps(coverage=100.0, seed=4, x=x)
    else:
        w = W.genome_overlaps(seed=1, x=x)
    w.meta["kind"] = kind
    if pairs and pairs < w.n_pairs:
        w = w.subset(np.arange(pairs))
    return w


def workload_config(w):
    return {"workload": WORKLOAD_NAME[w.meta.get("kind", "genome29x")],
            "genome_bp": w.meta["genome_len"],
            "coverage": w.meta["coverage"], "reads": w.n_reads, "pairs": w.n_pairs,
            "extensions": 2 * w.n_pairs, "read_len_mean": w.meta["mean_len"],
            "read_len_sd": w.meta["sd_len"], "error_rate": 0.12, "seed_len": 17,
            "scores": [w.match, w.mismatch, w.gap], "x": w.x, "seed": w.meta["seed"]}


# ---------------------------------------------------------------------------
# CPU oracle arm (cpu_baseline, and --impl reference)
# ---------------------------------------------------------------------------

def time_oracle(w, target_s, rng_seed=0):
    import numpy as np
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    probe = w.subset(np.sort(rng.choice(w.n_pairs, 200, replace=False)))
    t0 = time.perf_counter()
    _, c = oracle.align_pairs(probe.packed, probe.read_off, probe.read_len, probe.pairs,
                              w.match, w.mismatch, w.gap, w.x, nthreads=cores, with_cells=True)
    dt = time.perf_counter() - t0
    per_pair = dt / 200
    n = int(min(w.n_pairs, max(200, target_s / max(per_pair, 1e-6))))
    idx = np.sort(rng.choice(w.n_pairs, n, replace=False))
    s = w.subset(idx)
    t0 = time.perf_counter()
    _, c = oracle.align_pairs(s.packed, s.read_off, s.read_len, s.pairs, w.match, w.mismatch,
                              w.gap, w.x, nthreads=cores, with_cells=True)
    dt = time.perf_counter() - t0
    cells = int(c.sum())
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random pairs of {w.n_pairs} (seeded), {cores} threads, "
                      f"{cells / 1e9:.2f} Gcells in {dt:.1f} s",
            "pairs_per_s": n / dt, "seconds": dt}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    w = workload(args.x, args.pairs, args.workload)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1234)
    per_step_pairs = 1500
    tot_cells, tot_t, tot_pairs = 0, 0.0, 0
    for step in range(args.warmup + args.steps):
        per_step_pairs = min(per_step_pairs, w.n_pairs)
        idx = np.sort(rng.choice(w.n_pairs, per_step_pairs, replace=False))
        s = w.subset(idx)
        t0 = time.perf_counter()
        _, c = oracle.align_pairs(s.packed, s.read_off, s.read_len, s.pairs, w.match,
                                  w.mismatch, w.gap, w.x, nthreads=cores, with_cells=True)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            tot_cells += int(c.sum())
            tot_t += dt
            tot_pairs += per_step_pairs
    v = tot_cells / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step_pairs} random pairs per step, {cores} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "pairs_per_s": tot_pairs / tot_t}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def kernel_source_sha():
    """First 16 hex digits of the sha256 of the band kernels' device sources."""
    h = hashlib.sha256()
    for f in ("xd_types.cuh", "xd_device.cuh", "xd_lockstep16.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2309_07270_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha()
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel_tag and f.get("source_sha") == sha:
            try:
                return float(f["dram_bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def run_serving(w, sc, capacity_pairs_s, policies, rhos, seconds, device, tile=None):
    """25 producers with Poisson arrivals of U[1k, 20k]-pair batches drawn
    from the workload's pairs (seeds 100+p), at rho x the measured batched
    capacity.  Returns one summary per (rho, policy)."""
    from paper_2309_07270_gb300 import serving
    from paper_2309_07270_gb300 import workloads as W
    runs = []
    for rho in rhos:
        sched = W.serving_schedule(w.n_pairs, n_producers=25,
                                   rate_pairs_per_s=rho * capacity_pairs_s,
                                   duration_s=seconds, seed_base=100)
        for pol in policies:
            r = serving.run_policy(pol, w, sched, sc, device=device, tile=tile, rho=rho,
                                   offered=rho * capacity_pairs_s)
            s = r.summary()
            s["seconds"] = seconds
            runs.append(s)
    return runs


def run_ours(args):
    import numpy as np
    import torch

    from paper_2309_07270_gb300 import build as B
    from paper_2309_07270_gb300 import xdrop as X

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_name = f"cuda:{local}"
    B.build()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    w = workload(args.x, args.pairs, args.workload)
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    dev = X.DeviceInputs.from_workload(w, device=dev_name)
    batched = X.Aligner(device=local, mode=X.XDROP_MODE_BATCHED)
    if args.tile:
        spec = args.tile.lower()
        lanes, cpl = spec.rstrip("p").split("x")
        batched.set_tile(int(lanes), int(cpl) | (X.XDROP_TILE_PACKED16 if spec.endswith("p") else 0))
    stream = torch.cuda.ExternalStream(batched.stream(), device=dev_name)
    cells_task = batched.count_cells_device(dev, sc).cpu().numpy()
    cells = int(cells_task.sum())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev_name)  # > 129 MB L2

    def step(al, strm):
        flush.zero_()  # L2 flush between steps, outside the timed events
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(strm)
        t = al.submit_device(dev, sc)
        e1.record(strm)
        X.xdrop_sync(al.ctx, t)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), al.stats()

    for _ in range(args.warmup):
        step(batched, stream)
    # bit-exactness spot check of the benchmarked output against the oracle
    # lives in tests/; here the status words must all be OK.
    res = dev.results()
    assert (res["status"] == 0).all()
    spills = X.xdrop_last_spills(batched.ctx)
    cells_tier0 = cells - int(cells_task[spills].sum()) if spills.size else cells

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    step_ms, main_ms, launches = [], [], 0
    for _ in range(args.steps):
        ms, st = step(batched, stream)
        step_ms.append(ms)
        main_ms.append(st["main_kernel_ms"])
        launches += st["launches"]
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()

    mean_ms = max_over_ranks(statistics.mean(step_ms), dev_name)
    value = ws * cells / (mean_ms * 1e-3) / 1e9
    pairs_s = ws * w.n_pairs / (mean_ms * 1e-3)

    # plain per-10,000-pair form, same inputs, same first tile and arithmetic
    plain = None
    if not args.no_plain:
        pal = X.Aligner(device=local, mode=X.XDROP_MODE_PLAIN)
        pal.set_tile(*batched.tile())
        pstream = torch.cuda.ExternalStream(pal.stream(), device=dev_name)
        for _ in range(2):
            step(pal, pstream)
        pms = [step(pal, pstream)[0] for _ in range(max(2, min(args.steps, 3)))]
        assert (dev.results() == res).all()
        pm = statistics.mean(pms)
        pt = pal.tile()
        assert pt == batched.tile()
        plain = {"value": cells / (pm * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": pm,
                 "pairs_per_s": w.n_pairs / (pm * 1e-3),
                 "tile": f"{pt[0]} lanes x {pt[1] & 0xff} cells"
                         + (" (16-bit packed)" if pt[1] & X.XDROP_TILE_PACKED16 else "")
                         + ", the batched form's first tile",
                 "launch": "one launch of the first tile per 10,000-pair sub-batch in pair "
                           "order (no binning, no graph, no autotuning), then the same wider tiers"}
        pal.close()

    # end to end through the host-memory call (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        def pinned(a):
            t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy()).pin_memory()
            return t.numpy().view(a.dtype)
        hp, ho, hl = pinned(w.packed), pinned(w.read_off), pinned(w.read_len)
        hpairs = pinned(w.pairs)
        hout = torch.zeros(w.n_pairs * 28, dtype=torch.uint8).pin_memory().numpy().view(X.RESULT_DTYPE)
        ets = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = X.xdrop_submit(batched.ctx, hp, ho, hl, hpairs, sc, hout)
            X.xdrop_sync(batched.ctx, t)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                ets.append(dt)
        assert (hout.view(np.int32) == res.view(np.int32)).all()
        em = max_over_ranks(statistics.mean(ets), dev_name)
        e2e = {"value": ws * cells / em / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(hp.nbytes + ho.nbytes + hl.nbytes + hpairs.nbytes),
               "d2h_bytes_per_step": int(hout.nbytes), "pairs_per_s": ws * w.n_pairs / em,
               "ms_per_step": em * 1e3, "call": "xdrop_submit + xdrop_sync (host buffers)"}

    # roofline of the dominant kernel: first-tier persistent band kernel,
    # against the int32 issue limit (SMs x 128 lanes x clock)
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * INT32_LANES_PER_SM * sm_max * 1e6 / 1e12
    main_mean = statistics.mean(main_ms) if main_ms and min(main_ms) > 0 else None
    achieved = (INT_OPS_PER_CELL * cells_tier0 / (main_mean * 1e-3) / 1e12) if main_mean else None
    tile = batched.tile()
    packed = bool(tile[1] & X.XDROP_TILE_PACKED16)
    cpl = tile[1] & 0xff
    if packed:
        kname = f"lockstep16_kernel<{tile[0]},{cpl // 2}>"
    else:
        kname = f"lockstep_kernel<{tile[0]},{cpl}>"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tintop/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_from_profile(kname),
            "kernel": kname,
            "kernel_ms": main_mean,
            "tcups": (cells_tier0 / (main_mean * 1e-3) / 1e12) if main_mean else None,
            "peak_basis": f"{props.multi_processor_count} SMs x {INT32_LANES_PER_SM} int32 lanes/clk "
                          f"x {sm_max:.0f} MHz (max SM clock): the int32 issue limit",
            "ops_per_cell": INT_OPS_PER_CELL, "cells_in_kernel": cells_tier0,
            "step_frac": INT_OPS_PER_CELL * cells / (mean_ms * 1e-3) / 1e12 / peak,
            "packed16": packed,
            # each packed lane op does two 16-bit cells: against twice the
            # int32 issue limit the same kernel reads as this fraction
            "frac_int16x2_issue": (achieved / (2 * peak)) if (achieved and packed) else None}

    serving_runs = None
    if not args.no_serve:
        serving_runs = run_serving(w, sc, pairs_s / ws, ["device-loop"], [0.75],
                                   args.serve_seconds, local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(w, args.cpu_seconds)

    seeds = None
    if rank == 0 and ws == 1 and not args.no_seeds:
        seeds = seed_discovery_runs()

    if rank == 0:
        cfg = workload_config(w)
        if args.pairs:
            cfg["workload"] += f"-first-{w.n_pairs}-pairs"
        cfg.update({"l2": "flushed between steps (256 MiB write outside the timed events)",
                    "form": "batched: binned persistent kernel in a CUDA graph",
                    "tile0": f"{tile[0]} lanes x {cpl} cells" + (" (16-bit packed)" if packed else ""),
                    "cells": cells,
                    "parallelism": f"{ws} independent replica(s), no collective"})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int16x2" if packed else "int32", "data": "synthetic", "config": cfg,
                "pairs_per_s": pairs_s, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "plain": plain,
                "batched_over_plain": (value / plain["value"]) if plain else None,
                "serving": serving_runs[0] if serving_runs else None,
                "seed_discovery": seeds,
                "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
    batched.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_serve_sweep(args):
    """Serving sweep: capacity from a short batched measurement, then every
    launch policy at three loads.  Prints one JSON line."""
    import torch

    from paper_2309_07270_gb300 import build as B
    from paper_2309_07270_gb300 import xdrop as X
    B.build()
    w = workload(args.x, args.pairs, args.workload)
    sc = X.scoring(w.match, w.mismatch, w.gap, w.x)
    dev = X.DeviceInputs.from_workload(w)
    with X.Aligner(mode=X.XDROP_MODE_BATCHED) as al:
        times = []
        for k in range(6):
            al.align_device(dev, sc)
            if k >= 3:
                times.append(al.stats()["kernel_ms"])
        ms = min(times)
    del dev
    torch.cuda.empty_cache()
    capacity = w.n_pairs / (ms * 1e-3)
    runs = run_serving(w, sc, capacity, ["device-loop", "per-producer-streams", "ring-subbatch",
                                         "ring-batch"], [0.5, 0.75, 1.0], args.serve_seconds, 0)
    print(json.dumps({"metric": METRIC, "mode": "serving sweep", "capacity_pairs_per_s": capacity,
                      "producers": 25, "batch_pairs": [1000, 20000],
                      "config": workload_config(w), "runs": runs}), flush=True)
    return 0


def seed_discovery_runs(genome=1_000_000, timeout_s=240):
    """Seed discovery (the upstream row: reliable 31-mers and candidate
    pairs) beside the headline: both products (row-wise, the default, and
    sort-based) on 29x reads of a genome of `genome` bases, each timed by
    `bench.py --seeds` in a process of its own, so that nothing there can
    touch the alignment numbers above.  A failed run is reported, not
    raised."""
    out = {"workload": f"reads-29x-genome{genome}-err1pct, k=31, window [20, 50]",
           "timing": "CUDA events around the library's pipeline, median of 3 steps"}
    keep = ("value", "unit", "ms_per_step", "host_ms_per_step", "product", "candidates",
            "reverse_strand", "candidates_sha256", "occurrences", "nonzeros", "reads",
            "cpu_baseline", "roofline")
    for name, extra in (("rowwise", ["--seeds-cpu"]), ("sort", ["--seeds-sort"])):
        cmd = [sys.executable, os.path.abspath(__file__), "--seeds", "--seeds-genome", str(genome),
               "--steps", "3", "--warmup", "1"] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
        except subprocess.TimeoutExpired:
            out[name] = {"error": f"no result within {timeout_s} s"}
            continue
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode == 0 and lines:
            d = json.loads(lines[-1])
            out[name] = {k: d.get(k) for k in keep}
        else:
            tail = (r.stderr.strip().splitlines() or ["(no output)"])[-1]
            out[name] = {"error": f"exit {r.returncode}: {tail[:300]}"}
    digests = [out[n].get("candidates_sha256") for n in ("rowwise", "sort")]
    out["products_agree"] = (digests[0] == digests[1]) if all(digests) else None
    return out


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback: 6.8 TB/s, one earlier GB300 copy measurement"


def seed_algorithmic_bytes(read_set_bytes, occurrences, nonzeros, candidates):
    """Bytes seed discovery must move by its method: the packed read set
    read once, every k-mer occurrence's 64-bit code written once and read
    once, every nonzero of the read-by-k-mer matrix A written once and read
    once (8 B each way), and the candidate records (20 B pair + 4 B count)
    written once."""
    return read_set_bytes + 16 * occurrences + 16 * nonzeros + 24 * candidates


def run_seeds(args):
    """Seed discovery at the paper's parameters (k = 31, stride 1, frequency
    window [20, 50]) on 29x coverage of a random genome of --seeds-genome
    bases, reads of mean 10 kb with 1 % errors from both strands.  One step
    = one xdrop_find_candidates over the resident reads (the row-wise
    product, or the sort-based one with --seeds-sort), timed with the CUDA
    events the library records around its pipeline (the candidates' copy to
    host included) and, beside it, on the host around the synchronous call;
    reloading the reads between steps, outside the timed region, drops the
    cached result.  Prints one JSON line: k-mer occurrences per second."""
    import numpy as np

    from paper_2309_07270_gb300 import build as B
    from paper_2309_07270_gb300 import workloads as W
    from paper_2309_07270_gb300 import xdrop as X
    B.build()
    k, lo, hi = 31, 20, 50
    packed, off, lens = W.sequencing_reads(args.seeds_genome, 29, 10_000, 6_000, 1_000, seed=29,
                                           error_rate=0.01)
    n_occ = int(np.maximum(lens.astype(np.int64) - (k - 1), 0).sum())
    host, dev, products = [], [], set()
    with X.Aligner() as al:
        for step in range(args.warmup + args.steps):
            X.xdrop_load_reads(al.ctx, packed, off, lens)
            t0 = time.perf_counter()
            pairs, shared = X.xdrop_find_candidates(al.ctx, k, lo, hi, 1, not args.seeds_sort)
            dt = time.perf_counter() - t0
            st = X.xdrop_get_seed_stats(al.ctx)
            if step >= args.warmup:
                host.append(dt * 1e3)
                dev.append(st["ms"])
                products.add(st["product"])
    ms = statistics.median(dev)
    cpu = None
    if args.seeds_cpu:  # the oracle as it stands, one core, on a small read set of the same recipe
        from oracle import seeds as S
        g = 20_000
        sp, so, sl = W.sequencing_reads(g, 29, 10_000, 6_000, 1_000, seed=29, error_rate=0.01)
        s_occ = int(np.maximum(sl.astype(np.int64) - (k - 1), 0).sum())
        t0 = time.perf_counter()
        S.candidate_pairs(sp, so, sl, k=k, lo=lo, hi=hi)
        dt = time.perf_counter() - t0
        cpu = {"value": s_occ / dt, "unit": "occurrences/s", "cores": 1, "kind": "oracle",
               "sample": f"29x reads of a {g}-base genome, 1% errors ({s_occ} occurrences), "
                         f"one call, {dt:.1f} s"}
    names = {X.XDROP_SEEDS_SORT: "sort", X.XDROP_SEEDS_ROWWISE: "rowwise"}
    nnz = int(st["nonzeros"])
    roof = None
    if nnz:  # the row-wise product ran and counted A's nonzeros
        alg = seed_algorithmic_bytes(int(packed.nbytes), n_occ, nnz, len(pairs))
        peak, basis = hbm_peak_gbs()
        gbs = alg / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "traffic": None, "algorithmic_bytes": alg, "peak_basis": basis,
                "bytes_basis": "2-bit read set read once + 16 B per k-mer occurrence (its 64-bit "
                               "code written once and read once) + 16 B per nonzero of A "
                               "(written once, read once) + 24 B per candidate record"}
    print(json.dumps({"metric": f"seed discovery, k-mer occurrences/s (k={k}, window [{lo}, {hi}])",
                      "value": n_occ / (ms * 1e-3), "unit": "occurrences/s", "ms_per_step": ms,
                      "host_ms_per_step": statistics.median(host), "steps": args.steps,
                      "warmup": args.warmup, "higher_is_better": True,
                      "product": "+".join(sorted(names[p] for p in products)),
                      "candidates": int(len(pairs)), "reverse_strand": int((pairs["b"] >> 31).sum()),
                      "candidates_sha256": hashlib.sha256(pairs.tobytes() + shared.tobytes())
                      .hexdigest()[:16],
                      "cpu_baseline": cpu,
                      "reads": int(len(lens)), "occurrences": n_occ, "nonzeros": nnz,
                      "roofline": roof, "data": "synthetic",
                      "config": {"workload": f"reads-29x-genome{args.seeds_genome}-err1pct",
                                 "timing": "CUDA events around the library's pipeline"}}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.seeds:
        return run_seeds(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
