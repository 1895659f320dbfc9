"""Benchmark: events/s of CA seeding + broken-line fit on one GB300, batched/served vs plain.

Workload: the 256-event batch (barrel geometry, per-event track count uniform in 200..6000,
pT 1-10 GeV, |eta| < 1, noise-free helices; ~0.8 M tracks, ~3.2 M hits per batch).  One step =
the whole hot path (sort, doublets, CA connect, ntuplets, selection, fit) over the batch, replayed
from a captured CUDA graph with the inputs already in device memory.  Between timed steps the L2
is flushed by writing a 512 MB buffer (outside the timed events).

Also reported: per-stage device times and the doublet kernel's fraction of the measured HBM
bandwidth; the plain path (one event per launch sequence); end to end through the serving API
with host buffers (H2D/D2H inside); p50/p99 latency of Poisson-arriving events; the FP64 oracle on
the host cores (bounded sample).  `--impl reference` times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch256_barrel_T200-6000"
METRIC = "events/s (CA seeding + broken-line fit)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pxr", choices=["pxr", "reference"])
    ap.add_argument("--cut", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fit", default="mixed", choices=["fp64", "mixed", "fp32"])
    ap.add_argument("--events", type=int, default=256)
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/serving/cpu legs")
    ap.add_argument("--serve-rate", type=float, default=5000.0)
    ap.add_argument("--no-tune", action="store_true", help="built-in bin count and grid sizes")
    ap.add_argument("--bins", type=int, default=0, help="phi bins per layer (skips tuning)")
    ap.add_argument("--grid", default="", help="CTAs per SM per stage, 6 comma-separated values "
                    "(sort,doublets,connect,walk,select,fit; skips tuning)")
    ap.add_argument("--tune-cache", default=os.path.join(os.path.expanduser("~"), ".cache", "pxr",
                                                         "tune.json"))
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_batch(n_events, seed0):
    from paper_2104_06573_gb300 import synth
    counts = synth.batch_track_counts(n_events, seed0)
    return counts, [synth.make_event(seed0 + e, counts[e]) for e in range(n_events)]


# ---------------------------------------------------------------------------------------------
# host-core oracle baseline (spawned processes: one event per process, all cores)
# ---------------------------------------------------------------------------------------------
def _oracle_event(args):
    seed, T = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2104_06573_gb300 import synth
    ev = synth.make_event(seed, T)
    P = synth.params_barrel_quadruplets()
    t0 = time.perf_counter()
    r = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, P)
    return time.perf_counter() - t0, len(r["tuples"])


def cpu_baseline(seeds_counts, cores):
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_event, seeds_counts, chunksize=1)
    wall = time.perf_counter() - t0
    return len(seeds_counts) / wall, wall, sum(r[0] for r in res)


def oracle_sample(n_events):
    """A bounded sample of the batch workload: events spread over the track-count range."""
    from paper_2104_06573_gb300 import synth
    counts = synth.batch_track_counts(256, 0)
    idx = np.linspace(0, 255, n_events).astype(int)
    return [(int(i), int(counts[i])) for i in idx]


# ---------------------------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------------------------
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample = oracle_sample(min(32, 2 * cores))
    for _ in range(args.warmup):
        cpu_baseline(sample[:cores], cores)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        v, wall, cpu_s = cpu_baseline(sample, cores)
        n += len(sample)
    wall = time.perf_counter() - t0
    value = n / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_events": len(sample)},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{len(sample)} events of the batch spread over 200-6000 "
                                       f"tracks, one event per process"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def doublet_traffic(cells, n_phi_bins):
    """DRAM bytes of one k_doublets launch from the committed ncu capture (scaled by cells, the
    units the launch processes), or None when the kernel source or the bin count (which sets the
    candidates per cell) differs from the capture's."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_doublets_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2104_06573_gb300", "csrc", "k_graph.cu")).read()
        a = src.index("__global__ void __launch_bounds__(256) k_doublets(")
        b = src.index("void launch_doublets(")
        if hashlib.sha256(src[a:b].encode()).hexdigest()[:16] != rec["source_sha16"]:
            return None
        if int(rec.get("n_phi_bins", -1)) != int(n_phi_bins):
            return None
        return rec["dram_bytes_per_cell"] * cells
    except (OSError, ValueError, KeyError):
        return None


def doublet_algorithmic_bytes(layer_counts, pairs, n_cells):
    """16 B per hit read per layer pair it takes part in, 8 B per inner hit and pair for the two
    bucket offsets of its window, 8 B per cell written."""
    b = 0
    for lc in layer_counts:
        for a, o in pairs:
            b += 16 * (lc[a] + lc[o]) + 8 * lc[a]
    return b + 8 * n_cells


def run_pxr(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2104_06573_gb300 import pxr, shard, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    cut = pxr.CUT_FP32 if args.cut == "fp32" else pxr.CUT_FP64
    fit = {"fp64": pxr.FIT_FP64, "mixed": pxr.FIT_MIXED, "fp32": pxr.FIT_FP32}[args.fit]
    P = synth.params_barrel_quadruplets()
    params = pxr.params_from(P, cut_mode=cut, fit_mode=fit)
    # each rank processes its own batch of events (event sharding, no collective)
    counts, evs = make_batch(args.events, seed0=shard.rank_seed0(rank))
    off = np.zeros(len(evs) + 1, np.uint32)
    off[1:] = np.cumsum([e.n for e in evs])
    cat = lambda k: np.concatenate([getattr(e, k) for e in evs])
    hx, hy, hz, hl = cat("x"), cat("y"), cat("z"), cat("layer")
    x = torch.from_numpy(hx).to(dev)
    y = torch.from_numpy(hy).to(dev)
    z = torch.from_numpy(hz).to(dev)
    layer = torch.from_numpy(hl.view(np.int16)).to(dev)
    layer_counts = [np.bincount(e.layer, minlength=4) for e in evs]
    n_hits = int(off[-1])

    budget = 64 << 30
    arena = torch.empty(budget, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pxr.Context(device=local, mem_budget_bytes=budget, arena=arena,
                      stream=stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    tuning = None
    if args.bins or args.grid:
        grid = [int(v) for v in args.grid.split(",")] if args.grid else [0] * 6
        from paper_2104_06573_gb300 import autotune
        params = autotune._with(params, args.bins or 0, grid)
        tuning = {"n_phi_bins": args.bins, "grid_per_sm": grid}
    elif not args.no_tune:
        # phi-bin count and per-stage grid sizes picked on this batch (outside the timed region)
        from paper_2104_06573_gb300 import autotune
        with torch.cuda.stream(stream):
            params, tuning = autotune.tune_plan(ctx, off, x, y, z, layer, params, stream=stream,
                                                cache=args.tune_cache, flush=flush.zero_)
        torch.cuda.synchronize()
    plan = pxr.Plan(ctx, off, x, y, z, layer, params, use_graph=True)

    def step_events(n):
        return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(n)]

    for _ in range(args.warmup):
        flush.zero_()
        plan.pxr_plan_run(stream)
    torch.cuda.synchronize()
    ev = step_events(args.steps)
    clocks = Clocks(local)
    clocks.start()
    shard.barrier()
    torch.cuda.synchronize()
    stage = np.zeros(5)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            plan.pxr_plan_run(stream)
            ev[k][1].record(stream)
            stream.synchronize()
            stage += np.array(plan.pxr_plan_stage_ms())
    torch.cuda.synchronize()
    shard.barrier()
    clk = clocks.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    total_ms = float(step_ms.sum())
    total_ms = shard.max_over_ranks(total_ms, device=dev)
    value = args.events * world * args.steps / (total_ms / 1e3)
    stage /= args.steps

    cnt = plan.pxr_plan_counts()
    assert not cnt["flags"].any(), "capacity overflow in the timed batch"
    cells = int(cnt["cells"].sum())
    n_tracks = int(cnt["tracks"].sum())
    layer_counts = [[int(v) for v in lc] for lc in layer_counts]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    alg = doublet_algorithmic_bytes(layer_counts, P.pairs, cells)
    k4_ms = stage[1]
    achieved = alg / (k4_ms / 1e3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"cuts {args.cut}, fit {args.fit}", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": args.events * world,
                       "hits_per_step": n_hits * world, "l2": "flushed (512 MB write) between steps",
                       "launch": "captured CUDA graph, inputs resident",
                       "tuning": tuning and {k: tuning[k] for k in ("n_phi_bins", "grid_per_sm")}},
            "gpu_launches": plan.pxr_plan_launches() * args.steps,
            "stage_ms": dict(zip(["sort", "doublets", "connect", "ntuplets+select",
                                  "fit+output"], [round(v, 4) for v in stage])),
            "roofline": {"kernel": "k_doublets", "bound": "hbm", "achieved": achieved,
                         "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "peak_source": peak_src,
                         "traffic": doublet_traffic(cells, params.n_phi_bins),
                         "algorithmic_bytes": alg, "cells": cells},
            "clocks": clk, "tracks_per_step": n_tracks * world}

    if not args.no_extras and rank == 0:
        line.update(extras(args, ctx, pxr, synth, P, params, evs, off, x, y, z, layer, dev,
                           stream, value))
    plan.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extras(args, ctx, pxr, synth, P, params, evs, off, x, y, z, layer, dev, stream, value):
    import torch
    out = {}
    # plain path: one event per launch sequence, sequential, inputs resident
    plans = [pxr.Plan(ctx, [0, int(off[e + 1] - off[e])], x[int(off[e]):], y[int(off[e]):],
                      z[int(off[e]):], layer[int(off[e]):], params, use_graph=False)
             for e in range(len(evs))]
    for p in plans[:8]:
        p.pxr_plan_run(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for p in plans:
        p.pxr_plan_run(stream)
    b.record(stream)
    torch.cuda.synchronize()
    plain = len(plans) / (a.elapsed_time(b) / 1e3)
    for p in plans:
        p.close()
    out["plain"] = {"value": plain, "unit": "events/s",
                    "how": "one event per launch sequence, no graph, same stream"}
    out["batched_over_plain"] = value / plain

    # end to end through the serving API with host buffers (copies inside the timed region)
    with pxr.Context(device=dev.index, mem_budget_bytes=48 << 30, max_batch_events=256) as sctx:
        def serve_all():
            t0 = time.perf_counter()
            tickets = [sctx.pxr_submit_event(e.x, e.y, e.z, e.layer, params) for e in evs]
            done = 0
            while done < len(tickets):
                done += len(sctx.pxr_poll(timeout_us=100000))
            d2h = 0
            for t in tickets:
                r = sctx.pxr_fetch_tracks(t)
                d2h += r["n"] * (1 + 4 * pxr.MAX_HITS + 6 * 8 + 2) + 8
            return time.perf_counter() - t0, d2h
        serve_all()
        times = []
        for _ in range(3):
            dt, d2h = serve_all()
            times.append(dt)
        e2e = len(evs) / float(np.median(times))
        out["e2e"] = {"value": e2e, "unit": "events/s",
                      "h2d_bytes_per_step": int(sum(14 * e.n for e in evs)),
                      "d2h_bytes_per_step": int(d2h),
                      "how": "pxr_submit_event x256 (host arrays) + pxr_poll + pxr_fetch_tracks"}

        # Poisson arrivals: latency submit -> fetchable
        rate = args.serve_rate
        n_req = int(min(6000, max(500, rate * 1.5)))
        arr, tcount = synth.serving_stream(rate, n_req, seed=1)
        pool = [synth.event_serving(1000 + k, int(tcount[k])) for k in range(64)]
        t_sub, t_done = {}, {}
        start = time.perf_counter()
        k = 0
        pending = 0
        while k < n_req or pending:
            now = time.perf_counter() - start
            while k < n_req and arr[k] <= now:
                e = pool[k % len(pool)]
                t = sctx.try_submit_event(e.x, e.y, e.z, e.layer, params)
                if t is None:
                    break
                t_sub[t] = time.perf_counter()
                k += 1
                pending += 1
            for t in sctx.pxr_poll(timeout_us=50 if k < n_req else 20000):
                t_done[t] = time.perf_counter()
                sctx.pxr_fetch_tracks(t)
                pending -= 1
        lat = np.array([t_done[t] - t_sub[t] for t in t_sub]) * 1e3
        span = max(t_done.values()) - min(t_sub.values())
        out["serving"] = {"rate_hz": rate, "events": n_req, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "events_per_s": n_req / span,
                          "tracks": "lognormal median 1500, sigma 0.8, cap 8000; smeared barrel"}

    # host-core oracle on a bounded sample of the same workload
    cores = os.cpu_count() or 1
    sample = oracle_sample(min(32, 2 * cores))
    v, wall, cpu_s = cpu_baseline(sample, cores)
    out["cpu_baseline"] = {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
                           "sample": f"{len(sample)} events spread over the batch's 200-6000 "
                                     f"track range, one event per process ({wall:.1f} s)"}
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_pxr(args, rank, world, local)


if __name__ == "__main__":
    main()
