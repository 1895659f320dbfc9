"""Autotuner of the batch path: phi-bin count and per-stage grid sizes.

Neither choice changes a result (the bin window is wider than the cut, and every kernel strides
over its work whatever its grid), only the time.  The tuner times candidate settings on the
caller's own batch, with the plan's per-stage device timers, and keeps the fastest:

1. the bin count over ``BINS`` (it changes the candidate windows of the doublet and CA stages,
   so the whole step is compared);
2. then, one stage at a time with the others held, the CTAs-per-SM cap of that stage over
   ``GRIDS`` (coordinate descent; the stages run one after another, so their times add).

The search itself (:func:`search`) takes any ``measure`` function, so it is tested on the CPU
with a synthetic cost; :func:`tune_plan` measures with real plans.  Results are cached in a JSON
file keyed by the workload's shape (:func:`cache_key`).
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from typing import Callable, Sequence

BINS = (128, 256, 512, 1024)
GRIDS = (2, 4, 8, 16, 32)
N_STAGES = 6                                # sort, doublets, connect, walk, select, fit
DEFAULT_GRID = (0,) * N_STAGES              # 0: the library's built-in value


def search(measure: Callable[[int, Sequence[int]], float], bins: Sequence[int] = BINS,
           grids: Sequence[int] = GRIDS, stages: Sequence[int] = range(N_STAGES)):
    """Coordinate descent: best bin count with built-in grids, then each stage's grid cap.

    measure(n_phi_bins, grid_per_sm) returns the time of one step (any unit; smaller is better).
    Returns (n_phi_bins, grid_per_sm list, best time, number of measurements).
    """
    calls = 0

    def m(nb, g):
        nonlocal calls
        calls += 1
        return measure(nb, tuple(g))

    grid = list(DEFAULT_GRID)
    best_nb, best_t = None, float("inf")
    for nb in bins:
        t = m(nb, grid)
        if t < best_t:
            best_nb, best_t = nb, t
    for k in stages:
        best_g = grid[k]
        for g in grids:
            trial = list(grid)
            trial[k] = g
            t = m(best_nb, trial)
            if t < best_t:
                best_g, best_t = g, t
        grid[k] = best_g
    return best_nb, grid, best_t, calls


def cache_key(params, n_events: int, n_hits: int) -> str:
    """Workload shape: geometry and cut/fit modes (hashed), events and hits (to 1/16 decades)."""
    geo = (int(params.n_layers), tuple(int(v) for v in params.layer_is_disk[:params.n_layers]),
           tuple((int(params.pair_inner[k]), int(params.pair_outer[k]))
                 for k in range(params.n_pairs)),
           int(params.min_hits), int(params.max_hits), int(params.cut_mode),
           int(params.fit_mode), round(float(params.phi_window), 9))
    h = hashlib.sha256(repr(geo).encode()).hexdigest()[:12]
    return f"{h}-E{n_events}-N{round(16 * math.log10(max(n_hits, 1)))}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, value: dict) -> None:
    c = load_cache(path)
    c[key] = value
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_plan(ctx, hit_offsets, x, y, z, layer, params, stream=None, reps: int = 5,
              bins: Sequence[int] = BINS, grids: Sequence[int] = GRIDS, cache: str | None = None,
              flush=None):
    """Tune n_phi_bins and grid_per_sm of `params` on this batch (device inputs); returns a copy
    of params with the choice filled in and a dict describing it.  `flush()` (optional) runs
    before every timed step (an L2 flush on the same stream).  A setting's time is the fastest of
    its `reps` steps: interference from other work on the device only ever adds time."""
    import numpy as np

    from . import pxr

    n_events = len(hit_offsets) - 1
    n_hits = int(hit_offsets[-1])
    key = cache_key(params, n_events, n_hits)
    if cache:
        hit = load_cache(cache).get(key)
        if hit:
            return _with(params, hit["n_phi_bins"], hit["grid_per_sm"]), dict(hit, cached=True)

    def measure(nb, grid):
        p = _with(params, nb, grid)
        plan = pxr.Plan(ctx, hit_offsets, x, y, z, layer, p, use_graph=True)
        try:
            times = []
            for r in range(reps + 1):
                if flush is not None:
                    flush()
                plan.pxr_plan_run(stream)
                if r:                                           # first run warms up
                    times.append(sum(plan.pxr_plan_stage_ms()))
            if plan.pxr_plan_counts()["flags"].any():           # a capacity ran out: reject
                return float("inf")
            return float(np.min(times))
        finally:
            plan.close()

    nb, grid, t, calls = search(measure, bins, grids)
    info = {"n_phi_bins": nb, "grid_per_sm": list(grid), "step_ms": t, "trials": calls,
            "stages": list(pxr.STAGES)}
    if cache:
        store_cache(cache, key, info)
    return _with(params, nb, grid), info


def _with(params, nb, grid):
    import ctypes as C
    from . import pxr
    p = pxr.pxr_params()
    C.memmove(C.byref(p), C.byref(params), C.sizeof(p))
    p.n_phi_bins = int(nb)
    for k, v in enumerate(grid):
        p.grid_per_sm[k] = int(v)
    return p
