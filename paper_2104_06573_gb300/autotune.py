"""Autotuner of the batch path: phi-bin count, per-stage grid sizes and threads per block.

None of these choices changes a result (the bin window is wider than the cut, and every kernel
strides over its work whatever its launch shape), only the time.  The tuner times candidate
settings on the caller's own batch, with the plan's per-stage device timers, and keeps the
fastest:

1. the bin count over ``BINS`` (it changes the candidate windows of the doublet and CA stages,
   so the whole step is compared);
2. then, one stage at a time with the others held, the CTAs-per-SM cap of that stage over
   ``GRIDS`` and, for the stages whose kernels take any of several block sizes (``BLOCKS``:
   the sort, the doublets and the fit), the threads per CTA (coordinate descent; the stages run
   one after another, so their times add).

The search itself (:func:`search`) takes any ``measure`` function, so it is tested on the CPU
with a synthetic cost; :func:`tune_plan` measures with real plans.  Results are cached in a JSON
file keyed by the GPU's name, a hash of every parameter the tuner does not choose and the
batch's size (:func:`cache_key`).
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from typing import Callable, Sequence

BINS = (64, 128, 256, 512, 1024)
GRIDS = (2, 4, 8, 16, 32)
N_STAGES = 6                                # sort, doublets, connect, walk, select, fit
DEFAULT_GRID = (0,) * N_STAGES              # 0: the library's built-in value
# threads per CTA each stage's kernels accept besides the built-in (0); the CA, walk and
# selection kernels tie a CTA to a fixed chunk of work and take the built-in only
BLOCKS = {0: (256, 512, 1024), 1: (64, 128, 256), 5: (32, 64, 128, 256)}


def search(measure: Callable[[int, Sequence[int], Sequence[int]], float],
           bins: Sequence[int] = BINS, grids: Sequence[int] = GRIDS,
           stages: Sequence[int] = range(N_STAGES), blocks: dict = BLOCKS):
    """Coordinate descent: best bin count with built-in launch shapes, then per stage its grid
    cap and (where ``blocks`` lists candidates for it) its threads per CTA.

    measure(n_phi_bins, grid_per_sm, block_threads) returns the time of one step (any unit;
    smaller is better).  Returns (n_phi_bins, grid_per_sm list, block_threads list, best time,
    number of measurements).
    """
    calls = 0

    def m(nb, g, t):
        nonlocal calls
        calls += 1
        return measure(nb, tuple(g), tuple(t))

    grid = list(DEFAULT_GRID)
    block = [0] * N_STAGES
    best_nb, best_t = None, float("inf")
    for nb in bins:
        t = m(nb, grid, block)
        if t < best_t:
            best_nb, best_t = nb, t
    for k in stages:
        for axis, values in ((grid, grids), (block, blocks.get(k, ()))):
            best_v = axis[k]
            for v in values:
                axis[k] = v
                t = m(best_nb, grid, block)
                if t < best_t:
                    best_v, best_t = v, t
            axis[k] = best_v
    return best_nb, grid, block, best_t, calls


def config_hash(params) -> str:
    """Hash of every field of `params` except the ones the tuner chooses."""
    import ctypes as C
    q = type(params)()
    C.memmove(C.byref(q), C.byref(params), C.sizeof(q))
    q.n_phi_bins = 0
    for k in range(N_STAGES):
        q.grid_per_sm[k] = 0
        q.block_threads[k] = 0
    return hashlib.sha256(C.string_at(C.byref(q), C.sizeof(q))).hexdigest()[:16]


def cache_key(params, n_events: int, n_hits: int, gpu: str = "") -> str:
    """GPU name, configuration hash, events and hits (to 1/16 decades)."""
    name = "".join(c if c.isalnum() else "_" for c in gpu) or "any"
    return (f"{name}-{config_hash(params)}-E{n_events}"
            f"-N{round(16 * math.log10(max(n_hits, 1)))}")


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
              bins: Sequence[int] = BINS, grids: Sequence[int] = GRIDS, blocks: dict = BLOCKS,
              cache: str | None = None, flush=None, gpu: str | None = None):
    """Tune n_phi_bins, grid_per_sm and block_threads of `params` on this batch (device inputs);
    returns a copy of params with the choice filled in and a dict describing it.  `flush()`
    (optional) runs before every timed step (an L2 flush on the same stream).  A setting's time is
    the fastest of its `reps` steps: interference from other work on the device only ever adds
    time.  `gpu` names the device in the cache key (default: torch's name of the current CUDA
    device)."""
    import numpy as np

    from . import pxr

    n_events = len(hit_offsets) - 1
    n_hits = int(hit_offsets[-1])
    if gpu is None:
        import torch
        gpu = torch.cuda.get_device_name(torch.cuda.current_device())
    key = cache_key(params, n_events, n_hits, gpu)
    if cache:
        hit = load_cache(cache).get(key)
        if hit:
            return (_with(params, hit["n_phi_bins"], hit["grid_per_sm"], hit["block_threads"]),
                    dict(hit, cached=True))

    def measure(nb, grid, block):
        p = _with(params, nb, grid, block)
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

    nb, grid, block, t, calls = search(measure, bins, grids, blocks=blocks)
    info = {"n_phi_bins": nb, "grid_per_sm": list(grid), "block_threads": list(block),
            "step_ms": t, "trials": calls, "stages": list(pxr.STAGES), "gpu": gpu, "key": key}
    if cache:
        store_cache(cache, key, info)
    return _with(params, nb, grid, block), info


def _with(params, nb, grid, block=None):
    import ctypes as C
    from . import pxr
    p = pxr.pxr_params()
    C.memmove(C.byref(p), C.byref(params), C.sizeof(p))
    p.n_phi_bins = int(nb)
    for k, v in enumerate(grid):
        p.grid_per_sm[k] = int(v)
    for k, v in enumerate(block or ()):
        p.block_threads[k] = int(v)
    return p
