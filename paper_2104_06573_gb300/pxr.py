"""ctypes binding of the pxr C ABI (include/pxr.h): argument marshalling only.

Every step of the reconstruction runs in the CUDA library paper_2104_06573_gb300/_build/libpxr.so
(with PXR_CHECKED=1 in the environment: libpxr_checked.so, the same library with device-side
bounds checks that report PXR_EBOUNDS instead of touching memory outside an array).
There is no CPU fallback: if the library is missing or no GB300 is present, the calls raise.
Device pointers may be passed as integers or as torch tensors (their data_ptr() is used).
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpxr_checked.so" if os.environ.get("PXR_CHECKED") == "1"
                        else "libpxr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pxr.h")

MAX_LAYERS, MAX_PAIRS, MAX_HITS = 16, 32, 6
OK, EINVAL, EAGAIN, ENOMEM, EOVERFLOW, ETIMEDOUT, ECUDA, ETRUNC, ENOTFOUND, EBUSY, EBOUNDS = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10)
CUT_FP64, CUT_FP32 = 0, 1
FIT_FP64, FIT_MIXED, FIT_FP32, FIT_RIEMANN, FIT_SPLIT = 0, 1, 2, 3, 4
PRESET_BARREL, PRESET_PHASE1 = 0, 1
NONE = 0xFFFFFFFF


class PxrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pxr error {code}: {msg}")
        self.code = code


class pxr_params(C.Structure):
    _fields_ = [("n_layers", C.c_uint32), ("layer_is_disk", C.c_uint8 * MAX_LAYERS),
                ("n_pairs", C.c_uint32), ("pair_inner", C.c_uint8 * MAX_PAIRS),
                ("pair_outer", C.c_uint8 * MAX_PAIRS), ("root_layer_mask", C.c_uint32),
                ("drop_suffixes", C.c_uint32), ("min_hits", C.c_uint32),
                ("max_hits", C.c_uint32), ("cut_mode", C.c_uint32), ("fit_mode", C.c_uint32),
                ("phi_window", C.c_double), ("cos_phi_window", C.c_double),
                ("theta_cut", C.c_double), ("dca_cut", C.c_double), ("bfield", C.c_double),
                ("sigma_rphi", C.c_double), ("sigma_z", C.c_double),
                ("x_over_x0", C.c_double), ("n_phi_bins", C.c_uint32),
                ("max_cells_per_event", C.c_uint32), ("max_tuples_per_event", C.c_uint32),
                ("grid_per_sm", C.c_uint32 * 6), ("block_threads", C.c_uint32 * 6),
                ("pt_min", C.c_double), ("chi2_max", C.c_double),
                ("clean_shared", C.c_uint32), ("fit_cov", C.c_uint32),
                ("vertexing", C.c_uint32), ("vtx_min_tracks", C.c_uint32), ("vtx_gap", C.c_double)]


class pxr_config(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget_bytes", C.c_size_t), ("arena", C.c_void_p),
                ("stream", C.c_void_p), ("max_batch_events", C.c_uint32),
                ("max_batch_hits", C.c_uint32), ("max_inflight", C.c_uint32),
                ("keep_debug", C.c_uint32)]


class pxr_tracks(C.Structure):
    # the array fields are raw addresses (the C struct's typed pointers have the same layout)
    _fields_ = [("capacity", C.c_uint32), ("n_tracks", C.c_uint32), ("status", C.c_int32),
                ("n_hits", C.c_void_p), ("hit_idx", C.c_void_p), ("pt", C.c_void_p),
                ("phi", C.c_void_p), ("cot_theta", C.c_void_p), ("dxy", C.c_void_p),
                ("dz", C.c_void_p), ("chi2", C.c_void_p), ("charge", C.c_void_p),
                ("fit_status", C.c_void_p), ("quality", C.c_void_p), ("cov", C.c_void_p),
                ("vertex", C.c_void_p), ("n_vertices", C.c_uint32), ("vtx_z", C.c_void_p),
                ("vtx_z_err", C.c_void_p), ("vtx_sum_pt2", C.c_void_p),
                ("vtx_n_tracks", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def declared_functions():
    """Names of the functions declared in include/pxr.h."""
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pxr_\w+)\s*\(", src, re.M)))


def load(build_if_missing: bool = False):
    """Load libpxr.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError(f"{LIB_PATH} not built: run __graft_entry__.build()")
            from . import build_lib
            build_lib.build()
        L = C.CDLL(LIB_PATH)
        vp, u32, i32 = C.c_void_p, C.c_uint32, C.c_int
        P = C.POINTER
        sig = {
            "pxr_version": (C.c_char_p, []),
            "pxr_last_error": (C.c_char_p, []),
            "pxr_params_init": (i32, [P(pxr_params), i32]),
            "pxr_params_check": (i32, [P(pxr_params)]),
            "pxr_create": (i32, [P(pxr_config), P(vp)]),
            "pxr_destroy": (None, [vp]),
            "pxr_submit_event": (i32, [vp, vp, vp, vp, vp, u32, P(pxr_params), P(C.c_uint64)]),
            "pxr_submit_events": (i32, [vp, u32, vp, vp, vp, vp, vp, P(pxr_params), vp]),
            "pxr_poll": (i32, [vp, P(C.c_uint64), u32, P(u32), i32]),
            "pxr_fetch_events": (i32, [vp, u32, vp, vp, vp, vp, P(pxr_tracks)]),
            "pxr_fetch_tracks": (i32, [vp, C.c_uint64, P(pxr_tracks)]),
            "pxr_fetch_debug": (i32, [vp, C.c_uint64, i32, P(u32), u32, P(u32)]),
            "pxr_plan_create": (i32, [vp, u32, P(u32), vp, vp, vp, vp, P(pxr_params), i32,
                                      P(vp)]),
            "pxr_plan_run": (i32, [vp, vp]),
            "pxr_plan_tracks": (i32, [vp, u32, P(pxr_tracks)]),
            "pxr_plan_debug": (i32, [vp, u32, i32, P(u32), u32, P(u32)]),
            "pxr_plan_launches": (i32, [vp]),
            "pxr_plan_count_ca_tests": (i32, [vp, vp, P(C.c_uint64)]),
            "pxr_plan_counts": (i32, [vp, P(u32)]),
            "pxr_plan_stage_ms": (i32, [vp, P(C.c_float), i32, P(i32)]),
            "pxr_plan_destroy": (None, [vp]),
            "pxr_fit_batch": (i32, [vp, u32, vp, vp, vp, vp, vp, u32, P(pxr_params), vp, vp, vp,
                                    vp, vp, vp, vp, vp, vp]),
            "pxr_doublets_noalloc": (i32, [vp, vp, vp, vp, u32, P(pxr_params), vp, vp, u32, vp,
                                           vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(rc):
    if rc != OK:
        raise PxrError(rc, load().pxr_last_error().decode())
    return rc


def ptr(x):
    """Address of a torch tensor, a numpy array, a torch stream or an integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "cuda_stream"):          # torch.cuda.Stream
        return x.cuda_stream
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


# -- parameters ------------------------------------------------------------------------------
STAGES = ("sort", "doublets", "connect", "walk", "select", "fit")   # PXR_STAGE_* order


def params_from(p, cut_mode=CUT_FP64, fit_mode=FIT_FP64, n_phi_bins=0, max_cells=0,
                max_tuples=0, grid_per_sm=None, pt_min=0.0, chi2_max=0.0,
                clean_shared=False, fit_cov=False, vertexing=False, vtx_min_tracks=2,
                vtx_gap=0.05) -> pxr_params:
    """Marshal any object with the workload fields (n_layers, layer_is_disk, pairs, root_mask,
    drop_suffixes, min_hits, max_hits, phi_window, cos_phi_window, cuts, field, errors).
    grid_per_sm: optional CTAs-per-SM caps per stage (STAGES order; 0 = built-in).
    pt_min, chi2_max, clean_shared: the track selection (0 / False: off); fit_cov: compute the
    tracks' covariances (the fetched 'cov' field, [n, 15]; NaN otherwise); vertexing,
    vtx_min_tracks, vtx_gap: primary vertices from the kept tracks."""
    o = pxr_params()
    o.n_layers = p.n_layers
    for i, v in enumerate(p.layer_is_disk):
        o.layer_is_disk[i] = int(v)
    o.n_pairs = len(p.pairs)
    for i, (a, b) in enumerate(p.pairs):
        o.pair_inner[i] = a
        o.pair_outer[i] = b
    o.root_layer_mask = p.root_mask
    o.drop_suffixes = 1 if p.drop_suffixes else 0
    o.min_hits, o.max_hits = p.min_hits, p.max_hits
    o.cut_mode, o.fit_mode = cut_mode, fit_mode
    o.phi_window, o.cos_phi_window = p.phi_window, p.cos_phi_window
    o.theta_cut, o.dca_cut = p.theta_cut, p.dca_cut
    o.bfield, o.sigma_rphi, o.sigma_z, o.x_over_x0 = p.bfield, p.sigma_rphi, p.sigma_z, p.x_over_x0
    o.n_phi_bins = n_phi_bins
    o.max_cells_per_event, o.max_tuples_per_event = max_cells, max_tuples
    for k, v in enumerate(grid_per_sm or ()):
        o.grid_per_sm[k] = int(v)
    o.pt_min, o.chi2_max = float(pt_min), float(chi2_max)
    o.clean_shared = 1 if clean_shared else 0
    o.fit_cov = 1 if fit_cov else 0
    o.vertexing = 1 if vertexing else 0
    o.vtx_min_tracks, o.vtx_gap = int(vtx_min_tracks), float(vtx_gap)
    return o


Q_GOOD, Q_KEPT = 1, 2             # pxr_tracks.quality bits


def pxr_params_check(p: pxr_params) -> None:
    _check(load().pxr_params_check(C.byref(p)))


def pxr_params_init(preset: int) -> pxr_params:
    p = pxr_params()
    _check(load().pxr_params_init(C.byref(p), preset))
    return p


# -- tracks ----------------------------------------------------------------------------------
TRACK_FIELDS = ("pt", "phi", "cot_theta", "dxy", "dz", "chi2")


# per-track record layout of one fetch: (field, numpy dtype, values per track)
_TRACK_LAYOUT = (("n_hits", np.uint8, 1), ("hit_idx", np.uint32, MAX_HITS),
                 ("pt", np.float64, 1), ("phi", np.float64, 1), ("cot_theta", np.float64, 1),
                 ("dxy", np.float64, 1), ("dz", np.float64, 1), ("chi2", np.float64, 1),
                 ("charge", np.int8, 1), ("fit_status", np.int8, 1), ("quality", np.uint8, 1),
                 ("vertex", np.int32, 1), ("vtx_z", np.float64, 1), ("vtx_z_err", np.float64, 1),
                 ("vtx_sum_pt2", np.float64, 1), ("vtx_n_tracks", np.uint32, 1),
                 ("cov", np.float64, 15))
_VERTEX_FIELDS = ("vtx_z", "vtx_z_err", "vtx_sum_pt2", "vtx_n_tracks")


def _read_tracks(call, cov=False) -> dict:
    """Ask for the track count, then fill arrays of exactly that size (one allocation, the
    library writes straight into it; nothing is copied afterwards).  The covariance array is
    requested only with cov (it holds NaN unless the covariance was computed)."""
    layout = _TRACK_LAYOUT if cov else _TRACK_LAYOUT[:-1]
    t = pxr_tracks()
    t.capacity = 0
    rc = call(t)
    if rc not in (OK, ETRUNC):
        _check(rc)
    n = t.n_tracks
    if rc == OK:                                        # no tracks: the call is complete
        out = {"n": 0, "status": t.status, "n_vertices": 0}
        for name, dt, k in layout:
            out[name] = np.zeros((0, k) if k > 1 else 0, dt)
        return out
    while True:
        sizes = [np.dtype(dt).itemsize * k * max(n, 1) for _, dt, k in layout]
        offs = np.concatenate([[0], np.cumsum([(z + 15) // 16 * 16 for z in sizes])])
        buf = np.empty(int(offs[-1]), np.uint8)
        base = buf.ctypes.data
        t = pxr_tracks()
        t.capacity = n
        for (name, _, _), off in zip(layout, offs[:-1]):
            setattr(t, name, base + int(off))
        rc = call(t)
        if rc == ETRUNC:                                # (the count cannot grow; defensive)
            n = t.n_tracks
            continue
        _check(rc)
        out = {"n": n, "status": t.status, "n_vertices": t.n_vertices}
        for (name, dt, k), off in zip(layout, offs[:-1]):
            a = np.frombuffer(buf, dt, n * k, int(off))
            out[name] = a.reshape(n, k) if k > 1 else a
        for name in _VERTEX_FIELDS:                      # the vertex arrays hold n_vertices
            out[name] = out[name][:t.n_vertices]
        return out


def _read_debug(call, what, cap_hint=1 << 16) -> np.ndarray:
    per = (2, 3, MAX_HITS)[what]
    cap = cap_hint
    while True:
        buf = np.zeros(cap, np.uint32)
        n = C.c_uint32(0)
        rc = call(buf.ctypes.data_as(C.POINTER(C.c_uint32)), cap, C.byref(n))
        if rc == ETRUNC:
            cap = n.value * per + 16
            continue
        _check(rc)
        return buf[: n.value * per].reshape(n.value, per).copy()


# -- context ---------------------------------------------------------------------------------
class Context:
    """pxr_create / pxr_destroy and the serving calls."""

    def __init__(self, device=0, mem_budget_bytes=2 << 30, arena=None, stream=None,
                 max_batch_events=256, max_batch_hits=0, max_inflight=2, keep_debug=False):
        L = load()
        cfg = pxr_config()
        cfg.device = device
        cfg.mem_budget_bytes = mem_budget_bytes
        cfg.arena = ptr(arena)
        cfg.stream = ptr(stream)
        cfg.max_batch_events = max_batch_events
        cfg.max_batch_hits = max_batch_hits
        cfg.max_inflight = max_inflight
        cfg.keep_debug = 1 if keep_debug else 0
        h = C.c_void_p()
        _check(L.pxr_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self._arena_ref = arena          # keep caller memory alive

    def close(self):
        if self.h:
            load().pxr_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # serving
    def pxr_submit_event(self, x, y, z, layer, params: pxr_params) -> int:
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        z = np.ascontiguousarray(z, np.float32)
        layer = np.ascontiguousarray(layer, np.uint16)
        t = C.c_uint64(0)
        _check(load().pxr_submit_event(self.h, x.ctypes.data, y.ctypes.data, z.ctypes.data,
                                       layer.ctypes.data, len(x), C.byref(params), C.byref(t)))
        return t.value

    def try_submit_event(self, x, y, z, layer, params):
        """Like pxr_submit_event but returns None on PXR_EAGAIN (budget full now)."""
        try:
            return self.pxr_submit_event(x, y, z, layer, params)
        except PxrError as e:
            if e.code == EAGAIN:
                return None
            raise

    def pxr_submit_events(self, hit_offsets, x, y, z, layer, params: pxr_params) -> list:
        """Many events in one call (hits back to back, event e at [hit_offsets[e],
        hit_offsets[e+1])); returns their tickets."""
        off = np.ascontiguousarray(hit_offsets, np.uint32)
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        z = np.ascontiguousarray(z, np.float32)
        layer = np.ascontiguousarray(layer, np.uint16)
        n = len(off) - 1
        t = np.zeros(max(n, 1), np.uint64)
        _check(load().pxr_submit_events(self.h, n, off.ctypes.data, x.ctypes.data,
                                        y.ctypes.data, z.ctypes.data, layer.ctypes.data,
                                        C.byref(params), t.ctypes.data))
        return [int(v) for v in t[:n]]

    def pxr_fetch_events(self, tickets, cov: bool = False, out=None) -> dict:
        """Tracks of finished events in one set of arrays: 'track_offsets' [n+1] delimit each
        event's rows, 'vertex_offsets' [n+1] its vertices, 'event_status' [n] its status.
        out: optional dict of preallocated arrays (as returned), reused when large enough."""
        tk = np.ascontiguousarray(tickets, np.uint64)
        n = len(tk)
        toff = np.zeros(n + 1, np.uint32)
        voff = np.zeros(n + 1, np.uint32)
        st = np.zeros(max(n, 1), np.int32)
        layout = _TRACK_LAYOUT if cov else _TRACK_LAYOUT[:-1]

        def call(t):
            return load().pxr_fetch_events(self.h, n, tk.ctypes.data, toff.ctypes.data,
                                           voff.ctypes.data, st.ctypes.data, C.byref(t))
        cap = 0
        if out is not None:
            cap = min(len(out[name]) for name, _, _ in layout)
        while True:
            if out is None or cap == 0:
                t = pxr_tracks()
                t.capacity = 0
                rc = call(t)
                if rc not in (OK, ETRUNC):
                    _check(rc)
                if rc == OK:
                    res = {name: np.zeros((0, k) if k > 1 else 0, dt) for name, dt, k in layout}
                    break
                cap = t.n_tracks
                out = {name: np.empty((cap, k) if k > 1 else cap, dt) for name, dt, k in layout}
            t = pxr_tracks()
            t.capacity = cap
            for name, _, _ in layout:
                setattr(t, name, out[name].ctypes.data)
            rc = call(t)
            if rc == ETRUNC:
                out, cap = None, 0
                continue
            _check(rc)
            res = {name: out[name][:t.n_tracks] for name, _, _ in layout}
            for name in _VERTEX_FIELDS:
                res[name] = out[name][:t.n_vertices]
            break
        res.update(track_offsets=toff, vertex_offsets=voff, event_status=st[:n],
                   n=int(toff[-1]), status=int(st[:n].min()) if n else OK)
        return res

    def pxr_poll(self, cap=4096, timeout_us=0) -> list:
        done = (C.c_uint64 * cap)()
        n = C.c_uint32(0)
        _check(load().pxr_poll(self.h, done, cap, C.byref(n), timeout_us))
        return [done[i] for i in range(n.value)]

    def pxr_fetch_tracks(self, ticket: int, cov: bool = False) -> dict:
        """Tracks of a finished event (cov: also the covariances, if they were computed)."""
        return _read_tracks(lambda t: load().pxr_fetch_tracks(self.h, ticket, C.byref(t)), cov)

    def pxr_fetch_debug(self, ticket: int, what: int) -> np.ndarray:
        return _read_debug(lambda b, cap, n: load().pxr_fetch_debug(self.h, ticket, what, b, cap,
                                                                    n), what)

    def pxr_fit_batch(self, m, nh, x, y, z, layer, stride, params, out, stream=None):
        """Fit-only path; all arrays are device tensors/pointers; out: dict of device outputs
        (pt, phi, cot_theta, dxy, dz, chi2, charge, fit_status)."""
        _check(load().pxr_fit_batch(self.h, m, ptr(nh), ptr(x), ptr(y), ptr(z), ptr(layer),
                                    stride, C.byref(params), ptr(out["pt"]), ptr(out["phi"]),
                                    ptr(out["cot_theta"]), ptr(out["dxy"]), ptr(out["dz"]),
                                    ptr(out["chi2"]), ptr(out["charge"]),
                                    ptr(out["fit_status"]), ptr(stream)))


class Plan:
    """Device-resident batch: pxr_plan_create / run / tracks / debug / destroy."""

    def __init__(self, ctx: Context, hit_offsets, x, y, z, layer, params: pxr_params,
                 use_graph=True):
        off = np.ascontiguousarray(hit_offsets, np.uint32)
        h = C.c_void_p()
        _check(load().pxr_plan_create(ctx.h, len(off) - 1,
                                      off.ctypes.data_as(C.POINTER(C.c_uint32)), ptr(x), ptr(y),
                                      ptr(z), ptr(layer), C.byref(params),
                                      1 if use_graph else 0, C.byref(h)))
        self.h = h
        self.ctx = ctx
        self.n_events = len(off) - 1
        self.with_cov = bool(params.fit_cov)
        self._refs = (x, y, z, layer)      # the caller's device inputs stay alive

    def pxr_plan_run(self, stream=None):
        _check(load().pxr_plan_run(self.h, ptr(stream)))

    def pxr_plan_tracks(self, e: int, cov=None) -> dict:
        """Tracks of event e (cov: with the covariance array; default: when the plan's
        parameters ask for covariances)."""
        return _read_tracks(lambda t: load().pxr_plan_tracks(self.h, e, C.byref(t)),
                            self.with_cov if cov is None else cov)

    def pxr_plan_debug(self, e: int, what: int) -> np.ndarray:
        return _read_debug(lambda b, cap, n: load().pxr_plan_debug(self.h, e, what, b, cap, n),
                           what)

    def pxr_plan_launches(self) -> int:
        return load().pxr_plan_launches(self.h)

    def pxr_plan_count_ca_tests(self, stream=None) -> tuple:
        """One untimed run with the CA stage counting its work: (r-z tests, DCA tests)."""
        out = (C.c_uint64 * 2)()
        _check(load().pxr_plan_count_ca_tests(self.h, ptr(stream), out))
        return int(out[0]), int(out[1])

    def pxr_plan_counts(self) -> dict:
        """Per-event counters of the last run: cells, edges, tuples, flags, tracks."""
        out = np.zeros(5 * self.n_events, np.uint32)
        _check(load().pxr_plan_counts(self.h, out.ctypes.data_as(C.POINTER(C.c_uint32))))
        out = out.reshape(5, self.n_events)
        return dict(zip(("cells", "edges", "tuples", "flags", "tracks"), out))

    def pxr_plan_stage_ms(self) -> list:
        ms = (C.c_float * 8)()
        n = C.c_int(0)
        _check(load().pxr_plan_stage_ms(self.h, ms, 8, C.byref(n)))
        return [ms[i] for i in range(n.value)]

    def close(self):
        if self.h:
            if self.ctx.h:                 # a closed context has destroyed its plans already
                load().pxr_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pxr_doublets_noalloc(x, y, z, layer, n_hits, params, cells_inner, cells_outer, cap, n_cells,
                         flags=None, stream=None):
    """Allocation-free doublets of one event (all arrays device tensors or pointers)."""
    _check(load().pxr_doublets_noalloc(ptr(x), ptr(y), ptr(z), ptr(layer), n_hits,
                                       C.byref(params), ptr(cells_inner), ptr(cells_outer), cap,
                                       ptr(n_cells), ptr(flags), ptr(stream)))


def pxr_version() -> str:
    return load().pxr_version().decode()
