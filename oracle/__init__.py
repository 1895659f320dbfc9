"""FP64 CPU oracle of the pixel-track hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this package.  The
product library never loads it.  It shares no code with the CUDA path; the only common input is
the synthetic event generator.

`build()` compiles `pxr_oracle.c` with gcc (`-O2 -ffp-contract=off`: no fused multiply-add, so that
every cut quantity is the exact IEEE operation sequence written in the C source).  The functions
below are thin ctypes wrappers; all arithmetic lives in the C file, except the track selection
(`select_tracks`), written here in plain Python from its definition.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pxr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
MAXH = 8
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (seconds)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(C.Structure):
    _fields_ = [("n_layers", C.c_uint32), ("layer_is_disk", C.c_uint8 * 16),
                ("n_pairs", C.c_uint32), ("pair_inner", C.c_uint8 * 32),
                ("pair_outer", C.c_uint8 * 32), ("root_mask", C.c_uint32),
                ("drop_suffixes", C.c_uint32), ("min_hits", C.c_uint32),
                ("max_hits", C.c_uint32), ("cos_phi_window", C.c_double),
                ("theta_cut", C.c_double), ("dca_cut", C.c_double), ("bfield", C.c_double),
                ("sigma_rphi", C.c_double), ("sigma_z", C.c_double), ("x_over_x0", C.c_double)]


class OrcTrack(C.Structure):
    _fields_ = [("pt", C.c_double), ("phi", C.c_double), ("cot_theta", C.c_double),
                ("dxy", C.c_double), ("dz", C.c_double), ("chi2", C.c_double),
                ("charge", C.c_int32), ("status", C.c_int32)]


class OrcResult(C.Structure):
    _fields_ = [("n_hits", C.c_uint32), ("n_cells", C.c_uint32),
                ("cell_in", C.POINTER(C.c_uint32)), ("cell_out", C.POINTER(C.c_uint32)),
                ("n_edges", C.c_uint32), ("edge_a", C.POINTER(C.c_uint32)),
                ("edge_b", C.POINTER(C.c_uint32)), ("n_tuples", C.c_uint32),
                ("tup_n", C.POINTER(C.c_uint8)), ("tup_hits", C.POINTER(C.c_uint32)),
                ("fit", C.POINTER(OrcTrack))]


TRACK_DTYPE = np.dtype([("pt", "f8"), ("phi", "f8"), ("cot_theta", "f8"), ("dxy", "f8"),
                        ("dz", "f8"), ("chi2", "f8"), ("charge", "i4"), ("status", "i4")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            d = C.c_double
            L.orc_radius.restype = d
            L.orc_radius.argtypes = [d, d]
            L.orc_doublet_pass.restype = C.c_int
            L.orc_doublet_pass.argtypes = [d] * 5
            L.orc_theta_pass.restype = C.c_int
            L.orc_theta_pass.argtypes = [d] * 7
            L.orc_dca.restype = d
            L.orc_dca.argtypes = [d] * 6
            L.orc_dca_pass.restype = C.c_int
            L.orc_dca_pass.argtypes = [d] * 7
            dp = C.POINTER(C.c_double)
            L.orc_bl_solve.restype = C.c_int
            L.orc_bl_solve.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int, dp, dp]
            L.orc_fit_one.restype = C.c_int
            L.orc_fit_one.argtypes = [C.c_int, dp, dp, dp, C.POINTER(C.c_uint16),
                                      C.POINTER(OrcParams), C.POINTER(OrcTrack)]
            L.orc_fit_cov.restype = C.c_int
            L.orc_fit_cov.argtypes = [C.c_int, dp, dp, dp, C.POINTER(C.c_uint16),
                                      C.POINTER(OrcParams), C.POINTER(OrcTrack), dp]
            L.orc_riemann_batch.restype = None
            L.orc_riemann_batch.argtypes = [C.c_uint32, C.POINTER(C.c_uint8), dp, dp, dp,
                                            C.POINTER(C.c_uint16), C.c_uint32,
                                            C.POINTER(OrcParams), C.POINTER(OrcTrack)]
            L.orc_fit_batch.restype = None
            L.orc_fit_batch.argtypes = [C.c_uint32, C.POINTER(C.c_uint8), dp, dp, dp,
                                        C.POINTER(C.c_uint16), C.c_uint32,
                                        C.POINTER(OrcParams), C.POINTER(OrcTrack)]
            L.orc_reconstruct.restype = C.POINTER(OrcResult)
            L.orc_reconstruct.argtypes = [C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                          C.POINTER(C.c_float), C.POINTER(C.c_uint16),
                                          C.POINTER(OrcParams), C.c_int]
            L.orc_reconstruct_w.restype = C.POINTER(OrcResult)
            L.orc_reconstruct_w.argtypes = [C.c_uint32, C.POINTER(C.c_float),
                                            C.POINTER(C.c_float), C.POINTER(C.c_float),
                                            C.POINTER(C.c_uint16), C.POINTER(OrcParams), C.c_int,
                                            C.c_int]
            L.orc_free.restype = None
            L.orc_free.argtypes = [C.POINTER(OrcResult)]
            _lib = L
    return _lib


def make_params(p) -> OrcParams:
    """Marshal any object with the workload fields (geometry, pairs, cuts, fit constants)."""
    o = OrcParams()
    o.n_layers = p.n_layers
    for i, v in enumerate(p.layer_is_disk):
        o.layer_is_disk[i] = int(v)
    o.n_pairs = len(p.pairs)
    for i, (a, b) in enumerate(p.pairs):
        o.pair_inner[i] = a
        o.pair_outer[i] = b
    o.root_mask = p.root_mask
    o.drop_suffixes = 1 if p.drop_suffixes else 0
    o.min_hits = p.min_hits
    o.max_hits = p.max_hits
    o.cos_phi_window = p.cos_phi_window
    o.theta_cut = p.theta_cut
    o.dca_cut = p.dca_cut
    o.bfield = p.bfield
    o.sigma_rphi = p.sigma_rphi
    o.sigma_z = p.sigma_z
    o.x_over_x0 = p.x_over_x0
    return o


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# -- single quantities -----------------------------------------------------------------------
def radius(x, y):
    return lib().orc_radius(float(x), float(y))


def doublet_pass(xi, yi, xo, yo, cw) -> bool:
    return bool(lib().orc_doublet_pass(xi, yi, xo, yo, cw))


def theta_pass(ri, zi, rj, zj, rk, zk, t) -> bool:
    return bool(lib().orc_theta_pass(ri, zi, rj, zj, rk, zk, t))


def dca(xi, yi, xj, yj, xk, yk) -> float:
    return lib().orc_dca(xi, yi, xj, yj, xk, yk)


def bl_solve(s, meas, w, kvar, curv: bool):
    """Broken-line normal-equation solve; returns (solution, chi2) or None on failure."""
    n = len(s)
    s = np.ascontiguousarray(s, np.float64)
    meas = np.ascontiguousarray(meas, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    kvar = np.ascontiguousarray(kvar, np.float64)
    x = np.zeros(n + 1, np.float64)
    chi2 = C.c_double(0.0)
    rc = lib().orc_bl_solve(n, _ptr(s, C.c_double), _ptr(meas, C.c_double), _ptr(w, C.c_double),
                            _ptr(kvar, C.c_double), 1 if curv else 0, _ptr(x, C.c_double),
                            C.byref(chi2))
    if rc != 0:
        return None
    return (x if curv else x[:n]), chi2.value


# -- fits ------------------------------------------------------------------------------------
def fit_one(X, Y, Z, layers, params) -> np.void:
    n = len(X)
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    Z = np.ascontiguousarray(Z, np.float64)
    L = np.ascontiguousarray(layers, np.uint16)
    P = make_params(params)
    out = OrcTrack()
    lib().orc_fit_one(n, _ptr(X, C.c_double), _ptr(Y, C.c_double), _ptr(Z, C.c_double),
                      _ptr(L, C.c_uint16), C.byref(P), C.byref(out))
    rec = np.zeros((), TRACK_DTYPE)
    for k in TRACK_DTYPE.names:
        rec[k] = getattr(out, k)
    return rec


def fit_batch(nh, X, Y, Z, layers, params) -> np.ndarray:
    """Fit m ntuplets; X, Y, Z, layers are [m, k] arrays (k <= 8), nh the hit counts."""
    nh = np.ascontiguousarray(nh, np.uint8)
    m, k = np.shape(X)
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    Z = np.ascontiguousarray(Z, np.float64)
    L = np.ascontiguousarray(layers, np.uint16)
    P = make_params(params)
    out = np.zeros(m, TRACK_DTYPE)
    lib().orc_fit_batch(m, _ptr(nh, C.c_uint8), _ptr(X, C.c_double), _ptr(Y, C.c_double),
                        _ptr(Z, C.c_double), _ptr(L, C.c_uint16), k, C.byref(P),
                        out.ctypes.data_as(C.POINTER(OrcTrack)))
    return out


def riemann_batch(nh, X, Y, Z, layers, params) -> np.ndarray:
    """Riemann fits of m ntuplets ([m, k] arrays as for fit_batch)."""
    nh = np.ascontiguousarray(nh, np.uint8)
    m, k = np.shape(X)
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    Z = np.ascontiguousarray(Z, np.float64)
    L = np.ascontiguousarray(layers, np.uint16)
    P = make_params(params)
    out = np.zeros(m, TRACK_DTYPE)
    lib().orc_riemann_batch(m, _ptr(nh, C.c_uint8), _ptr(X, C.c_double), _ptr(Y, C.c_double),
                            _ptr(Z, C.c_double), _ptr(L, C.c_uint16), k, C.byref(P),
                            out.ctypes.data_as(C.POINTER(OrcTrack)))
    return out


COV_PARAMS = ("qoverpt", "phi", "cot_theta", "dxy", "dz")


def fit_cov_batch(nh, X, Y, Z, layers, params):
    """Fits and covariances of (q/pT, phi, cot, dxy, dz) of m ntuplets ([m, k] arrays as for
    fit_batch).  Returns (fits, cov [m, 15] upper triangles row by row; NaN where the fit or the
    covariance failed).  The covariance is the fitted values' (the inverse normal matrices of the
    two broken lines) propagated through the conversion linearised by central differences."""
    nh = np.ascontiguousarray(nh, np.uint8)
    m = len(nh)
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    Z = np.ascontiguousarray(Z, np.float64)
    L = np.ascontiguousarray(layers, np.uint16)
    P = make_params(params)
    fits = np.zeros(m, TRACK_DTYPE)
    cov = np.full((m, 15), np.nan)
    out = OrcTrack()
    c15 = (C.c_double * 15)()
    lb = lib()
    for t in range(m):
        n = int(nh[t])
        rc = lb.orc_fit_cov(n, _ptr(X[t], C.c_double), _ptr(Y[t], C.c_double),
                            _ptr(Z[t], C.c_double), _ptr(L[t], C.c_uint16), C.byref(P),
                            C.byref(out), c15)
        for k in TRACK_DTYPE.names:
            fits[t][k] = getattr(out, k)
        if rc == 0:
            cov[t] = np.frombuffer(c15, np.float64)
    return fits, cov


def cov_matrix(c15):
    """Full symmetric 5 x 5 matrices from upper triangles ([..., 15] -> [..., 5, 5])."""
    c15 = np.asarray(c15)
    M = np.zeros(c15.shape[:-1] + (5, 5))
    k = 0
    for i in range(5):
        for j in range(i, 5):
            M[..., i, j] = M[..., j, i] = c15[..., k]
            k += 1
    return M


# -- whole event -----------------------------------------------------------------------------
def reconstruct(x, y, z, layer, params, stage: int = 4, windowed: bool = False) -> dict:
    """Doublets, CA edges, ntuplets and fits of one event (caller hit order).  windowed: the
    doublets by the azimuth-sorted windowed search (the same cells in the same order; the timed
    CPU baseline uses it) instead of every hit pair.

    Returns a dict with 'cells' [nc, 2] (inner, outer hit), 'edges' [ne, 2] (cell A, cell B),
    'tuples' [nt, 8] (hits, 0xFFFFFFFF padded), 'tuple_n' [nt], 'fits' (structured [nt]).
    """
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    layer = np.ascontiguousarray(layer, np.uint16)
    P = make_params(params)
    L = lib()
    rp = L.orc_reconstruct_w(len(x), _ptr(x, C.c_float), _ptr(y, C.c_float),
                             _ptr(z, C.c_float), _ptr(layer, C.c_uint16), C.byref(P), stage,
                             1 if windowed else 0)
    if not rp:
        raise ValueError("oracle rejected the input (layer id, limits) or ran out of memory")
    try:
        r = rp.contents
        out = {}
        nc = r.n_cells
        cells = np.zeros((nc, 2), np.uint32)
        if nc:
            cells[:, 0] = np.ctypeslib.as_array(r.cell_in, (nc,))
            cells[:, 1] = np.ctypeslib.as_array(r.cell_out, (nc,))
        out["cells"] = cells
        if stage >= 2:
            ne = r.n_edges
            edges = np.zeros((ne, 2), np.uint32)
            if ne:
                edges[:, 0] = np.ctypeslib.as_array(r.edge_a, (ne,))
                edges[:, 1] = np.ctypeslib.as_array(r.edge_b, (ne,))
            out["edges"] = edges
        if stage >= 3:
            nt = r.n_tuples
            tup = np.full((nt, MAXH), 0xFFFFFFFF, np.uint32)
            tn = np.zeros(nt, np.uint8)
            if nt:
                tup[:] = np.ctypeslib.as_array(r.tup_hits, (nt * MAXH,)).reshape(nt, MAXH)
                tn[:] = np.ctypeslib.as_array(r.tup_n, (nt,))
            out["tuples"] = tup
            out["tuple_n"] = tn
        if stage >= 4:
            nt = r.n_tuples
            fits = np.zeros(nt, TRACK_DTYPE)
            if nt:
                raw = np.ctypeslib.as_array(C.cast(r.fit, C.POINTER(C.c_uint8)),
                                            (nt * C.sizeof(OrcTrack),))
                fits[:] = np.frombuffer(raw.tobytes(), TRACK_DTYPE)
            out["fits"] = fits
        return out
    finally:
        L.orc_free(rp)


# -- track selection -------------------------------------------------------------------------
Q_GOOD, Q_KEPT = 1, 2


def select_tracks(tuples, tuple_n, fits, pt_min=0.0, chi2_max=0.0, clean_shared=False):
    """Quality bits of each fitted track (the selection step that follows the fit; the paper
    names the Tracks product, §2, but defines no selection, so this is the library's reading).

    GOOD: fit status 0, a finite chi2, pT >= pt_min (no cut when pt_min is 0) and chi2/ndof <=
    chi2_max (no cut when chi2_max is 0), with ndof = max(2 n - 5, 1) for n hits (two
    measurements per hit, five helix parameters).
    KEPT: GOOD and, with clean_shared, no other GOOD track that shares a hit with it ranks
    strictly better; a track ranks better when it has more hits, or as many hits and a smaller
    chi2/ndof.  One round: a track is dropped by a better one even when that one is dropped in
    turn.  Without clean_shared, KEPT = GOOD.
    """
    nt = len(tuple_n)
    good = [False] * nt
    rank = [None] * nt
    hits = []
    for t in range(nt):
        n = int(tuple_n[t])
        hits.append([int(h) for h in tuples[t][:n]])
        ndof = max(2 * n - 5, 1)
        r = float(fits[t]["chi2"]) / ndof
        ok = int(fits[t]["status"]) == 0 and np.isfinite(float(fits[t]["chi2"]))
        if ok and pt_min > 0:
            ok = float(fits[t]["pt"]) >= pt_min
        if ok and chi2_max > 0:
            ok = r <= chi2_max
        good[t] = ok
        rank[t] = (-n, r)
    users = {}
    for t in range(nt):
        if good[t]:
            for h in hits[t]:
                users.setdefault(h, []).append(t)
    q = np.zeros(nt, np.uint8)
    for t in range(nt):
        if not good[t]:
            continue
        kept = True
        if clean_shared:
            for h in hits[t]:
                for u in users[h]:
                    if u != t and rank[u] < rank[t]:
                        kept = False
        q[t] = Q_GOOD | (Q_KEPT if kept else 0)
    return q


# -- primary vertices ------------------------------------------------------------------------
def find_vertices(fits, quality, gap, min_tracks):
    """Primary vertices of one event from its fitted tracks (the vertexing step that follows the
    tracks, §2; the paper defines no algorithm, so this is the library's reading).

    Tracks taken: the KEPT ones with a finite dz.  Sorted by dz (equal dz: the track order), a
    track joins the cluster of the one before it when their dz differ by at most `gap` (cm).
    Clusters of at least `min_tracks` tracks are vertices: z the mean dz, z_err the standard
    error of the mean (sqrt(sum (dz - z)^2 / (n (n - 1)))), the track count and the sum of pT^2.
    Vertices are ordered by sum pT^2, largest first (equal sums: smaller z first).
    Returns (vertices: dict of arrays z, z_err, n_tracks, sum_pt2; per-track vertex index, -1
    for tracks in no vertex)."""
    nt = len(quality)
    take = [t for t in range(nt) if (quality[t] & Q_KEPT) and np.isfinite(fits[t]["dz"])]
    take.sort(key=lambda t: (float(fits[t]["dz"]), t))
    clusters = []
    for t in take:
        if clusters and float(fits[t]["dz"]) - float(fits[clusters[-1][-1]]["dz"]) <= gap:
            clusters[-1].append(t)
        else:
            clusters.append([t])
    verts = []
    for c in clusters:
        n = len(c)
        if n < min_tracks:
            continue
        dz = [float(fits[t]["dz"]) for t in c]
        z = sum(dz) / n
        ss = sum((v - z) ** 2 for v in dz)
        err = math.sqrt(ss / (n * (n - 1))) if n > 1 else 0.0
        pt2 = sum(float(fits[t]["pt"]) ** 2 for t in c)
        verts.append((pt2, z, err, n, c))
    verts.sort(key=lambda v: (-v[0], v[1]))
    vid = np.full(nt, -1, np.int32)
    for k, v in enumerate(verts):
        for t in v[4]:
            vid[t] = k
    out = {"z": np.array([v[1] for v in verts]), "z_err": np.array([v[2] for v in verts]),
           "n_tracks": np.array([v[3] for v in verts], np.uint32),
           "sum_pt2": np.array([v[0] for v in verts])}
    return out, vid
