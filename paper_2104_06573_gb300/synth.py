"""Seeded synthetic pixel-hit events: the one input module shared by the oracle and the CUDA path.

The paper measures on simulated top-quark-pair events with about 50 pileup collisions, read as raw
pixel data (paper, §2, workload paragraph).  That data set is not available here, so every workload
is synthetic: charged tracks from the beam line follow helices in a 3.8 T solenoid and leave one hit
where they cross a detector layer.  The shapes are those of the five workloads of this project:

  * barrel-only events of 100 tracks, noise-free (the small parity event),
  * dense Phase-1-like events of 2000 tracks with forward disks, hit smearing and 20 % noise hits,
  * batches of 256 barrel events with 200..6000 tracks each,
  * a million smeared barrel ntuplets for the fit precision study,
  * a stream of events with log-normal track counts and Poisson arrival times.

This module draws random numbers and places hits on helices.  It contains none of the method's
arithmetic (no cut, no graph step, no fit).  Random numbers come from SplitMix64 (G. Steele, D. Lea,
C. Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value i of stream (seed, stream_id) is mix(state0 + (i + 1) * golden).

Units: cm, GeV, T, rad.  Layer ids: barrel 0..3, +z disks 4..6, -z disks 7..9.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64)
# ----------------------------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Sequential reader of one SplitMix64 stream, identified by (seed, stream_id)."""

    def __init__(self, seed: int, stream_id: int = 0):
        with np.errstate(over="ignore"):
            s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
            t = np.array([stream_id & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
            self._state0 = _mix64(s * _GOLDEN + t * _STREAM_MUL + _GOLDEN)[0]
        self._next = 0

    def raw(self, n: int) -> np.ndarray:
        i = np.arange(self._next + 1, self._next + 1 + n, dtype=np.uint64)
        self._next += n
        with np.errstate(over="ignore"):
            return _mix64(self._state0 + i * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.raw(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        # Box-Muller transform on two uniforms; 1 - u lies in (0, 1] so the log is finite.
        u1 = 1.0 - self.uniform(n)
        u2 = self.uniform(n)
        return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)


# ----------------------------------------------------------------------------------------------
# Detector and cut configuration (inputs shared by both sides)
# ----------------------------------------------------------------------------------------------
K_PT = 0.299792458e-2          # pT [GeV] = K_PT * B [T] * R [cm]
BFIELD = 3.8
BARREL_R = (2.9, 6.8, 10.9, 16.0)
BARREL_HALF_Z = 26.7
DISK_Z = (29.1, 39.6, 51.6)
DISK_RMIN, DISK_RMAX = 4.5, 16.0
MAX_LAYERS = 16


def layer_tables(with_disks: bool):
    """(n_layers, position, is_disk): barrel radius or signed disk z per layer id."""
    pos = list(BARREL_R)
    is_disk = [0, 0, 0, 0]
    if with_disks:
        pos += list(DISK_Z) + [-z for z in DISK_Z]
        is_disk += [1] * 6
    return len(pos), pos, is_disk


PAIRS_BARREL = ((0, 1), (1, 2), (2, 3))
PAIRS_PHASE1 = ((0, 1), (1, 2), (2, 3),
                (0, 4), (1, 4), (2, 4), (0, 7), (1, 7), (2, 7),
                (4, 5), (5, 6), (7, 8), (8, 9))


@dataclass
class Params:
    """Geometry, layer pairs, cuts and fit constants of one workload (plain data)."""
    n_layers: int
    layer_pos: list
    layer_is_disk: list
    pairs: tuple
    root_layers: tuple
    drop_suffixes: bool
    min_hits: int
    max_hits: int
    phi_window: float = 0.05
    theta_cut: float = 0.002
    dca_cut: float = 0.15
    bfield: float = BFIELD
    sigma_rphi: float = 10e-4
    sigma_z: float = 20e-4
    x_over_x0: float = 0.02
    cos_phi_window: float = field(init=False)

    def __post_init__(self):
        # cos(w) is computed once here and handed to both implementations as an input.
        self.cos_phi_window = math.cos(self.phi_window)

    @property
    def root_mask(self) -> int:
        m = 0
        for layer in self.root_layers:
            m |= 1 << layer
        return m


def params_barrel_quadruplets() -> Params:
    """Barrel-only workload: quadruplets only, roots on layer 0."""
    n, pos, disk = layer_tables(False)
    return Params(n, pos, disk, PAIRS_BARREL, (0,), False, 4, 4)


def params_phase1() -> Params:
    """Barrel + disks workload: triplets and quadruplets (up to 5 hits), roots on layers 0 and 1
    with suffix removal."""
    n, pos, disk = layer_tables(True)
    return Params(n, pos, disk, PAIRS_PHASE1, (0, 1), True, 3, 5)


# ----------------------------------------------------------------------------------------------
# Helix placement
# ----------------------------------------------------------------------------------------------
@dataclass
class Tracks:
    pt: np.ndarray
    phi0: np.ndarray
    cot: np.ndarray
    q: np.ndarray
    zv: np.ndarray

    def __len__(self):
        return len(self.pt)


@dataclass
class Event:
    x: np.ndarray          # float32 [n]
    y: np.ndarray
    z: np.ndarray
    layer: np.ndarray      # uint16 [n]
    track: np.ndarray      # int32 [n], -1 for noise hits
    x64: np.ndarray        # float64 positions before rounding to float32 (for closed-form checks)
    y64: np.ndarray
    z64: np.ndarray
    tracks: Tracks

    @property
    def n(self) -> int:
        return len(self.x)


def radius_of(pt):
    return np.asarray(pt, dtype=np.float64) / (K_PT * BFIELD)


def draw_tracks(rng: Rng, n: int, pt_mode: str, pt_lo: float, pt_hi: float, eta_max: float,
                zv_sigma: float = 5.0) -> Tracks:
    if pt_mode == "uniform":
        pt = rng.uniform(n, pt_lo, pt_hi)
    elif pt_mode == "power3":          # density proportional to pT^-3 above pt_lo
        pt = pt_lo / np.sqrt(1.0 - rng.uniform(n))
    elif pt_mode == "loguniform":
        pt = np.exp(rng.uniform(n, math.log(pt_lo), math.log(pt_hi)))
    else:
        raise ValueError(pt_mode)
    eta = rng.uniform(n, -eta_max, eta_max)
    phi0 = rng.uniform(n, -math.pi, math.pi)
    q = np.where(rng.uniform(n) < 0.5, 1, -1).astype(np.int32)
    zv = rng.normal(n, zv_sigma)
    return Tracks(pt, phi0, np.sinh(eta), q, zv)


def helix_points(tr: Tracks, with_disks: bool):
    """Crossings of each helix (from (0, 0, zv)) with every layer.

    A track of transverse radius R = pT / (K_PT B) and charge q starting along phi0 has, after a
    transverse path s, the position 2R sin(s / 2R) (cos a, sin a) with a = phi0 - q s / (2R), and
    z = zv + s cot(theta).  Returns flat arrays (track, layer, s, x, y, z) in FP64.
    """
    R = radius_of(tr.pt)
    out = []
    idx = np.arange(len(tr))
    for lid, rho in enumerate(BARREL_R):
        ok = rho < 2.0 * R
        half = np.arcsin(np.minimum(rho / (2.0 * R), 1.0))
        s = 2.0 * R * half
        z = tr.zv + s * tr.cot
        ok &= np.abs(z) < BARREL_HALF_Z
        a = tr.phi0 - tr.q * half
        out.append((idx[ok], np.full(ok.sum(), lid), s[ok], rho * np.cos(a[ok]),
                    rho * np.sin(a[ok]), z[ok]))
    if with_disks:
        for side, base in ((1.0, 4), (-1.0, 7)):
            for k, zd in enumerate(DISK_Z):
                zd = side * zd
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = (zd - tr.zv) / tr.cot
                ok = np.isfinite(s) & (s > 0) & (s < math.pi * R)
                s = np.where(ok, s, 0.0)
                rho = 2.0 * R * np.sin(s / (2.0 * R))
                ok &= (rho >= DISK_RMIN) & (rho <= DISK_RMAX)
                a = tr.phi0 - tr.q * s / (2.0 * R)
                out.append((idx[ok], np.full(ok.sum(), base + k), s[ok], rho[ok] * np.cos(a[ok]),
                            rho[ok] * np.sin(a[ok]), np.full(ok.sum(), zd)))
    cols = [np.concatenate([o[c] for o in out]) for c in range(6)]
    order = np.lexsort((cols[2], cols[0]))          # by track, then path length
    return tuple(c[order] for c in cols)


def _smear(rng: Rng, layer, x, y, z, with_disks, sigma_rphi, sigma_z):
    n = len(x)
    phi = np.arctan2(y, x)
    d_rphi = rng.normal(n, sigma_rphi)
    d_other = rng.normal(n, sigma_z)
    disk = layer >= 4
    ur_x, ur_y = np.cos(phi), np.sin(phi)
    x = x - ur_y * d_rphi + np.where(disk, ur_x * d_other, 0.0)
    y = y + ur_x * d_rphi + np.where(disk, ur_y * d_other, 0.0)
    z = z + np.where(disk, 0.0, d_other)
    return x, y, z


def _noise(rng: Rng, layer_counts, n_noise):
    p = layer_counts / max(1, layer_counts.sum())
    cdf = np.cumsum(p)
    lay = np.minimum(np.searchsorted(cdf, rng.uniform(n_noise), side="right"), len(p) - 1)
    phi = rng.uniform(n_noise, -math.pi, math.pi)
    zb = rng.uniform(n_noise, -BARREL_HALF_Z, BARREL_HALF_Z)
    rd = np.sqrt(rng.uniform(n_noise, DISK_RMIN ** 2, DISK_RMAX ** 2))
    rho = np.where(lay < 4, np.array(BARREL_R + (0.0,) * 6)[lay], rd)
    disk_z = np.array((0.0,) * 4 + DISK_Z + tuple(-z for z in DISK_Z))
    z = np.where(lay < 4, zb, disk_z[lay])
    return lay, rho * np.cos(phi), rho * np.sin(phi), z


def make_event(seed: int, n_tracks: int, *, with_disks=False, pt_mode="uniform", pt_lo=1.0,
               pt_hi=10.0, eta_max=1.0, smear=False, noise_frac=0.0, shuffle=True,
               n_vertices: int = 0) -> Event:
    """n_vertices > 0: the tracks come from that many primary vertices (z ~ N(0, 5 cm)), each
    track from a uniformly drawn one; otherwise every track has its own origin z ~ N(0, 5 cm)."""
    rng = Rng(seed, 1)
    tr = draw_tracks(rng, n_tracks, pt_mode, pt_lo, pt_hi, eta_max)
    if n_vertices > 0:
        vr = Rng(seed, 5)
        vz = vr.normal(n_vertices, 5.0)
        owner = np.minimum((vr.uniform(n_tracks) * n_vertices).astype(np.int64), n_vertices - 1)
        tr = Tracks(tr.pt, tr.phi0, tr.cot, tr.q, vz[owner])
    tid, lay, _s, x, y, z = helix_points(tr, with_disks)
    if smear:
        x, y, z = _smear(Rng(seed, 2), lay, x, y, z, with_disks, 10e-4, 20e-4)
    tid = tid.astype(np.int32)
    if noise_frac > 0:
        counts = np.bincount(lay, minlength=10 if with_disks else 4).astype(np.float64)
        n_noise = int(round(noise_frac * len(x)))
        nl, nx, ny, nz = _noise(Rng(seed, 3), counts, n_noise)
        lay = np.concatenate([lay, nl])
        x, y, z = np.concatenate([x, nx]), np.concatenate([y, ny]), np.concatenate([z, nz])
        tid = np.concatenate([tid, np.full(n_noise, -1, np.int32)])
    if shuffle:
        perm = np.argsort(Rng(seed, 4).uniform(len(x)), kind="stable")
        lay, x, y, z, tid = lay[perm], x[perm], y[perm], z[perm], tid[perm]
    return Event(x.astype(np.float32), y.astype(np.float32), z.astype(np.float32),
                 lay.astype(np.uint16), tid, x, y, z, tr)


def event_barrel(seed: int = 0, n_tracks: int = 100) -> Event:
    """Barrel-only event: pT uniform 1-10 GeV, |eta| < 1, no smearing or noise."""
    return make_event(seed, n_tracks)


def event_phase1(seed: int = 0, n_tracks: int = 2000) -> Event:
    """Dense event with disks: pT ~ pT^-3 above 0.5 GeV, |eta| < 2.5, smearing, 20 % noise."""
    return make_event(seed, n_tracks, with_disks=True, pt_mode="power3", pt_lo=0.5, pt_hi=0.0,
                      eta_max=2.5, smear=True, noise_frac=0.2)


def batch_track_counts(n_events: int = 256, seed0: int = 0, lo: int = 200, hi: int = 6000):
    return [int(Rng(seed0 + e, 0).integers(1, lo, hi)[0]) for e in range(n_events)]


def batch_barrel(n_events: int = 256, seed0: int = 0, lo: int = 200, hi: int = 6000):
    """Batch of barrel events with per-event track count uniform in [lo, hi]."""
    counts = batch_track_counts(n_events, seed0, lo, hi)
    return [make_event(seed0 + e, counts[e]) for e in range(n_events)]


@dataclass
class TupletBatch:
    """Ntuplets for the fit study: hits (FP32 and FP64) per ntuplet, padded to 4."""
    n_hits: np.ndarray       # uint8 [m]
    x: np.ndarray            # float32 [m, 4]
    y: np.ndarray
    z: np.ndarray
    layer: np.ndarray        # uint16 [m, 4]
    x64: np.ndarray
    y64: np.ndarray
    z64: np.ndarray
    tracks: Tracks


def fit_tuplets(n: int = 1_000_000, seed: int = 0, triplet_frac: float = 0.3,
                smear: bool = True) -> TupletBatch:
    """Smeared barrel ntuplets, pT log-uniform 0.5-100 GeV; 30 % become triplets by dropping the
    outermost hit.  Only tracks with all four barrel hits are kept."""
    rng = Rng(seed, 11)
    m = int(n * 1.3) + 64
    tr = draw_tracks(rng, m, "loguniform", 0.5, 100.0, 1.0)
    tid, lay, _s, x, y, z = helix_points(tr, False)
    if smear:
        x, y, z = _smear(Rng(seed, 12), lay, x, y, z, False, 10e-4, 20e-4)
    cnt = np.bincount(tid, minlength=m)
    full = np.nonzero(cnt == 4)[0][:n]
    if len(full) < n:
        raise RuntimeError("not enough four-hit tracks drawn")
    start = np.concatenate([[0], np.cumsum(cnt)])[full]
    sel = start[:, None] + np.arange(4)[None, :]
    nh = np.where(Rng(seed, 13).uniform(n) < triplet_frac, 3, 4).astype(np.uint8)
    t = Tracks(tr.pt[full], tr.phi0[full], tr.cot[full], tr.q[full], tr.zv[full])
    return TupletBatch(nh, x[sel].astype(np.float32), y[sel].astype(np.float32),
                       z[sel].astype(np.float32), lay[sel].astype(np.uint16), x[sel], y[sel],
                       z[sel], t)


def serving_stream(rate_hz: float, n_events: int, seed: int = 0, median: float = 1500.0,
                   sigma: float = 0.8, cap: int = 8000):
    """Poisson arrivals (seconds from start) and log-normal track counts, capped."""
    rng = Rng(seed, 21)
    gaps = -np.log(1.0 - rng.uniform(n_events)) / rate_hz
    t = np.cumsum(gaps)
    counts = np.minimum(np.round(median * np.exp(rng.normal(n_events, sigma))), cap)
    counts = np.maximum(counts, 1).astype(np.int64)
    return t, counts


def event_serving(seed: int, n_tracks: int) -> Event:
    """Barrel geometry with hit smearing (no noise): the events of the serving stream."""
    return make_event(seed, n_tracks, smear=True)
