"""Pins of the oracle's doublet -> CA -> ntuplet chain by brute force on tiny events, and
invariants on a full dense event.

The brute force does not walk a cell graph.  It enumerates every hit sequence h1..hn whose
consecutive layers form allowed pairs, whose consecutive hits pass the azimuth window (computed
here with atan2) and whose consecutive triples pass the r-z alignment (bend angle from atan2) and
the DCA cut (circle solved as a linear system).  The emitted set is then, by definition, the
sequences starting on a root layer that are maximal (no valid extension) or have max_hits hits,
with at least min_hits hits, minus the strict suffixes of other emitted sequences when that option
is on.  Tiny events keep the enumeration small; every evaluated cut quantity is checked to lie
well away from its threshold so that the two formulations cannot disagree by rounding.
"""
import math

import numpy as np
import pytest

from paper_2104_06573_gb300 import synth


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


class Brute:
    def __init__(self, x, y, z, layer, P):
        self.X = np.asarray(x, np.float64)
        self.Y = np.asarray(y, np.float64)
        self.Z = np.asarray(z, np.float64)
        self.L = np.asarray(layer)
        self.P = P
        self.phi = np.arctan2(self.Y, self.X)
        self.r = np.hypot(self.X, self.Y)
        self.pairs = set(map(tuple, P.pairs))
        self.min_margin = math.inf

    def _margin(self, q, thr):
        self.min_margin = min(self.min_margin, abs(q - thr) / thr)

    def doublet(self, a, b):
        if (int(self.L[a]), int(self.L[b])) not in self.pairs:
            return False
        d = abs(_wrap(self.phi[b] - self.phi[a]))
        self._margin(d, self.P.phi_window)
        return d <= self.P.phi_window

    def triple(self, a, b, c):
        r, z = self.r, self.Z
        a1 = math.atan2(z[b] - z[a], r[b] - r[a])
        a2 = math.atan2(z[c] - z[b], r[c] - r[b])
        s = abs(math.sin(a2 - a1))
        self._margin(s, self.P.theta_cut)
        if s > self.P.theta_cut:
            return False
        px = self.X[[a, b, c]]
        py = self.Y[[a, b, c]]
        A = np.c_[px, py, np.ones(3)]
        if abs(np.linalg.det(A)) < 1e-12:
            # collinear: distance of the origin from the line
            dx, dy = px[2] - px[0], py[2] - py[0]
            dca = abs(px[0] * dy - py[0] * dx) / math.hypot(dx, dy)
        else:
            D, E, F = np.linalg.solve(A, -(px ** 2 + py ** 2))
            c0 = np.array([-D / 2, -E / 2])
            dca = abs(math.hypot(*c0) - math.sqrt(c0 @ c0 - F))
        self._margin(dca, self.P.dca_cut)
        return dca <= self.P.dca_cut

    def cells(self):
        n = len(self.X)
        return {(a, b) for a in range(n) for b in range(n) if self.doublet(a, b)}

    def edges(self):
        cells = self.cells()
        by_in = {}
        for a, b in cells:
            by_in.setdefault(a, []).append(b)
        out = set()
        for a, b in cells:
            for c in by_in.get(b, []):
                if self.triple(a, b, c):
                    out.add((a, b, c))
        return out

    def ntuplets(self):
        n = len(self.X)
        P = self.P

        def ext(seq):
            res = []
            for h in range(n):
                if self.doublet(seq[-1], h) and self.triple(seq[-2], seq[-1], h):
                    res.append(seq + [h])
            return res

        emitted = []
        stack = [[a, b] for a in range(n) for b in range(n)
                 if (P.root_mask >> int(self.L[a])) & 1 and self.doublet(a, b)]
        while stack:
            seq = stack.pop()
            nxt = ext(seq)
            if len(seq) >= P.max_hits or not nxt:
                if len(seq) >= P.min_hits:
                    emitted.append(tuple(seq))
                continue
            stack.extend(nxt)
        em = set(emitted)
        assert len(em) == len(emitted)
        if P.drop_suffixes:
            drop = {q[k:] for q in em for k in range(1, len(q) - 1)}
            em = {t for t in em if t not in drop}
        return em


def _tiny_event(seed, n_tracks, with_disks, n_noise, sector=0.08):
    rng = synth.Rng(seed, 50)
    tr = synth.draw_tracks(rng, n_tracks, "uniform", 0.6, 4.0, 2.2 if with_disks else 1.0)
    tr.phi0 = rng.uniform(n_tracks, 0.0, sector)
    tid, lay, _s, x, y, z = synth.helix_points(tr, with_disks)
    # smear a little so that the CA cuts have something to reject
    x = x + rng.normal(len(x), 5e-3)
    y = y + rng.normal(len(y), 5e-3)
    z = z + rng.normal(len(z), 5e-3)
    if n_noise:
        nl = rng.integers(n_noise, 0, 9 if with_disks else 3)
        ph = rng.uniform(n_noise, -0.05, sector + 0.05)
        rho = np.where(nl < 4, np.array(synth.BARREL_R + (0.0,) * 6)[nl],
                       rng.uniform(n_noise, 5.0, 15.0))
        dz = np.array((0.0,) * 4 + synth.DISK_Z + tuple(-v for v in synth.DISK_Z))
        zz = np.where(nl < 4, rng.uniform(n_noise, -20, 20), dz[nl])
        lay = np.concatenate([lay, nl])
        x = np.concatenate([x, rho * np.cos(ph)])
        y = np.concatenate([y, rho * np.sin(ph)])
        z = np.concatenate([z, zz])
    perm = np.argsort(rng.uniform(len(x)))
    return (x[perm].astype(np.float32), y[perm].astype(np.float32), z[perm].astype(np.float32),
            lay[perm].astype(np.uint16))


CASES = [
    # seed, tracks, disks, noise, loosen cuts
    (1, 6, False, 6, False),
    (2, 8, False, 4, True),
    (3, 5, True, 6, False),
    (4, 7, True, 5, True),
    (5, 9, False, 0, True),
    (6, 6, True, 8, True),
]


@pytest.mark.parametrize("seed,ntr,disks,noise,loose", CASES)
def test_bruteforce_chain_sets(orc, seed, ntr, disks, noise, loose):
    P = synth.params_phase1() if disks else synth.params_barrel_quadruplets()
    if loose:
        P.theta_cut = 0.05
        P.dca_cut = 1.0
    x, y, z, lay = _tiny_event(seed, ntr, disks, noise)
    assert len(x) <= 60
    res = orc.reconstruct(x, y, z, lay, P, stage=3)
    bf = Brute(x, y, z, lay, P)

    cells = {tuple(map(int, c)) for c in res["cells"]}
    assert cells == bf.cells()
    assert len(cells) == len(res["cells"])                      # no duplicates

    cl = res["cells"]
    edges = {(int(cl[a, 0]), int(cl[a, 1]), int(cl[b, 1])) for a, b in res["edges"]}
    assert edges == bf.edges()

    tup = {tuple(int(h) for h in row[:n]) for row, n in zip(res["tuples"], res["tuple_n"])}
    assert len(tup) == len(res["tuples"])
    want = bf.ntuplets()
    assert tup == want
    # the cases must exercise the graph: some ntuplets, some rejected triples
    assert len(want) >= 1
    assert bf.min_margin > 1e-7, bf.min_margin


@pytest.mark.parametrize("seed,min_h,max_h", [(21, 3, 3), (22, 2, 3), (23, 3, 4)])
def test_bruteforce_length_cap(orc, seed, min_h, max_h):
    """A path that reaches max_hits while it could still grow is emitted once, capped."""
    P = synth.params_barrel_quadruplets()
    P.theta_cut, P.dca_cut = 0.05, 1.0
    P.min_hits, P.max_hits = min_h, max_h
    x, y, z, lay = _tiny_event(seed, 7, False, 5)
    res = orc.reconstruct(x, y, z, lay, P, stage=3)
    tup = {tuple(int(h) for h in row[:n]) for row, n in zip(res["tuples"], res["tuple_n"])}
    want = Brute(x, y, z, lay, P).ntuplets()
    assert tup == want
    assert any(len(t) == max_h for t in want)


def test_bruteforce_suffix_rule_is_exercised(orc):
    """With roots on layers 0 and 1, some layer-1 chains are suffixes and must be dropped."""
    P = synth.params_phase1()
    P.theta_cut = 0.05
    P.dca_cut = 1.0
    x, y, z, lay = _tiny_event(11, 8, True, 4)
    P_keep = synth.params_phase1()
    P_keep.theta_cut, P_keep.dca_cut, P_keep.drop_suffixes = 0.05, 1.0, False
    kept = orc.reconstruct(x, y, z, lay, P_keep, stage=3)
    dropped = orc.reconstruct(x, y, z, lay, P, stage=3)
    assert len(kept["tuples"]) > len(dropped["tuples"])
    tup = {tuple(int(h) for h in row[:n]) for row, n in zip(dropped["tuples"],
                                                            dropped["tuple_n"])}
    assert tup == Brute(x, y, z, lay, P).ntuplets()


def test_invariants_dense_event(orc):
    P = synth.params_phase1()
    ev = synth.event_phase1(0)
    res = orc.reconstruct(ev.x, ev.y, ev.z, ev.layer, P, stage=3)
    n = ev.n
    pairs = set(map(tuple, P.pairs))
    cells = res["cells"]
    assert cells.max() < n
    lay = ev.layer.astype(int)
    assert all((lay[a], lay[b]) in pairs for a, b in cells)
    cellset = {tuple(map(int, c)) for c in cells}
    assert len(cellset) == len(cells)
    edges = res["edges"]
    assert np.all(cells[edges[:, 0], 1] == cells[edges[:, 1], 0])   # A.outer == B.inner
    edgeset = {(int(cells[a, 0]), int(cells[a, 1]), int(cells[b, 1])) for a, b in edges}
    tuples = [tuple(int(h) for h in row[:k]) for row, k in zip(res["tuples"], res["tuple_n"])]
    assert len(set(tuples)) == len(tuples)
    for t in tuples:
        assert P.min_hits <= len(t) <= P.max_hits
        assert (P.root_mask >> lay[t[0]]) & 1
        for a, b in zip(t, t[1:]):
            assert (a, b) in cellset                        # consecutive hits form a cell
        for a, b, c in zip(t, t[1:], t[2:]):
            assert (a, b, c) in edgeset                     # consecutive cells share a hit
    ts = set(tuples)
    for t in tuples:
        for k in range(1, len(t) - 1):
            assert t[k:] not in ts                          # no strict suffix survives
    # most generated tracks with >= 3 hits on a chain are found
    assert len(tuples) > 0.8 * 2000
