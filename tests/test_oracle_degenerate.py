"""Pins of the oracle at the method's degenerate inputs, each with a result fixed by the
definitions of the doublet, the CA edge and the ntuplet (§2 of the paper states the problem only;
the definitions are the readings the library documents):

* an event with no hits, or with hits on one layer only, has no cells;
* a layer id outside the geometry is rejected;
* every hit given twice multiplies the sets by closed-form factors: a cell joins two hits, so
  each original cell appears 2^2 times, each edge (three hits) 2^3 times and each quadruplet
  2^4 times, and every copy of a quadruplet carries the original's fit;
* exactly straight radial tracks (infinite radius: the DCA's collinear branch) are found,
  including on both sides of the azimuth seam at phi = +-pi, and the fit reports that it found
  no circle.
"""
import numpy as np
import pytest

import oracle
from paper_2104_06573_gb300 import synth


def run(x, y, z, layer, P):
    return oracle.reconstruct(np.asarray(x, np.float32), np.asarray(y, np.float32),
                              np.asarray(z, np.float32), np.asarray(layer, np.uint16), P)


def tuple_set(out):
    return {tuple(int(h) for h in t[:n]) for t, n in zip(out["tuples"], out["tuple_n"])}


def test_empty_and_single_layer_events():
    P = synth.params_barrel_quadruplets()
    e = np.zeros(0, np.float32)
    out = run(e, e, e, np.zeros(0, np.uint16), P)
    assert out["cells"].shape == (0, 2) and out["edges"].shape == (0, 2)
    assert out["tuples"].shape[0] == 0 and len(out["fits"]) == 0
    ev = synth.event_barrel(3, 40)
    on0 = ev.layer == 0
    out = run(ev.x[on0], ev.y[on0], ev.z[on0], ev.layer[on0], P)
    assert len(out["cells"]) == 0 and len(out["tuples"]) == 0


def test_layer_outside_geometry_is_rejected():
    P = synth.params_barrel_quadruplets()
    ev = synth.event_barrel(4, 10)
    bad = ev.layer.copy()
    bad[3] = P.n_layers
    with pytest.raises(ValueError):
        run(ev.x, ev.y, ev.z, bad, P)


def test_duplicated_hits_multiply_the_sets():
    P = synth.params_barrel_quadruplets()
    ev = synth.event_barrel(7, 60)
    base = run(ev.x, ev.y, ev.z, ev.layer, P)
    n = len(ev.x)
    dup = run(*(np.concatenate([a, a]) for a in (ev.x, ev.y, ev.z, ev.layer)), P)
    assert len(base["tuples"]) > 20
    assert len(dup["cells"]) == 4 * len(base["cells"])
    assert len(dup["edges"]) == 8 * len(base["edges"])
    assert len(dup["tuples"]) == 16 * len(base["tuples"])
    # every duplicate quadruplet maps back onto an original one with the original's fit
    fit_of = {tuple(int(h) for h in t[:k]): f
              for t, k, f in zip(base["tuples"], base["tuple_n"], base["fits"])}
    for t, k, f in zip(dup["tuples"], dup["tuple_n"], dup["fits"]):
        g = fit_of[tuple(int(h) % n for h in t[:k])]
        for name in ("pt", "phi", "cot_theta", "dxy", "dz", "chi2"):
            assert f[name] == g[name] or (np.isnan(f[name]) and np.isnan(g[name]))
        assert f["status"] == g["status"] and f["charge"] == g["charge"]


def test_straight_radial_tracks_across_the_seam():
    P = synth.params_barrel_quadruplets()
    xs, ys, zs, ls, want = [], [], [], [], set()
    # phi = +pi (y = +0.0), phi = -pi (y = -0.0) and phi = 0, each a straight radial track
    for y0, x_sign, cot, z0 in [(0.0, -1.0, 0.3, 1.0), (-0.0, -1.0, -0.2, -2.0),
                                (0.0, 1.0, 0.1, 0.5)]:
        hits = []
        for lid, r in enumerate(synth.BARREL_R):
            hits.append(len(xs))
            xs.append(x_sign * r); ys.append(y0); zs.append(z0 + cot * r); ls.append(lid)
        want.add(tuple(hits))
    out = run(xs, ys, zs, ls, P)
    assert tuple_set(out) == want
    # y = +0.0 and y = -0.0 are the same direction: the two seam tracks form cells with each
    # other too: 3 cells per track plus, per layer pair, one cross cell in each direction
    assert len(out["cells"]) == 3 * 3 + 2 * 3
    # collinear hits: no circle; the fit reports status 1 (collinear) instead of a radius
    assert np.all(out["fits"]["status"] == 1)
