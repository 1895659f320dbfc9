"""Pins of the oracle's Riemann fit: exact circles and helices (closed form), the circle through
three points, displaced circles (dxy), rotation about the beam line, and the chi2 of smeared
tracks without material."""
import math

import numpy as np

import oracle
from paper_2104_06573_gb300 import synth
from test_oracle_fit import K


def test_exact_helices():
    P = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(3000, seed=5, triplet_frac=0.3, smear=False)
    r = oracle.riemann_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    t = tb.tracks
    assert np.all(r["status"] == 0)
    assert np.all(r["charge"] == t.q)
    assert np.max(np.abs(r["pt"] / t.pt - 1)) < 1e-9
    dphi = (r["phi"] - t.phi0 + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(dphi)) < 1e-9
    assert np.max(np.abs(r["cot_theta"] - t.cot)) < 1e-9
    assert np.max(np.abs(r["dxy"])) < 1e-8
    assert np.max(np.abs(r["dz"] - t.zv)) < 1e-8
    assert np.max(r["chi2"]) < 1e-6


def circle_points(cx, cy, R, angles, z0=0.0, cot=0.0):
    x = cx + R * np.cos(angles)
    y = cy + R * np.sin(angles)
    s = R * (angles - angles[0])
    return x, y, z0 + cot * np.abs(s)


def test_displaced_circle_and_three_points():
    """A circle not through the beam line: dxy = q (|C| - R), pT = K B R; with three hits the
    fitted circle is the one through them."""
    P = synth.params_barrel_quadruplets()
    for cx, cy, R, sense in [(30.0, 40.0, 49.0, 1), (-100.0, 20.0, 101.5, -1), (5.0, -200.0, 199.0, 1)]:
        d = math.hypot(cx, cy)
        a0 = math.atan2(-cy, -cx)               # the point nearest the origin
        ang = a0 + sense * np.array([0.06, 0.12, 0.2, 0.3]) * (50.0 / R)
        x, y, z = circle_points(cx, cy, R, ang, 1.0, 0.5)
        for n in (3, 4):
            r = oracle.riemann_batch(np.array([n], np.uint8), x[None, :n], y[None, :n],
                                     z[None, :n], np.arange(4, dtype=np.uint16)[None, :n], P)[0]
            assert r["status"] == 0
            q = -sense
            assert r["charge"] == q
            assert abs(r["pt"] / (K * P.bfield * R) - 1) < 1e-9
            assert abs(r["dxy"] - q * (d - R)) < 1e-8


def test_rotation_about_the_beam_line():
    P = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(500, seed=8, smear=True)
    a = 0.7
    c, s = math.cos(a), math.sin(a)
    x2, y2 = c * tb.x64 - s * tb.y64, s * tb.x64 + c * tb.y64
    r1 = oracle.riemann_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    r2 = oracle.riemann_batch(tb.n_hits, x2, y2, tb.z64, tb.layer, P)
    for k in ("pt", "cot_theta", "dxy", "dz", "chi2"):
        assert np.allclose(r1[k], r2[k], rtol=1e-7, atol=1e-9), k
    dphi = (r2["phi"] - r1["phi"] - a + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(dphi)) < 1e-9


def test_chi2_of_smeared_tracks():
    """Smeared helices without material: chi2 / (2n - 5) averages ~1 (the plane fit on the
    paraboloid is close to the geometric circle fit at these curvatures)."""
    P = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(4000, seed=6, triplet_frac=0.0, smear=True)
    r = oracle.riemann_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    ok = r["status"] == 0
    m = np.mean(r["chi2"][ok] / 3.0)
    print("chi2/ndf", m)
    assert abs(m - 1.0) < 0.06
