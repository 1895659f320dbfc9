"""Pins of the oracle's three CA cut quantities against geometry it does not use.

The oracle evaluates the doublet window in dot-product form, the r-z alignment as a cross product
over norms and the DCA through a closed-form circle centre.  Here each is checked against an
independent construction: azimuths from atan2, bend angles from atan2 in the r-z plane, and
circles of known centre and radius (or the circle solved as a linear system).  Hand cases with
exact coordinates come from tests/golden/cut_cases.txt.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cut_cases.txt")


def _golden(kind):
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line and line[0] == kind:
                rows.append([float(v) for v in line[1:]])
    return rows


def test_golden_dca(orc):
    rows = _golden("dca")
    assert len(rows) >= 6
    for xi, yi, xj, yj, xk, yk, want in rows:
        got = orc.dca(xi, yi, xj, yj, xk, yk)
        assert abs(got - want) <= 1e-12 * max(1.0, want), (xi, yi, got, want)
        # the DCA is a property of the circle: any order of the three points gives it
        got2 = orc.dca(xk, yk, xi, yi, xj, yj)
        assert abs(got2 - want) <= 1e-12 * max(1.0, want)


def test_golden_theta(orc):
    rows = _golden("theta")
    assert len(rows) >= 6
    for ri, zi, rj, zj, rk, zk, t, want in rows:
        assert orc.theta_pass(ri, zi, rj, zj, rk, zk, t) == bool(want), (rj, zk)


def test_golden_doublet(orc):
    rows = _golden("doublet")
    assert len(rows) >= 5
    for xi, yi, xo, yo, w, want in rows:
        assert orc.doublet_pass(xi, yi, xo, yo, math.cos(w)) == bool(want), (xi, yi, xo, yo)


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


def test_doublet_equals_azimuth_window(orc):
    rng = np.random.default_rng(1)
    w = 0.05
    cw = math.cos(w)
    n_pass = 0
    for _ in range(20000):
        ri, ro = rng.uniform(2, 17, 2)
        pi = rng.uniform(-math.pi, math.pi)
        po = pi + rng.uniform(-0.1, 0.1)
        xi, yi = ri * math.cos(pi), ri * math.sin(pi)
        xo, yo = ro * math.cos(po), ro * math.sin(po)
        d = abs(_wrap(math.atan2(yo, xo) - math.atan2(yi, xi)))
        if abs(d - w) < 1e-9:
            continue
        want = d <= w
        n_pass += want
        assert orc.doublet_pass(xi, yi, xo, yo, cw) == want
        assert orc.doublet_pass(xo, yo, xi, yi, cw) == want          # symmetric in the pair
    assert 5000 < n_pass < 15000


def test_theta_equals_bend_angle(orc):
    rng = np.random.default_rng(2)
    t = 0.002
    n_pass = 0
    for _ in range(20000):
        r = np.sort(rng.uniform(2, 17, 3))
        z0 = rng.uniform(-20, 20)
        slope = rng.uniform(-3, 3)
        zs = z0 + slope * (r - r[0])
        # bend the outer segment by a small angle of either sign
        bend = rng.uniform(-0.004, 0.004)
        a1 = math.atan2(zs[1] - zs[0], r[1] - r[0])
        L = math.hypot(r[2] - r[1], zs[2] - zs[1])
        rk, zk = r[1] + L * math.cos(a1 + bend), zs[1] + L * math.sin(a1 + bend)
        a_ang = math.atan2(zs[1] - zs[0], r[1] - r[0])
        b_ang = math.atan2(zk - zs[1], rk - r[1])
        s = abs(math.sin(b_ang - a_ang))
        if abs(s - t) < 1e-9:
            continue
        want = s <= t
        n_pass += want
        assert orc.theta_pass(r[0], zs[0], r[1], zs[1], rk, zk, t) == want
    assert 5000 < n_pass < 15000


def test_dca_known_circles(orc):
    rng = np.random.default_rng(3)
    for _ in range(5000):
        R = math.exp(rng.uniform(math.log(5), math.log(5e4)))
        ang = rng.uniform(-math.pi, math.pi)
        dist = R + rng.uniform(-0.5, 0.5)           # |c| - R in [-0.5, 0.5]
        cx, cy = dist * math.cos(ang), dist * math.sin(ang)
        # three points on the circle near the origin side, spread like pixel layers
        base = ang + math.pi
        spread = min(1.0, 16.0 / R)
        th = base + np.sort(rng.uniform(-spread, spread, 3))
        p = [(cx + R * math.cos(a), cy + R * math.sin(a)) for a in th]
        want = abs(math.hypot(cx, cy) - R)
        got = orc.dca(*p[0], *p[1], *p[2])
        # the construction itself rounds the points at the 1e-16 * R level; the DCA of a circle
        # of radius R moves by about that much
        tol = 1e-9 * max(1.0, R / 100.0) + 1e-12
        assert abs(got - want) <= tol, (R, got, want)


def test_dca_against_linear_circle_solve(orc):
    """Circle through three points from x^2+y^2+Dx+Ey+F=0 solved as a linear system."""
    rng = np.random.default_rng(4)
    for _ in range(5000):
        pts = rng.uniform(-16, 16, (3, 2))
        A = np.c_[pts, np.ones(3)]
        rhs = -(pts ** 2).sum(1)
        if abs(np.linalg.det(A)) < 1e-3:
            continue
        D, E, F = np.linalg.solve(A, rhs)
        c = np.array([-D / 2, -E / 2])
        R = math.sqrt(c @ c - F)
        want = abs(math.hypot(*c) - R)
        got = orc.dca(*pts[0], *pts[1], *pts[2])
        assert abs(got - want) <= 1e-9 * max(1.0, R), (got, want)


def test_dca_invariances(orc):
    rng = np.random.default_rng(5)
    for _ in range(2000):
        pts = rng.uniform(-16, 16, (3, 2))
        d0 = orc.dca(*pts[0], *pts[1], *pts[2])
        a = rng.uniform(-math.pi, math.pi)
        Rm = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        q = pts @ Rm.T
        assert orc.dca(*q[0], *q[1], *q[2]) == pytest.approx(d0, rel=1e-8, abs=1e-9)
        m = pts * np.array([1.0, -1.0])                  # mirror
        assert orc.dca(*m[0], *m[1], *m[2]) == pytest.approx(d0, rel=1e-8, abs=1e-9)


def test_dca_collinear_branch(orc):
    rng = np.random.default_rng(6)
    for _ in range(2000):
        # exactly collinear points on an axis-parallel line y = c (exact products)
        c = float(rng.integers(-64, 64)) / 8.0
        xs = np.sort(rng.integers(-128, 128, 3).astype(float) / 8.0)
        if len(set(xs)) < 3:
            continue
        got = orc.dca(xs[0], c, xs[1], c, xs[2], c)
        assert got == abs(c)
