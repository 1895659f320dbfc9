"""Pins of the oracle's broken-line fit against results fixed by geometry and linear algebra.

1. Closed form: hits exactly on a helix from (0, 0, zv) give back the generated pT, phi, cot(theta),
   dz = zv and dxy = 0 to 1e-9 (the reference circle is then the true circle, all offsets vanish).
2. Transverse displacement: the same helices moved by (dx, dy); dxy, phi and dz at the point of
   closest approach are computed here from the known circle.
3. Three smeared hits: the fit must return the circle through the three points, solved here as a
   linear system (the curvature correction and offsets must cancel exactly).
4. Stiff limit: with negligible multiple scattering the broken line is a rigid circle + straight
   line least-squares fit; compared with a geometric nonlinear least-squares fit (scipy).
5. Linear algebra: the normal-equation Cholesky solve equals numpy's lstsq of the stacked,
   weighted design matrix built from the definition of the residuals and kinks.
6. Symmetries: rotation, mirror and z-reflection act on the parameters as geometry says.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2104_06573_gb300 import synth

K = 0.299792458e-2


def _tracks(seed, n, pt_mode="loguniform", lo=0.5, hi=100.0, eta=2.5):
    rng = synth.Rng(seed, 99)
    return synth.draw_tracks(rng, n, pt_mode, lo, hi, eta)


def _per_track_hits(tr, with_disks):
    tid, lay, s, x, y, z = synth.helix_points(tr, with_disks)
    out = {}
    for t in np.unique(tid):
        m = tid == t
        out[int(t)] = (lay[m], x[m], y[m], z[m])
    return out


def _subsets(n):
    """index subsets of a track's hits: all, and inner 3 / 4."""
    subs = [list(range(n))]
    if n >= 4:
        subs.append([0, 1, 2])
        subs.append([0, 1, n - 1])
    if n >= 5:
        subs.append([0, 1, 2, 3])
    return subs


@pytest.mark.parametrize("with_disks", [False, True])
def test_closed_form_helix(orc, with_disks):
    p = synth.params_phase1() if with_disks else synth.params_barrel_quadruplets()
    tr = _tracks(7 if with_disks else 8, 3000)
    hits = _per_track_hits(tr, with_disks)
    n_checked = 0
    worst = np.zeros(5)
    for t, (lay, x, y, z) in hits.items():
        if len(x) < 3:
            continue
        for sub in _subsets(len(x)):
            f = orc.fit_one(x[sub], y[sub], z[sub], lay[sub], p)
            assert f["status"] == 0
            assert f["charge"] == tr.q[t]
            err = np.array([abs(f["pt"] / tr.pt[t] - 1),
                            abs(_wrap(f["phi"] - tr.phi0[t])),
                            abs(f["cot_theta"] - tr.cot[t]) / max(1.0, abs(tr.cot[t])),
                            abs(f["dz"] - tr.zv[t]) / max(1.0, abs(tr.zv[t])),
                            abs(f["dxy"])])
            worst = np.maximum(worst, err)
            assert f["chi2"] < 1e-6
            n_checked += 1
    assert n_checked > 2000
    assert np.all(worst < 1e-9), worst


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


def test_transverse_displacement(orc):
    """Helices from a displaced vertex: dxy, phi and dz at the point of closest approach."""
    p = synth.params_barrel_quadruplets()
    tr = _tracks(9, 2000, "uniform", 1.0, 100.0, 1.0)
    hits = _per_track_hits(tr, False)
    rng = np.random.default_rng(9)
    n = 0
    for t, (lay, x, y, z) in hits.items():
        if len(x) < 4:
            continue
        dx, dy = rng.uniform(-0.3, 0.3, 2)
        q = tr.q[t]
        R = tr.pt[t] / (K * synth.BFIELD)
        # true centre: to the right of the direction of motion for q > 0
        c = np.array([q * R * math.sin(tr.phi0[t]) + dx, -q * R * math.cos(tr.phi0[t]) + dy])
        dist = math.hypot(*c)
        dxy_true = q * (dist - R)
        e = -c / dist                                   # centre -> origin
        tang = np.array([e[1], -e[0]]) if q > 0 else np.array([-e[1], e[0]])
        phi_true = math.atan2(tang[1], tang[0])
        nv = (np.array([dx, dy]) - c) / R               # radial direction at the vertex
        orient = -q                                     # +1 counter-clockwise
        psi = math.atan2(orient * (nv[0] * e[1] - nv[1] * e[0]), nv @ e)
        dz_true = tr.zv[t] + tr.cot[t] * (R * psi)
        f = orc.fit_one(x + dx, y + dy, z, lay, p)
        assert f["status"] == 0
        assert abs(f["dxy"] - dxy_true) < 1e-9, (f["dxy"], dxy_true)
        assert abs(_wrap(f["phi"] - phi_true)) < 1e-9
        assert abs(f["dz"] - dz_true) < 1e-9
        assert abs(f["pt"] / tr.pt[t] - 1) < 1e-9
        n += 1
    assert n > 1000


def _circle3(px, py):
    A = np.c_[px, py, np.ones(3)]
    D, E, F = np.linalg.solve(A, -(px ** 2 + py ** 2))
    c = np.array([-D / 2, -E / 2])
    return c, math.sqrt(c @ c - F)


def test_three_hits_give_the_circle_through_them(orc):
    p = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(4000, seed=3)
    for t in range(4000):
        X, Y, Z, L = tb.x64[t, :3], tb.y64[t, :3], tb.z64[t, :3], tb.layer[t, :3]
        f = orc.fit_one(X, Y, Z, L, p)
        assert f["status"] == 0
        c, R = _circle3(X, Y)
        assert abs(f["pt"] / (K * synth.BFIELD * R) - 1) < 1e-7
        dist = math.hypot(*c)
        assert abs(f["dxy"] - f["charge"] * (dist - R)) < 1e-7 * max(1.0, R / 100)


def _geometric_fit(X, Y, Z):
    """Least-squares circle (geometric distances) + straight line in (s, z), and the track
    parameters at the point of closest approach, all computed here.

    The circle is parameterised by an offset u0 of hit 0 along the left normal of the chord, a
    rotation a of the chord direction and a signed curvature k (> 0 counter-clockwise); the distance
    of a point from it is written as F / (|k w - m| + 1) with F = k |w|^2 - 2 w.m, which stays well
    conditioned as k -> 0."""
    from scipy.optimize import least_squares
    x, y = X - X[0], Y - Y[0]
    ch = np.array([x[-1], y[-1]])
    t = ch / np.hypot(*ch)
    nu = np.array([-t[1], t[0]])
    c0, R0 = _circle3(x[[0, len(x) // 2, -1]], y[[0, len(x) // 2, -1]])
    k0 = (1.0 / R0) * (1.0 if c0 @ nu > 0 else -1.0)

    def frame(v):
        u0, a, k = v
        d = t * math.cos(a) + nu * math.sin(a)
        m = np.array([-d[1], d[0]])
        return u0 * nu, d, m, k

    def res(v):
        P0, d, m, k = frame(v)
        wx, wy = x - P0[0], y - P0[1]
        F = k * (wx * wx + wy * wy) - 2 * (wx * m[0] + wy * m[1])
        return F / (np.hypot(k * wx - m[0], k * wy - m[1]) + 1.0)

    sol = least_squares(res, [0.0, 0.0, k0], x_scale=[1e-3, 1e-3, abs(k0)], xtol=1e-15,
                        ftol=1e-15, gtol=1e-15)
    P0, d, m, k = frame(sol.x)
    c = P0 + m / k
    R = 1.0 / abs(k)
    orient = 1.0 if k > 0 else -1.0
    # path length along the fitted circle from hit 0's projection, in the direction of motion
    a0 = np.array([x[0], y[0]]) - c
    s = R * np.array([math.atan2(orient * (a0[0] * (y[i] - c[1]) - a0[1] * (x[i] - c[0])),
                                 a0 @ np.array([x[i] - c[0], y[i] - c[1]]))
                      for i in range(len(x))])
    (z0, cot), *_ = np.linalg.lstsq(np.c_[np.ones_like(s), s], Z, rcond=None)
    w = np.array([-X[0], -Y[0]]) - c                   # centre -> transverse origin
    dist = math.hypot(*w)
    e = w / dist
    tang = orient * np.array([-e[1], e[0]])
    r0 = a0 / math.hypot(*a0)
    psi = math.atan2(orient * (e[0] * r0[1] - e[1] * r0[0]), e @ r0)
    return dict(k=k, k_ref=k0, cot=cot, dxy=-orient * (dist - R),
                phi=math.atan2(tang[1], tang[0]), dz=z0 - cot * R * psi)


def test_stiff_limit_matches_geometric_fit(orc):
    """Negligible multiple scattering: the broken line is a rigid circle + line fit.  Its curvature
    must match the geometric fit to a small fraction of the correction it applies to the
    three-point reference circle (a wrong sign or factor in the curvature term moves it by the
    whole correction), plus the first-order term kappa0^2 u that the linearisation drops.  dxy,
    phi and dz agree to well below the effect of the offset u0 (~1e-3 cm) or of the curvature
    term in the starting direction (~1e-4 rad)."""
    p = synth.params_barrel_quadruplets()
    p.x_over_x0 = 1e-6
    tb = synth.fit_tuplets(600, seed=4)
    n_big = 0
    for t in range(600):
        X, Y, Z, L = tb.x64[t], tb.y64[t], tb.z64[t], tb.layer[t]
        f = orc.fit_one(X, Y, Z, L, p)
        assert f["status"] == 0
        if f["pt"] > 1000.0:
            # smearing made the track straight; kink weights of ~1e20 leave the normal
            # equations too ill-conditioned for a 1e-6 comparison
            continue
        k_bl = -f["charge"] * K * synth.BFIELD / f["pt"]          # signed, > 0 counter-clockwise
        g = _geometric_fit(X, Y, Z)
        corr = abs(g["k"] - g["k_ref"])
        assert abs(k_bl - g["k"]) <= 0.03 * corr + 5e-5 * abs(g["k"]), (t, k_bl, g)
        n_big += corr > 0.01 * abs(g["k"])
        assert abs(f["dxy"] - g["dxy"]) < 2e-5
        assert abs(_wrap(f["phi"] - g["phi"])) < 1e-5
        assert abs(f["dz"] - g["dz"]) < 1e-4
        # line: straight-line least squares of z against the path length along the three-point
        # reference circle (computed here), which is the abscissa the broken line uses
        nh = len(X)
        x, y = X - X[0], Y - Y[0]
        c, R = _circle3(x[[0, nh // 2, -1]], y[[0, nh // 2, -1]])
        orient = 1.0 if g["k_ref"] > 0 else -1.0
        a0 = -c
        s = np.array([R * math.atan2(orient * (a0[0] * (y[i] - c[1]) - a0[1] * (x[i] - c[0])),
                                     a0 @ np.array([x[i] - c[0], y[i] - c[1]]))
                      for i in range(nh)])
        (_z0, cot_ref), *_ = np.linalg.lstsq(np.c_[np.ones(nh), s], Z, rcond=None)
        assert abs(f["cot_theta"] - cot_ref) < 1e-5 * max(1.0, abs(cot_ref))
        assert abs(f["cot_theta"] - g["cot"]) < 1e-4 * max(1.0, abs(g["cot"]))
    assert n_big > 100            # the correction is exercised, not just the reference circle


def test_chi2_matches_smearing_with_disks(orc):
    """Stiff limit on smeared forward tracks (barrel + disk hits): with weights that match the
    generated errors (10 um in r-phi; 20 um in z on barrel layers and in r on disks, i.e.
    20 um * |cot| in z at fixed path length) the minimum chi2 follows chi2(2n - 5)."""
    P = synth.params_phase1()
    P.x_over_x0 = 1e-6
    rng = synth.Rng(21, 5)
    tr = synth.draw_tracks(rng, 6000, "uniform", 1.0, 10.0, 2.4)
    keep = np.abs(tr.cot) > math.sinh(1.6)
    tr = synth.Tracks(tr.pt[keep], tr.phi0[keep], tr.cot[keep], tr.q[keep], tr.zv[keep])
    tid, lay, _s, x, y, z = synth.helix_points(tr, True)
    ev_x, ev_y, ev_z = synth._smear(synth.Rng(21, 6), lay, x, y, z, True, 10e-4, 20e-4)
    chi, ndf, n_disk = 0.0, 0, 0
    for t in np.unique(tid):
        m = np.nonzero(tid == t)[0]
        if len(m) < 4:
            continue
        m = m[:5]
        f = orc.fit_one(ev_x[m], ev_y[m], ev_z[m], lay[m], P)
        if f["status"] != 0 or f["pt"] > 1000:
            continue
        chi += f["chi2"]
        ndf += 2 * len(m) - 5
        n_disk += int(np.sum(lay[m] >= 4))
    assert n_disk > 2000 and ndf > 3000
    print("chi2/ndf", chi / ndf)
    assert abs(chi / ndf - 1.0) < 0.08, chi / ndf


def _propagate_to_radius(P, d, q, R, rho):
    """Exact helix from point P (3D) with unit direction d to the cylinder of radius rho."""
    dT = math.hypot(d[0], d[1])
    phi_d = math.atan2(d[1], d[0])
    cot = d[2] / dT
    c = np.array([P[0] + q * R * math.sin(phi_d), P[1] - q * R * math.cos(phi_d)])
    rel = np.array([P[0], P[1]]) - c

    def pos(s):
        a = -q * s / R
        ca, sa = math.cos(a), math.sin(a)
        return c + np.array([ca * rel[0] - sa * rel[1], sa * rel[0] + ca * rel[1]])

    lo, hi = 0.0, None
    steps = np.linspace(0, math.pi * R, 2000)[1:]
    for s in steps:
        if math.hypot(*pos(s)) >= rho:
            hi = s
            break
        lo = s
    if hi is None:
        return None
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if math.hypot(*pos(mid)) >= rho:
            hi = mid
        else:
            lo = mid
    s = 0.5 * (lo + hi)
    xy = pos(s)
    a = phi_d - q * s / R
    dn = np.array([math.cos(a) * dT, math.sin(a) * dT, d[2]])
    return np.array([xy[0], xy[1], P[2] + s * cot]), dn / np.linalg.norm(dn)


def test_chi2_matches_multiple_scattering(orc):
    """Barrel tracks simulated with 3D scattering: at each layer the direction is turned by two
    independent Gaussian angles of width theta0 (Highland, path length through the layer from the
    exact incidence angle) perpendicular to it.  The fit's projected kink variances must then give
    chi2 following chi2(2n - 5)."""
    P = synth.params_barrel_quadruplets()
    rng = np.random.default_rng(33)
    chi, ndf, n = 0.0, 0, 0
    while n < 1500:
        pt = rng.uniform(0.6, 2.0)
        # forward-ish tracks: the projections 1 + cot^2 of the kink variances are ~2 here, so a
        # missing projection factor shows in the chi2
        eta = rng.uniform(0.7, 1.1) * (1 if rng.uniform() < 0.5 else -1)
        phi0 = rng.uniform(-math.pi, math.pi)
        q = 1 if rng.uniform() < 0.5 else -1
        R = pt / (K * synth.BFIELD)
        p = pt * math.cosh(eta)
        d = np.array([math.cos(phi0) / math.cosh(eta), math.sin(phi0) / math.cosh(eta),
                      math.tanh(eta)])
        Pt = np.array([0.0, 0.0, rng.normal(0, 5.0)])
        hits = []
        for li, rho in enumerate(synth.BARREL_R):
            res = _propagate_to_radius(Pt, d, q, R, rho)
            if res is None:
                break
            Pt, d = res
            hits.append(Pt.copy())
            nrm = np.array([Pt[0], Pt[1], 0.0]) / rho
            xx = P.x_over_x0 / abs(d @ nrm)
            th0 = 0.0136 / p * math.sqrt(xx) * (1 + 0.038 * math.log(xx))
            e1 = np.cross(d, [0.0, 0.0, 1.0])
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(d, e1)
            d = d + rng.normal(0, th0) * e1 + rng.normal(0, th0) * e2
            d /= np.linalg.norm(d)
        if len(hits) < 4 or max(abs(h[2]) for h in hits) > synth.BARREL_HALF_Z:
            continue
        H = np.array(hits)
        H[:, 0] += rng.normal(0, 1e-4, 4)        # 1 um smearing: scattering dominates
        H[:, 1] += rng.normal(0, 1e-4, 4)
        Pf = synth.params_barrel_quadruplets()
        Pf.sigma_rphi = 1.4e-4
        Pf.sigma_z = 1.0e-4
        f = orc.fit_one(H[:, 0], H[:, 1], H[:, 2], np.arange(4), Pf)
        assert f["status"] == 0
        chi += f["chi2"]
        ndf += 3
        n += 1
    print("chi2/ndf", chi / ndf)
    assert abs(chi / ndf - 1.0) < 0.1, chi / ndf


def _design(s, meas, w, kvar, curv):
    n = len(s)
    m = n + (1 if curv else 0)
    rows, rhs = [], []
    for i in range(n):
        r = np.zeros(m)
        r[i] = math.sqrt(w[i])
        rows.append(r)
        rhs.append(math.sqrt(w[i]) * meas[i])
    for j in range(1, n - 1):
        ds0, ds1 = s[j] - s[j - 1], s[j + 1] - s[j]
        r = np.zeros(m)
        # kink: slope after minus slope before, plus the curvature bend over the two half-gaps
        r[j + 1] += 1 / ds1
        r[j] -= 1 / ds1
        r[j] -= 1 / ds0
        r[j - 1] += 1 / ds0
        if curv:
            r[n] = 0.5 * (ds0 + ds1)
        rows.append(r / math.sqrt(kvar[j]))
        rhs.append(0.0)
    return np.array(rows), np.array(rhs)


@pytest.mark.parametrize("curv", [True, False])
def test_normal_equations_equal_lstsq(orc, curv):
    rng = np.random.default_rng(11)
    for _ in range(500):
        n = int(rng.integers(3, 9))
        s = np.cumsum(rng.uniform(2, 6, n)) - 2.0
        meas = rng.normal(0, 1e-3, n)
        w = rng.uniform(0.5, 2, n) * 1e6
        kvar = rng.uniform(0.5, 2, n) * 1e-6
        x, chi2 = orc.bl_solve(s, meas, w, kvar, curv)
        A, b = _design(s, meas, w, kvar, curv)
        ref, *_ = np.linalg.lstsq(A, b, rcond=None)
        scale = np.max(np.abs(ref)) + 1e-12
        assert np.max(np.abs(x - ref)) <= 1e-8 * scale
        assert chi2 == pytest.approx(float(np.sum((A @ ref - b) ** 2)), rel=1e-7, abs=1e-12)


def _exact_minimiser(s, meas, w, kvar, curv):
    """The broken line's chi2 minimiser in exact rational arithmetic: the normal equations in the
    offsets (and the curvature correction), written from the definition of the kinks, solved by
    Gaussian elimination on fractions (the inputs are doubles, so they are exact rationals)."""
    n = len(s)
    m = n + (1 if curv else 0)
    s, meas, w, kvar = ([Fraction(float(v)) for v in a] for a in (s, meas, w, kvar))
    A = [[Fraction(0)] * m for _ in range(m)]
    b = [Fraction(0)] * m
    for i in range(n):
        A[i][i] += w[i]
        b[i] += w[i] * meas[i]
    for j in range(1, n - 1):
        d0, d1 = s[j] - s[j - 1], s[j + 1] - s[j]
        g = [Fraction(0)] * m
        g[j - 1], g[j], g[j + 1] = 1 / d0, -1 / d0 - 1 / d1, 1 / d1
        if curv:
            g[n] = (d0 + d1) / 2
        for r in range(m):
            for c in range(m):
                A[r][c] += g[r] * g[c] / kvar[j]
    M = [A[r] + [b[r]] for r in range(m)]
    for k in range(m):
        for r in range(k + 1, m):
            f = M[r][k] / M[k][k]
            for c in range(k, m + 1):
                M[r][c] -= f * M[k][c]
    x = [Fraction(0)] * m
    for k in reversed(range(m)):
        x[k] = (M[k][m] - sum(M[k][c] * x[c] for c in range(k + 1, m))) / M[k][k]
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("curv", [True, False])
def test_broken_line_equals_exact_minimiser(orc, curv):
    """From soft to extremely stiff kinks (kink variances 1e-4 .. 1e-22 against measurement
    weights ~1e6, as nearly straight tracks with a large prefit momentum give), the solve equals
    the exact minimiser of the chi2 to FP64 accuracy (the stiff limit is the weighted
    least-squares line or parabola, which a solve of the offset normal equations in FP64 misses
    by up to 1e-3)."""
    rng = np.random.default_rng(29)
    for t in range(80):
        n = int(rng.integers(3, 7))
        s = np.cumsum(rng.uniform(2, 6, n)) - 2.0
        meas = rng.normal(0, 1e-3, n) + (0.3 * s if t % 2 else 0.0)
        w = rng.uniform(0.5, 2, n) * 1e6
        kvar = 10.0 ** rng.uniform(-22, -4) * rng.uniform(0.5, 2, n)
        x, chi2 = orc.bl_solve(s, meas, w, kvar, curv)
        ref = _exact_minimiser(s, meas, w, kvar, curv)
        assert np.max(np.abs(x[:n] - ref[:n])) <= 1e-9 * (np.max(np.abs(ref[:n])) + 1e-6), t
        if curv:     # the curvature correction, on the scale of the offsets' curvature
            scale = abs(ref[n]) + np.max(np.abs(meas)) / (s[-1] - s[0]) ** 2
            assert abs(x[n] - ref[n]) <= 1e-9 * scale, t


def test_curvature_term_sign(orc):
    """Offsets that follow -delta s^2 / 2 (a path bending more than the reference) are explained by
    delta alone, with no kink: the solution is exact and the chi2 vanishes."""
    s = np.array([0.0, 3.9, 8.0, 13.1])
    delta = 2e-4
    meas = -0.5 * delta * s ** 2 + 1e-3 * s
    x, chi2 = orc.bl_solve(s, meas, np.full(4, 1e6), np.full(4, 1e-8), True)
    assert x[4] == pytest.approx(delta, rel=1e-9)
    assert chi2 < 1e-18


def test_symmetries(orc):
    p = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(500, seed=5)
    for t in range(500):
        X, Y, Z, L = tb.x64[t], tb.y64[t], tb.z64[t], tb.layer[t]
        f = orc.fit_one(X, Y, Z, L, p)
        a = 0.7
        Xr = X * math.cos(a) - Y * math.sin(a)
        Yr = X * math.sin(a) + Y * math.cos(a)
        g = orc.fit_one(Xr, Yr, Z, L, p)
        assert g["pt"] == pytest.approx(f["pt"], rel=1e-9)
        assert g["dxy"] == pytest.approx(f["dxy"], rel=1e-6, abs=1e-11)
        assert abs(_wrap(g["phi"] - f["phi"] - a)) < 1e-9
        m = orc.fit_one(X, -Y, Z, L, p)        # mirror: charge, phi and dxy = q(|C| - R) flip
        assert m["charge"] == -f["charge"]
        assert abs(_wrap(m["phi"] + f["phi"])) < 1e-9
        assert m["pt"] == pytest.approx(f["pt"], rel=1e-9)
        assert m["dxy"] == pytest.approx(-f["dxy"], rel=1e-6, abs=1e-11)
        zr = orc.fit_one(X, Y, -Z, L, p)                      # z reflection
        assert zr["cot_theta"] == pytest.approx(-f["cot_theta"], rel=1e-9, abs=1e-12)
        assert zr["dz"] == pytest.approx(-f["dz"], rel=1e-9, abs=1e-11)
