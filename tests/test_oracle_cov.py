"""Pins of the oracle's track covariance (q/pT, phi, cot, dxy, dz).

The covariance is checked against what it must describe: the spread of fitted parameters around
the generated truth (pulls with unit width, with hit smearing alone and with simulated 3D
multiple scattering), the closed-form slope variance of a straight-line least-squares fit, and
its algebraic properties."""
import math

import numpy as np

import oracle
from paper_2104_06573_gb300 import synth
from test_oracle_fit import K, _propagate_to_radius


def pulls(fits, cov, truth):
    ok = (fits["status"] == 0) & np.all(np.isfinite(cov), axis=1)
    C = oracle.cov_matrix(cov[ok])
    est = np.stack([fits["charge"] / fits["pt"], fits["phi"], fits["cot_theta"], fits["dxy"],
                    fits["dz"]], 1)[ok]
    d = est - truth[ok]
    d[:, 1] = (d[:, 1] + np.pi) % (2 * np.pi) - np.pi
    sig = np.sqrt(np.stack([C[:, i, i] for i in range(5)], 1))
    return d / sig, ok


def test_pulls_smeared_helices():
    """Smeared helices (10 um r-phi, 20 um z) with negligible material: every parameter's pull
    has mean ~0 and width ~1."""
    P = synth.params_barrel_quadruplets()
    P.x_over_x0 = 1e-6
    tb = synth.fit_tuplets(3000, seed=5, triplet_frac=0.0)
    fits, cov = oracle.fit_cov_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    t = tb.tracks
    truth = np.stack([t.q / t.pt, t.phi0, t.cot, np.zeros(len(t.pt)), t.zv], 1)
    p, ok = pulls(fits, cov, truth)
    assert ok.mean() > 0.99
    print("pull mean", p.mean(0), "width", p.std(0))
    assert np.all(np.abs(p.mean(0)) < 0.08)
    assert np.all((p.std(0) > 0.93) & (p.std(0) < 1.08))


def test_pulls_with_multiple_scattering():
    """Low-momentum barrel tracks with simulated 3D scattering (Highland width) at the inner hits,
    where the broken line has its kinks, and 1 um smearing (r-phi, z): the covariance's kink terms must
    account for the spread.  (Material before the first hit is outside the fit's model: the
    parameters at the closest approach are the first segment's, extrapolated.)"""
    P = synth.params_barrel_quadruplets()
    Pf = synth.params_barrel_quadruplets()
    Pf.sigma_rphi = 1.0e-4
    Pf.sigma_z = 1.0e-4
    rng = np.random.default_rng(44)
    rows, truth = [], []
    while len(rows) < 1200:
        pt = rng.uniform(0.6, 2.0)
        eta = rng.uniform(-1.0, 1.0)
        phi0 = rng.uniform(-math.pi, math.pi)
        q = 1 if rng.uniform() < 0.5 else -1
        zv = rng.normal(0, 5.0)
        R = pt / (K * synth.BFIELD)
        p = pt * math.cosh(eta)
        d = np.array([math.cos(phi0) / math.cosh(eta), math.sin(phi0) / math.cosh(eta),
                      math.tanh(eta)])
        Pt = np.array([0.0, 0.0, zv])
        hits = []
        for li, rho in enumerate(synth.BARREL_R):
            res = _propagate_to_radius(Pt, d, q, R, rho)
            if res is None:
                break
            Pt, d = res
            hits.append(Pt.copy())
            if li not in (1, 2):
                continue
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
        # 1 um along r-phi and along z, the resolutions the fit is given
        rphi = rng.normal(0, 1e-4, 4) / np.hypot(H[:, 0], H[:, 1])
        H[:, 0], H[:, 1] = H[:, 0] - rphi * H[:, 1], H[:, 1] + rphi * H[:, 0]
        H[:, 2] += rng.normal(0, 1e-4, 4)
        rows.append(H)
        truth.append([q / pt, phi0, math.sinh(eta), 0.0, zv])
    H = np.array(rows)
    nh = np.full(len(H), 4, np.uint8)
    lay = np.tile(np.arange(4, dtype=np.uint16), (len(H), 1))
    fits, cov = oracle.fit_cov_batch(nh, H[:, :, 0], H[:, :, 1], H[:, :, 2], lay, Pf)
    p, ok = pulls(fits, cov, np.array(truth))
    assert ok.all()
    print("pull mean", p.mean(0), "width", p.std(0))
    assert np.all(np.abs(p.mean(0)) < 0.1)
    assert np.all((p.std(0) > 0.88) & (p.std(0) < 1.12))


def test_line_part_equals_least_squares_slope():
    """With (almost) no material the line kinks are stiff, the fitted z's lie on a line in (s, z), and
    the variance of cot is the closed-form slope variance sum(w) / (sum(w) sum(w s^2) -
    sum(w s)^2) of a weighted straight-line fit."""
    P = synth.params_barrel_quadruplets()
    # tiny material: the kinks are stiff (their freedom is ~1e-6 of the z errors) while the
    # normal matrix stays well enough conditioned in FP64 (~1e-5 at 100 GeV)
    P.x_over_x0 = 1e-8
    tb = synth.fit_tuplets(50, seed=9, triplet_frac=0.0, smear=False)
    fits, cov = oracle.fit_cov_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    w = 1.0 / P.sigma_z ** 2
    for t in range(50):
        x, y = tb.x64[t], tb.y64[t]
        # arc lengths along the generated circle (the reference circle through exact hits)
        R = tb.tracks.pt[t] / (K * synth.BFIELD)
        chord = np.hypot(x - x[0], y - y[0])
        s = 2 * R * np.arcsin(np.minimum(chord / (2 * R), 1.0))
        S0, S1, S2 = 4 * w, w * s.sum(), w * (s * s).sum()
        want = S0 / (S0 * S2 - S1 * S1)
        got = oracle.cov_matrix(cov[t])[2, 2]
        assert abs(got / want - 1) < 1e-4, (t, got, want)


def test_symmetric_positive_and_fit_unchanged():
    P = synth.params_barrel_quadruplets()
    tb = synth.fit_tuplets(500, seed=3)
    fits, cov = oracle.fit_cov_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    plain = oracle.fit_batch(tb.n_hits, tb.x64, tb.y64, tb.z64, tb.layer, P)
    assert fits.tobytes() == plain.tobytes()         # the covariance does not touch the fit
    ok = fits["status"] == 0
    C = oracle.cov_matrix(cov[ok])
    ev = np.linalg.eigvalsh(C)
    assert np.all(ev[:, 0] > -1e-12 * ev[:, -1])
    assert np.all(np.diagonal(C, axis1=1, axis2=2) > 0)
