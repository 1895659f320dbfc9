"""Host-side checks of the seeded synthetic workload generator."""
import math

import numpy as np

from paper_2104_06573_gb300 import synth


def test_splitmix_is_counter_based_and_seeded():
    a = synth.Rng(5, 1).raw(100)
    b = synth.Rng(5, 1)
    assert np.array_equal(a[:40], b.raw(40))
    assert np.array_equal(a[40:], b.raw(60))          # sequential reads continue the stream
    assert not np.array_equal(a, synth.Rng(6, 1).raw(100))
    assert not np.array_equal(a, synth.Rng(5, 2).raw(100))
    u = synth.Rng(0, 0).uniform(200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    g = synth.Rng(0, 3).normal(200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


def test_splitmix_reference_values():
    """SplitMix64 with state 0 yields 0xE220A8397B1DCDAF first (published test vector)."""
    z = np.array([0], dtype=np.uint64) + synth._GOLDEN
    with np.errstate(over="ignore"):
        assert int(synth._mix64(z)[0]) == 0xE220A8397B1DCDAF


def test_event_shapes_and_determinism():
    e = synth.event_barrel(0)
    e2 = synth.event_barrel(0)
    assert np.array_equal(e.x, e2.x) and np.array_equal(e.layer, e2.layer)
    assert e.x.dtype == np.float32 and e.layer.dtype == np.uint16
    assert 350 <= e.n <= 400
    assert set(np.unique(e.layer)) <= {0, 1, 2, 3}
    assert np.all(e.x == e.x64.astype(np.float32))
    r = np.hypot(e.x64, e.y64)
    radii = np.array(synth.BARREL_R)[e.layer]
    assert np.allclose(r, radii, rtol=0, atol=1e-9)
    assert np.all(np.abs(e.z64) < synth.BARREL_HALF_Z)


def test_dense_event_has_disks_and_noise():
    e = synth.event_phase1(0)
    assert 9000 < e.n < 11000
    assert np.sum(e.track < 0) > 0.15 * np.sum(e.track >= 0)
    assert set(np.unique(e.layer)) == set(range(10))
    disk = e.layer >= 4
    rd = np.hypot(e.x64[disk], e.y64[disk])
    assert rd.min() >= synth.DISK_RMIN - 0.01 and rd.max() <= synth.DISK_RMAX + 0.01


def test_batch_counts_in_range():
    c = synth.batch_track_counts(256)
    assert len(c) == 256 and min(c) >= 200 and max(c) <= 6000
    assert 2500 < np.mean(c) < 3700


def test_helix_hits_lie_on_generated_circles():
    rng = synth.Rng(3, 7)
    tr = synth.draw_tracks(rng, 200, "loguniform", 0.5, 100.0, 2.5)
    tid, lay, s, x, y, z = synth.helix_points(tr, True)
    R = synth.radius_of(tr.pt)[tid]
    q = tr.q[tid]
    cx = q * R * np.sin(tr.phi0[tid])
    cy = -q * R * np.cos(tr.phi0[tid])
    assert np.allclose(np.hypot(x - cx, y - cy) / R, 1.0, rtol=0, atol=1e-12)
    assert np.allclose(z, tr.zv[tid] + s * tr.cot[tid], atol=1e-9)


def test_serving_stream():
    t, n = synth.serving_stream(1000.0, 20000, seed=1)
    assert np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 1000.0) < 30
    assert n.max() <= 8000 and abs(np.median(n) - 1500) < 60


def test_fit_tuplets():
    tb = synth.fit_tuplets(10000, seed=2)
    assert tb.x.shape == (10000, 4)
    assert abs(np.mean(tb.n_hits == 3) - 0.3) < 0.02
    lp = np.log(tb.tracks.pt)
    assert lp.min() >= math.log(0.5) - 1e-9 and lp.max() <= math.log(100.0) + 1e-9
