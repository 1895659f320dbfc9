"""The oracle's windowed doublet search (azimuth-sorted outer hits, binary-searched window; the
timed CPU baseline runs it) against its all-pairs search, the definition: the same cells in the
same order, hence the same edges, ntuplets and fits, on tiny events (every chain enumerated by
brute force elsewhere), the phi = +-pi seam, duplicated hits, the dense event with disks and
noise, and barrel events of the batch workload."""
import numpy as np
import pytest

from paper_2104_06573_gb300 import synth

from test_oracle_bruteforce import CASES, _tiny_event

KEYS = ("cells", "edges", "tuples", "tuple_n")


def same(orc, x, y, z, lay, P):
    a = orc.reconstruct(x, y, z, lay, P)
    b = orc.reconstruct(x, y, z, lay, P, windowed=True)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["fits"], b["fits"])
    return len(a["cells"])


@pytest.mark.parametrize("seed,ntr,disks,noise,loose", CASES)
def test_windowed_equals_all_pairs_tiny(orc, seed, ntr, disks, noise, loose):
    P = synth.params_phase1() if disks else synth.params_barrel_quadruplets()
    x, y, z, lay = _tiny_event(seed, ntr, disks, noise)
    assert same(orc, x, y, z, lay, P) > 0


def test_windowed_equals_all_pairs_seam_and_duplicates(orc):
    P = synth.params_barrel_quadruplets()
    # hits on both sides of phi = +-pi (the window wraps), each given twice
    rng = np.random.default_rng(3)
    phi = np.concatenate([rng.uniform(np.pi - 0.08, np.pi, 20), rng.uniform(-np.pi, -np.pi + 0.08, 20)])
    lay = rng.integers(0, 4, len(phi)).astype(np.uint16)
    r = np.array(synth.BARREL_R)[lay]
    x = (r * np.cos(phi)).astype(np.float32)
    y = (r * np.sin(phi)).astype(np.float32)
    z = rng.uniform(-5, 5, len(phi)).astype(np.float32)
    x, y, z, lay = (np.concatenate([a, a]) for a in (x, y, z, lay))
    assert same(orc, x, y, z, lay, P) > 0


def test_windowed_equals_all_pairs_dense_and_batch_events(orc):
    ev = synth.event_phase1(0)
    assert same(orc, ev.x, ev.y, ev.z, ev.layer, synth.params_phase1()) > 200000
    P = synth.params_barrel_quadruplets()
    for seed, n in ((1, 200), (2, 1500), (3, 3000)):
        ev = synth.make_event(seed, n)
        assert same(orc, ev.x, ev.y, ev.z, ev.layer, P) > 0
