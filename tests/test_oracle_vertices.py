"""Pins of the oracle's primary-vertex finding: a hand-made track list whose clusters follow from
the definition by inspection, the handling of tracks that are not kept, and the purpose on
generated events with known vertices (found, and at the right z)."""
import math

import numpy as np

import oracle
from oracle import Q_GOOD, Q_KEPT
from paper_2104_06573_gb300 import synth

K = Q_GOOD | Q_KEPT


def fits_of(dz, pt):
    f = np.zeros(len(dz), oracle.TRACK_DTYPE)
    f["dz"], f["pt"] = dz, pt
    return f


def test_gap_clustering_by_hand():
    dz = [1.03, 0.0, 5.0, 0.02, 1.0, 0.01, 5.2]
    pt = [3.0, 1.0, 9.0, 1.0, 3.0, 1.0, 1.0]
    q = np.full(7, K, np.uint8)
    v, vid = oracle.find_vertices(fits_of(dz, pt), q, gap=0.05, min_tracks=2)
    # clusters: {0.0, 0.01, 0.02} (pt^2 sum 3), {1.0, 1.03} (18); {5.0} and {5.2} are singles
    assert v["n_tracks"].tolist() == [2, 3]                 # ordered by sum pT^2: 18, then 3
    assert np.allclose(v["z"], [1.015, 0.01])
    assert np.allclose(v["sum_pt2"], [18.0, 3.0])
    assert np.allclose(v["z_err"], [math.sqrt(2 * 0.015 ** 2 / 2), math.sqrt(2 * 0.01 ** 2 / 6)])
    assert vid.tolist() == [0, 1, -1, 1, 0, 1, -1]
    # gap at the threshold joins (inclusive); just above splits
    v, vid = oracle.find_vertices(fits_of([0.0, 0.05, 0.1000001], [1, 1, 1]), np.full(3, K, np.uint8),
                                  gap=0.05, min_tracks=2)
    assert v["n_tracks"].tolist() == [2] and vid.tolist() == [0, 0, -1]


def test_tracks_not_kept_are_ignored():
    dz = [0.0, 0.01, 0.02, 0.03]
    q = np.array([K, Q_GOOD, 0, K], np.uint8)           # only tracks 0 and 3 are kept
    v, vid = oracle.find_vertices(fits_of(dz, [1, 1, 1, 1]), q, gap=0.015, min_tracks=2)
    assert len(v["z"]) == 0                             # 0.0 and 0.03 are 0.03 apart
    v, vid = oracle.find_vertices(fits_of(dz, [1, 1, 1, 1]), q, gap=0.05, min_tracks=2)
    assert v["n_tracks"].tolist() == [2] and vid.tolist() == [0, -1, -1, 0]


def test_generated_vertices_are_found():
    """Smeared barrel event with 40 vertices: every generated vertex with at least 5 kept
    tracks has a found vertex within 0.02 cm unless another generated vertex lies within 0.1 cm
    of it (the gap clustering merges such pairs), and the found z's scatter about the truth by
    well under the gap."""
    P = synth.params_barrel_quadruplets()
    ev = synth.make_event(21, 2000, smear=True, n_vertices=40)
    r = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, P)
    q = oracle.select_tracks(r["tuples"], r["tuple_n"], r["fits"], clean_shared=True)
    v, vid = oracle.find_vertices(r["fits"], q, gap=0.05, min_tracks=2)
    truth_z = np.unique(ev.tracks.zv)
    # generated vertices and how many of their tracks were kept
    tids = [ev.track[r["tuples"][t, 0]] for t in range(len(q))]
    kept_z = [ev.tracks.zv[i] for i, t in zip(tids, range(len(q))) if i >= 0 and q[t] & Q_KEPT]
    zs, counts = np.unique(kept_z, return_counts=True)
    big = zs[counts >= 5]
    d = np.array([np.min(np.abs(v["z"] - z)) for z in big])
    near = np.array([np.sort(np.abs(truth_z - z))[1] < 0.1 for z in big])
    print("vertices", len(v["z"]), "generated", len(truth_z), "with >= 5 tracks", len(big),
          "close pairs", near.sum(), "median |dz|", np.median(d))
    assert np.all((d < 0.02) | near)
    assert np.median(d) < 0.002
