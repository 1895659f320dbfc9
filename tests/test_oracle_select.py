"""Pins of the oracle's track selection (quality cuts and shared-hit cleaning).

Hand-made track lists whose expected bits follow from the definition by inspection, the
definition's invariants on a dense event, and its purpose on generated events with known truth
(cleaning removes combinatorial fakes and keeps the generated tracks)."""
import numpy as np
import pytest

import oracle
from oracle import Q_GOOD, Q_KEPT
from paper_2104_06573_gb300 import synth

G, K = Q_GOOD, Q_GOOD | Q_KEPT


def tracks(rows):
    """rows: (hits, chi2, status, pt) -> tuples, tuple_n, fits as reconstruct returns them."""
    nt = len(rows)
    tup = np.full((nt, 8), 0xFFFFFFFF, np.uint32)
    tn = np.zeros(nt, np.uint8)
    fits = np.zeros(nt, oracle.TRACK_DTYPE)
    for t, (h, chi2, st, pt) in enumerate(rows):
        tup[t, :len(h)] = h
        tn[t] = len(h)
        fits[t]["chi2"], fits[t]["status"], fits[t]["pt"] = chi2, st, pt
    return tup, tn, fits


def test_rank_by_hits_then_chi2_one_round():
    # T0 and T1 share hit 1: equal length, T0 has the smaller chi2/ndof (0.5 vs 2.0): T1 drops.
    # T2 (a triplet with a tiny chi2) shares hit 7 with T1: T1 has more hits, so T2 drops too,
    # although T1 itself was dropped (one round).  T3 shares nothing.
    rows = [((1, 2, 3, 4), 1.5, 0, 2.0),        # ndof 3: 0.5
            ((1, 5, 6, 7), 6.0, 0, 2.0),        # 2.0
            ((7, 8, 9), 0.01, 0, 2.0),          # ndof 1: 0.01
            ((10, 11, 12, 13), 9.0, 0, 2.0)]
    q = oracle.select_tracks(*tracks(rows), clean_shared=True)
    assert q.tolist() == [K, G, G, K]
    # without cleaning every good track is kept
    assert oracle.select_tracks(*tracks(rows)).tolist() == [K, K, K, K]


def test_ties_keep_both_and_bad_fits_do_not_suppress():
    rows = [((1, 2, 3, 4), 3.0, 0, 1.0),
            ((4, 5, 6, 7), 3.0, 0, 1.0),        # shares hit 4, same rank: both kept
            ((7, 8, 9, 10, 11), 0.0, 3, 1.0),   # longer but its fit failed: not good, no effect
            ((20, 21, 22), 5.0, 1, 1.0)]
    q = oracle.select_tracks(*tracks(rows), clean_shared=True)
    assert q.tolist() == [K, K, 0, 0]


def test_cut_thresholds_inclusive_and_ndof():
    rows = [((1, 2, 3), 2.0, 0, 0.9),           # pT below 1.0
            ((4, 5, 6), 2.0, 0, 1.0),           # pT at the cut, chi2/ndof 2.0 at the cut
            ((7, 8, 9), 2.000001, 0, 5.0),      # chi2/ndof just above
            ((10, 11, 12, 13), 6.0, 0, 5.0),    # ndof 3: 2.0, at the cut
            ((14, 15, 16, 17, 18), 10.5, 0, 5.0),   # ndof 5: 2.1, above
            ((19, 20), 1.5, 0, 5.0)]            # 2 hits: ndof taken as 1
    q = oracle.select_tracks(*tracks(rows), pt_min=1.0, chi2_max=2.0)
    assert q.tolist() == [0, K, 0, K, 0, K]
    # a zero threshold is no cut
    assert (oracle.select_tracks(*tracks(rows)) == K).all()


def check_invariants(tup, tn, fits, q, clean):
    nt = len(tn)
    good = (q & Q_GOOD) != 0
    kept = (q & Q_KEPT) != 0
    assert not np.any(kept & ~good)
    if not clean:
        assert np.array_equal(kept, good)
        return
    hits = [set(int(h) for h in tup[t, :tn[t]]) for t in range(nt)]
    rank = [(-int(tn[t]), float(fits[t]["chi2"]) / max(2 * int(tn[t]) - 5, 1)) for t in range(nt)]
    by_hit = {}
    for t in np.flatnonzero(good):
        for h in hits[t]:
            by_hit.setdefault(h, []).append(int(t))
    for t in np.flatnonzero(good):
        rivals = {u for h in hits[t] for u in by_hit[h] if u != t}
        better = [u for u in rivals if rank[u] < rank[t]]
        assert bool(kept[t]) == (not better)
        # two kept tracks share a hit only when they rank equal
        for u in rivals:
            if kept[t] and kept[u]:
                assert rank[u] == rank[t]


@pytest.mark.parametrize("clean", [False, True])
def test_invariants_dense_event(clean):
    P = synth.params_phase1()
    ev = synth.event_phase1(3, 600)
    r = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, P)
    q = oracle.select_tracks(r["tuples"], r["tuple_n"], r["fits"], pt_min=0.6, chi2_max=20.0,
                             clean_shared=clean)
    good = (q & Q_GOOD) != 0
    assert 0 < good.sum() < len(q)            # the cuts act, and not on everything
    check_invariants(r["tuples"], r["tuple_n"], r["fits"], q, clean)


def truth_of(ev, tup, n):
    ids = ev.track[tup[:n]]
    return int(ids[0]) if ids[0] >= 0 and np.all(ids == ids[0]) else -1


def test_cleaning_removes_fakes_keeps_generated_tracks():
    """Smeared dense barrel event: the CA forms combinatorial fakes that share hits with the
    generated tracks.  Cleaning must lower the fake fraction and keep nearly every generated
    track that was found."""
    P = synth.params_barrel_quadruplets()
    ev = synth.make_event(11, 3000, smear=True)
    r = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, P)
    q = oracle.select_tracks(r["tuples"], r["tuple_n"], r["fits"], clean_shared=True)
    tid = np.array([truth_of(ev, r["tuples"][t], r["tuple_n"][t]) for t in range(len(q))])
    good = (q & Q_GOOD) != 0
    kept = (q & Q_KEPT) != 0
    fake_good = np.mean(tid[good] < 0)
    fake_kept = np.mean(tid[kept] < 0)
    print("fake fraction good", fake_good, "kept", fake_kept, "tracks", good.sum(), kept.sum())
    assert fake_good > 0.01                    # there are fakes to remove
    assert fake_kept < 0.5 * fake_good
    found = set(tid[good & (tid >= 0)])
    kept_true = set(tid[kept & (tid >= 0)])
    assert len(kept_true) >= 0.98 * len(found)
