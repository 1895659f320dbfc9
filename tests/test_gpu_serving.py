"""Serving path, many events per call: pxr_submit_events / pxr_fetch_events against the
one-event calls and the device-resident plan path (bit-exact: the same kernels, canonical track
order), including empty and one-hit events, capacity errors and all-or-nothing admission."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2104_06573_gb300 import pxr, synth  # noqa: E402

FIELDS = ("n_hits", "hit_idx", "pt", "phi", "cot_theta", "dxy", "dz", "chi2", "charge",
          "fit_status", "quality")


def _events():
    counts = [50, 3000, 0, 800, 1, 5000, 200, 1500]
    evs = [synth.event_serving(500 + k, n) for k, n in enumerate(counts)]
    off = np.zeros(len(evs) + 1, np.uint32)
    off[1:] = np.cumsum([e.n for e in evs])
    cat = lambda k: np.concatenate([getattr(e, k) for e in evs])
    return evs, off, cat("x"), cat("y"), cat("z"), cat("layer")


def _wait(ctx, tickets):
    done = set()
    while not set(tickets) <= done:
        done |= set(ctx.pxr_poll(timeout_us=200000))


def test_many_events_equal_single_calls_and_plan():
    P = synth.params_barrel_quadruplets()
    p = pxr.params_from(P, cut_mode=pxr.CUT_FP32, fit_mode=pxr.FIT_SPLIT)
    evs, off, x, y, z, layer = _events()
    with pxr.Context(device=0, mem_budget_bytes=8 << 30, max_batch_events=3) as ctx:
        many = ctx.pxr_submit_events(off, x, y, z, layer, p)
        _wait(ctx, many)
        got = ctx.pxr_fetch_events(many)
        single = [ctx.pxr_submit_event(e.x, e.y, e.z, e.layer, p) for e in evs]
        _wait(ctx, single)
        ones = [ctx.pxr_fetch_tracks(t) for t in single]
    assert list(got["event_status"]) == [pxr.OK] * len(evs)
    toff = got["track_offsets"]
    assert toff[-1] == got["n"] == sum(o["n"] for o in ones)
    for k, one in enumerate(ones):
        for f in FIELDS:
            assert np.array_equal(got[f][toff[k]:toff[k + 1]], one[f]), (k, f)
    # the device-resident plan path gives the same tracks
    dev = torch.device("cuda:0")
    with pxr.Context(device=0, mem_budget_bytes=4 << 30) as ctx:
        t = lambda a: torch.from_numpy(a).to(dev)
        plan = pxr.Plan(ctx, off, t(x), t(y), t(z), t(layer.view(np.int16)), p, use_graph=False)
        plan.pxr_plan_run()
        for k in range(len(evs)):
            r = plan.pxr_plan_tracks(k)
            for f in FIELDS:
                assert np.array_equal(r[f], ones[k][f]), (k, f)
        plan.close()


def test_fetch_events_capacity_and_unknown_ticket():
    P = synth.params_barrel_quadruplets()
    p = pxr.params_from(P, cut_mode=pxr.CUT_FP32)
    evs, off, x, y, z, layer = _events()
    import ctypes as C
    with pxr.Context(device=0, mem_budget_bytes=8 << 30) as ctx:
        tk = ctx.pxr_submit_events(off[:4], x, y, z, layer, p)
        _wait(ctx, tk)
        L = pxr.load()
        a = np.ascontiguousarray(tk, np.uint64)
        toff = np.zeros(len(tk) + 1, np.uint32)
        t = pxr.pxr_tracks()
        t.capacity = 5                                   # too small: totals set, tickets kept
        rc = L.pxr_fetch_events(ctx.h, len(tk), a.ctypes.data, toff.ctypes.data, None, None,
                                C.byref(t))
        assert rc == pxr.ETRUNC and t.n_tracks == toff[-1] > 5
        bad = np.array([tk[0], 123456789], np.uint64)
        rc = L.pxr_fetch_events(ctx.h, 2, bad.ctypes.data, toff.ctypes.data, None, None,
                                C.byref(t))
        assert rc == pxr.ENOTFOUND
        got = ctx.pxr_fetch_events(tk)                   # still all there
        assert got["n"] == toff[-1]
        with pytest.raises(pxr.PxrError) as e:
            ctx.pxr_fetch_events(tk)                     # released by the successful fetch
        assert e.value.code == pxr.ENOTFOUND


def test_submit_events_all_or_nothing():
    P = synth.params_barrel_quadruplets()
    p = pxr.params_from(P, cut_mode=pxr.CUT_FP32)
    evs, off, x, y, z, layer = _events()
    with pxr.Context(device=0, mem_budget_bytes=32 << 20) as ctx:
        with pytest.raises(pxr.PxrError) as e:          # together (or one alone) beyond it
            ctx.pxr_submit_events(off, x, y, z, layer, p)
        assert e.value.code in (pxr.EAGAIN, pxr.ENOMEM)
        assert ctx.pxr_poll(timeout_us=0) == []
        small = [evs[0], evs[2], evs[4]]                 # 50, 0 and 1 tracks
        soff = np.zeros(4, np.uint32)
        soff[1:] = np.cumsum([e.n for e in small])
        cat = lambda k: np.concatenate([getattr(e, k) for e in small])
        sx, sy, sz, sl = cat("x"), cat("y"), cat("z"), cat("layer")
        bad = sl.copy()
        bad[-1] = 50                                     # one bad layer id: nothing admitted
        with pytest.raises(pxr.PxrError) as e:
            ctx.pxr_submit_events(soff, sx, sy, sz, bad, p)
        assert e.value.code == pxr.EINVAL
        assert ctx.pxr_poll(timeout_us=0) == []
        tk = ctx.pxr_submit_events(soff, sx, sy, sz, sl, p)   # the small group fits
        _wait(ctx, tk)
        got = ctx.pxr_fetch_events(tk)
        assert got["n"] > 0 and list(got["event_status"]) == [pxr.OK] * 3
