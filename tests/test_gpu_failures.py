"""Failure handling of the library, exercised from the host (no GPU fault, trap or hang is ever
provoked): admission refusal when the memory budget is full, refusal of events that can never
fit it, malformed inputs, bounded polling, and injected arena allocation failures.  After each
failure the context must keep working and give correct results."""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2104_06573_gb300 import pxr, synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def ev_args(ev):
    return ev.x, ev.y, ev.z, ev.layer


def drain(ctx, tickets, timeout_s=60.0, seen=()):
    """Poll until every ticket has finished (`seen`: tickets an earlier poll already reported;
    a poll reports each finished ticket once), then fetch them."""
    done, t0 = set(seen) & set(tickets), time.time()
    while len(done) < len(tickets):
        done |= set(ctx.pxr_poll(timeout_us=100000))
        assert time.time() - t0 < timeout_s, "served events did not finish"
    return {t: ctx.pxr_fetch_tracks(t) for t in tickets}


def test_event_beyond_budget_is_refused_and_context_survives():
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    big, small = synth.event_barrel(1, 8000), synth.event_barrel(2, 50)
    with pxr.Context(device=0, mem_budget_bytes=16 << 20) as ctx:
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_submit_event(*ev_args(big), P)
        assert ei.value.code == pxr.ENOMEM
        t = ctx.pxr_submit_event(*ev_args(small), P)
        r = drain(ctx, [t])[t]
        assert r["status"] == pxr.OK and len(r["n_hits"]) > 0


def submit_until(ctx, ev, P, seen, timeout_s=60.0):
    """Submit, polling while the budget is full; tickets the polls report go into `seen`."""
    t0 = time.time()
    while True:
        t = ctx.try_submit_event(*ev_args(ev), P)
        if t is not None:
            return t
        seen.update(ctx.pxr_poll(timeout_us=10000))
        assert time.time() - t0 < timeout_s, "the budget never freed"


def test_full_budget_refuses_then_recovers():
    """A budget for one or two events: submissions beyond it are refused with EAGAIN (nothing is
    queued); after polling, the accepted and the resubmitted events complete with the tracks the
    same events give alone."""
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    evs = [synth.event_barrel(10 + k, 3000) for k in range(24)]
    budget = 8 << 20
    while True:                      # the smallest budget (doubling) that holds one event
        with pxr.Context(device=0, mem_budget_bytes=budget) as ctx:
            try:
                drain(ctx, [ctx.pxr_submit_event(*ev_args(evs[0]), P)])
                break
            except pxr.PxrError as e:
                assert e.code == pxr.ENOMEM
        budget *= 2
        assert budget <= 1 << 30
    with pxr.Context(device=0, mem_budget_bytes=budget) as ctx:
        accepted, refused = [], []
        for k, ev in enumerate(evs):
            t = ctx.try_submit_event(*ev_args(ev), P)
            (refused if t is None else accepted).append(k if t is None else (k, t))
        assert refused, "the budget never filled"
        res = drain(ctx, [t for _, t in accepted])
        seen = set()
        later = [(k, submit_until(ctx, evs[k], P, seen)) for k in refused[:3]]
        res.update(drain(ctx, [t for _, t in later], seen=seen))
    with pxr.Context(device=0, mem_budget_bytes=1 << 30) as ref:
        for k, t in accepted[:2] + later:
            a = next(iter(drain(ref, [ref.pxr_submit_event(*ev_args(evs[k]), P)]).values()))
            assert res[t]["status"] == pxr.OK
            assert np.array_equal(res[t]["hit_idx"], a["hit_idx"])
            assert np.array_equal(res[t]["pt"], a["pt"])


def test_malformed_inputs_are_refused():
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    ev = synth.event_barrel(3, 30)
    with pxr.Context(device=0, mem_budget_bytes=64 << 20) as ctx:
        x = ev.x.copy()
        x[5] = np.nan
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_submit_event(x, ev.y, ev.z, ev.layer, P)
        assert ei.value.code == pxr.EINVAL
        lay = ev.layer.copy()
        lay[3] = 7                       # the barrel geometry has 4 layers
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_submit_event(ev.x, ev.y, ev.z, lay, P)
        assert ei.value.code == pxr.EINVAL
        bad = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
        bad.theta_cut = -1.0
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_submit_event(*ev_args(ev), bad)
        assert ei.value.code == pxr.EINVAL
        # nothing was queued; polling returns at once, and a good event still goes through
        t0 = time.time()
        assert ctx.pxr_poll(timeout_us=0) == []
        assert time.time() - t0 < 1.0
        t = ctx.pxr_submit_event(*ev_args(ev), P)
        assert drain(ctx, [t])[t]["status"] == pxr.OK


def test_unknown_ticket_and_double_fetch():
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    with pxr.Context(device=0, mem_budget_bytes=64 << 20) as ctx:
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_fetch_tracks(12345)
        assert ei.value.code == pxr.ENOTFOUND
        t = ctx.pxr_submit_event(*ev_args(synth.event_barrel(4, 20)), P)
        drain(ctx, [t])
        with pytest.raises(pxr.PxrError) as ei:
            ctx.pxr_fetch_tracks(t)                 # released by the first fetch
        assert ei.value.code == pxr.ENOTFOUND


INJECT = r"""
import numpy as np, torch
from paper_2104_06573_gb300 import pxr, synth
ev = synth.event_barrel(5, 200)
dev = torch.device("cuda:0")
x, y, z = (torch.from_numpy(getattr(ev, k)).to(dev) for k in "xyz")
layer = torch.from_numpy(ev.layer.view(np.int16)).to(dev)
P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
with pxr.Context(device=0, mem_budget_bytes=256 << 20) as ctx:
    try:
        pxr.Plan(ctx, [0, ev.n], x, y, z, layer, P)
        print("FIRST OK")
    except pxr.PxrError as e:
        print("FIRST FAILED", e.code)
    plan = pxr.Plan(ctx, [0, ev.n], x, y, z, layer, P)
    plan.pxr_plan_run()
    print("SECOND TRACKS", len(plan.pxr_plan_tracks(0)["n_hits"]))
    plan.close()
"""


def test_injected_arena_failure_is_reported_and_recovered():
    """PXR_FAULT_ARENA=1 makes the first arena allocation of the process fail (a host-side
    hook): plan creation reports the error, and the next plan in the same context works."""
    env = dict(os.environ, PXR_FAULT_ARENA="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", INJECT], env=env, cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stdout.splitlines()
    assert any(l.startswith("FIRST FAILED") and int(l.split()[-1]) in (pxr.EAGAIN, pxr.ENOMEM)
               for l in lines), out.stdout
    n = [int(l.split()[-1]) for l in lines if l.startswith("SECOND TRACKS")]
    assert n and n[0] >= 150, out.stdout
