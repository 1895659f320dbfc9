"""The allocation-free doublet entry point against the regular device path.

pxr_doublets_noalloc exists for callers that cannot let a library allocate device memory (serving
loops that must not call cudaMalloc after start-up, applications whose device memory belongs to
their own pool).  It keeps its scratch in a fixed array in device global memory.  Here it is
called through the C ABI twice in a row, on two different events, and each call's cells must equal
the cells the existing plan path reports for the same event (integer sets: bit-exact).  The second
call checks that nothing from the first call leaks through the shared array.  Size limits are
rejected on the host before any launch.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2104_06573_gb300 import pxr, synth  # noqa: E402


def _dev(ev):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(ev.x).to(dev), torch.from_numpy(ev.y).to(dev),
            torch.from_numpy(ev.z).to(dev),
            torch.from_numpy(ev.layer.view(np.int16)).to(dev))


def _plan_cells(ctx, ev, params):
    x, y, z, layer = _dev(ev)
    plan = pxr.Plan(ctx, [0, ev.n], x, y, z, layer, params, use_graph=False)
    plan.pxr_plan_run()
    cells = plan.pxr_plan_debug(0, 0)
    plan.close()
    return {tuple(c) for c in cells.tolist()}, len(cells)


def _noalloc_call(ev, params, cap):
    """One call; returns (written cells as a list of pairs, cell count, flag word)."""
    dev = torch.device("cuda:0")
    x, y, z, layer = _dev(ev)
    inner = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    outer = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    pxr.pxr_doublets_noalloc(x, y, z, layer, ev.n, params, inner, outer, cap, n, flags)
    torch.cuda.synchronize()
    k = int(n.item())
    w = min(k, cap)
    got = np.stack([inner[:w].cpu().numpy().view(np.uint32),
                    outer[:w].cpu().numpy().view(np.uint32)], 1)
    return [tuple(c) for c in got.tolist()], k, int(flags.item())


def _noalloc_cells(ev, params, cap):
    cells, k, flags = _noalloc_call(ev, params, cap)
    assert flags == 0
    return set(cells), k


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = pxr.Context(device=0, mem_budget_bytes=4 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("cut", [pxr.CUT_FP32, pxr.CUT_FP64])
def test_noalloc_equals_plan_path_two_calls(ctx, cut):
    events = [(synth.event_phase1(3), synth.params_phase1()),
              (synth.event_barrel(7, 400), synth.params_barrel_quadruplets())]
    for ev, P in events:                       # two calls in a row, different events
        params = pxr.params_from(P, cut_mode=cut)
        want, n_want = _plan_cells(ctx, ev, params)
        got, n_got = _noalloc_cells(ev, params, cap=1 << 20)
        assert n_got == n_want > 0
        assert got == want


def test_noalloc_rejects_sizes_beyond_its_limits():
    P = pxr.params_from(synth.params_barrel_quadruplets())
    big = 65537
    dummy = 1 << 12                            # never dereferenced: rejected before any launch
    with pytest.raises(pxr.PxrError) as e1:
        pxr.pxr_doublets_noalloc(dummy, dummy, dummy, dummy, big, P, dummy, dummy, 16, dummy)
    assert e1.value.code == pxr.EINVAL and "65536" in str(e1.value)
    with pytest.raises(pxr.PxrError) as e2:
        pxr.pxr_doublets_noalloc(dummy, dummy, dummy, dummy, 10, P, dummy, dummy, (1 << 20) + 1,
                                 dummy)
    assert e2.value.code == pxr.EINVAL and "1048576" in str(e2.value)


def test_noalloc_overflow_then_full_call():
    """cap below the event's cell count: the full count is reported, flag bit 1 is set and the cap
    written pairs are distinct cells of the event.  A following call with room for every cell
    gives exactly the plan path's cells (nothing stale from the truncated call)."""
    P = synth.params_barrel_quadruplets()
    params = pxr.params_from(P, cut_mode=pxr.CUT_FP32)
    ev = synth.event_barrel(11, 400)
    c = pxr.Context(device=0, mem_budget_bytes=1 << 30)
    try:
        want, n_want = _plan_cells(c, ev, params)
    finally:
        c.close()
    cap = n_want // 3
    cells, k, flags = _noalloc_call(ev, params, cap)
    assert k == n_want > cap > 0
    assert flags & 1 and not flags & ~1
    assert len(cells) == cap and len(set(cells)) == cap and set(cells) <= want
    got, k2 = _noalloc_cells(ev, params, cap=1 << 20)
    assert k2 == n_want and got == want


def test_noalloc_bad_layer_id_flagged():
    """A hit whose layer id is beyond the geometry is left out and flagged (bit 8); every other
    cell is found exactly as the plan path finds it on the intact event."""
    P = synth.params_barrel_quadruplets()
    params = pxr.params_from(P, cut_mode=pxr.CUT_FP32)
    ev = synth.event_barrel(12, 300)
    c = pxr.Context(device=0, mem_budget_bytes=1 << 30)
    try:
        want, _ = _plan_cells(c, ev, params)
    finally:
        c.close()
    bad = int(np.flatnonzero(ev.layer == 1)[0])        # a hit that takes part in cells
    assert any(bad in cell for cell in want)
    layer = ev.layer.copy()
    layer[bad] = 200
    ev_bad = dataclasses.replace(ev, layer=layer)
    cells, k, flags = _noalloc_call(ev_bad, params, cap=1 << 20)
    assert flags == 8
    assert set(cells) == {cell for cell in want if bad not in cell} and k == len(cells)
