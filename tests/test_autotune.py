"""Autotuner: the coordinate-descent search on a synthetic cost (CPU), the cache, and (GPU) that
tuned settings change the time but not the result."""
import numpy as np
import pytest

from paper_2104_06573_gb300 import autotune, pxr, synth


def _cost(best_nb, best_grid):
    def measure(nb, grid):
        t = 10.0 + abs(np.log2(nb) - np.log2(best_nb))
        for k, g in enumerate(grid):
            eff = g if g else 8
            t += 0.1 * abs(np.log2(eff) - np.log2(best_grid[k]))
        return t
    return measure


def test_search_finds_separable_optimum():
    best_grid = [2, 32, 4, 16, 8, 2]
    nb, grid, t, calls = autotune.search(_cost(256, best_grid))
    assert nb == 256
    assert [g if g else 8 for g in grid] == best_grid     # built-in (0) counts as 8 here
    assert t == pytest.approx(10.0)
    assert calls == len(autotune.BINS) + autotune.N_STAGES * len(autotune.GRIDS)


def test_search_keeps_builtin_when_nothing_is_better():
    # a cost that every explicit grid value worsens: the built-in (0) stays
    def measure(nb, grid):
        return 1.0 + 0.5 * sum(1 for g in grid if g) + (0 if nb == 512 else 1)
    nb, grid, t, _ = autotune.search(measure)
    assert nb == 512 and grid == [0] * autotune.N_STAGES and t == 1.0


def test_cache_roundtrip_and_key(tmp_path):
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    Q = pxr.params_from(synth.params_phase1(), cut_mode=pxr.CUT_FP32)
    k1 = autotune.cache_key(P, 256, 3_200_000)
    assert k1 == autotune.cache_key(P, 256, 3_250_000)          # same shape bucket
    assert k1 != autotune.cache_key(Q, 256, 3_200_000)          # other geometry
    assert k1 != autotune.cache_key(P, 64, 3_200_000)
    path = str(tmp_path / "tune.json")
    autotune.store_cache(path, k1, {"n_phi_bins": 256, "grid_per_sm": [1, 2, 3, 4, 5, 6]})
    assert autotune.load_cache(path)[k1]["grid_per_sm"] == [1, 2, 3, 4, 5, 6]
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


def test_with_copies_and_sets_fields():
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    Q = autotune._with(P, 1024, [3, 0, 5, 0, 0, 7])
    assert Q.n_phi_bins == 1024 and list(Q.grid_per_sm) == [3, 0, 5, 0, 0, 7]
    assert P.n_phi_bins == 0 and list(P.grid_per_sm) == [0] * 6
    assert Q.cos_phi_window == P.cos_phi_window and Q.n_pairs == P.n_pairs


@pytest.mark.gpu
def test_tuned_settings_do_not_change_results(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    evs = [synth.event_serving(500 + k, n) for k, n in enumerate([300, 2500, 40, 1200])]
    off = np.zeros(len(evs) + 1, np.uint32)
    off[1:] = np.cumsum([e.n for e in evs])
    cat = lambda k: np.concatenate([getattr(e, k) for e in evs])
    x, y, z = (torch.from_numpy(cat(k)).to(dev) for k in "xyz")
    layer = torch.from_numpy(cat("layer").view(np.int16)).to(dev)
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32,
                        fit_mode=pxr.FIT_MIXED)
    with pxr.Context(device=0, mem_budget_bytes=4 << 30) as ctx:
        cache = str(tmp_path / "tune.json")
        T, info = autotune.tune_plan(ctx, off, x, y, z, layer, P, reps=1, bins=(256, 1024),
                                     grids=(1, 32), cache=cache)
        assert info["trials"] == 2 + 6 * 2 and info["n_phi_bins"] in (256, 1024)
        _, again = autotune.tune_plan(ctx, off, x, y, z, layer, P, cache=cache)
        assert again.get("cached") and again["grid_per_sm"] == info["grid_per_sm"]
        out = []
        for prm in (P, T):
            plan = pxr.Plan(ctx, off, x, y, z, layer, prm, use_graph=True)
            plan.pxr_plan_run()
            out.append([plan.pxr_plan_tracks(e) for e in range(len(evs))])
            plan.close()
    for a, b in zip(*out):
        for k in pxr.TRACK_FIELDS:
            assert np.array_equal(a[k], b[k]), k
