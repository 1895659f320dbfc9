"""Autotuner: the coordinate-descent search on a synthetic cost (CPU), the cache and its key,
the library's check of the launch-shape fields, and (GPU) that tuned settings change the time
but not the result."""
import numpy as np
import pytest

from paper_2104_06573_gb300 import autotune, pxr, synth


def _cost(best_nb, best_grid, best_block):
    """A separable cost with its minimum at (best_nb, best_grid, best_block); the built-in
    values (0) count as grid 8 and block 256."""
    def measure(nb, grid, block):
        t = 10.0 + abs(np.log2(nb) - np.log2(best_nb))
        for k, g in enumerate(grid):
            t += 0.1 * abs(np.log2(g if g else 8) - np.log2(best_grid[k]))
        for k, b in enumerate(block):
            t += 0.01 * abs(np.log2(b if b else 256) - np.log2(best_block[k]))
        return t
    return measure


def test_search_finds_separable_optimum():
    best_grid = [2, 32, 4, 16, 8, 2]
    best_block = [512, 64, 256, 256, 256, 32]
    nb, grid, block, t, calls = autotune.search(_cost(64, best_grid, best_block))
    assert nb == 64                                       # the smallest bin count is searched
    assert [g if g else 8 for g in grid] == best_grid
    assert [b if b else 256 for b in block] == best_block
    assert block[2] == block[3] == block[4] == 0          # stages without a block axis
    assert t == pytest.approx(10.0)
    n_blocks = sum(len(v) for v in autotune.BLOCKS.values())
    assert calls == len(autotune.BINS) + autotune.N_STAGES * len(autotune.GRIDS) + n_blocks


def test_search_block_axis_per_stage():
    # only the fit stage's block size matters: the search finds it and leaves the others built-in
    def measure(nb, grid, block):
        return 1.0 + (0 if block[5] == 64 else 1) + 0.5 * sum(1 for g in grid if g) + \
            0.5 * sum(1 for k, b in enumerate(block) if b and k != 5)
    nb, grid, block, t, _ = autotune.search(measure)
    assert grid == [0] * autotune.N_STAGES and block == [0, 0, 0, 0, 0, 64] and t == 1.0


def test_search_keeps_builtin_when_nothing_is_better():
    # a cost that every explicit launch shape worsens: the built-in (0) stays
    def measure(nb, grid, block):
        return 1.0 + 0.5 * sum(1 for g in grid if g) + 0.5 * sum(1 for b in block if b) + \
            (0 if nb == 512 else 1)
    nb, grid, block, t, _ = autotune.search(measure)
    assert nb == 512 and grid == [0] * autotune.N_STAGES and block == [0] * autotune.N_STAGES
    assert t == 1.0


def test_cache_roundtrip_and_key(tmp_path):
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    Q = pxr.params_from(synth.params_phase1(), cut_mode=pxr.CUT_FP32)
    gpu = "NVIDIA GB300"
    k1 = autotune.cache_key(P, 256, 3_200_000, gpu)
    assert k1.startswith("NVIDIA_GB300-")
    assert k1 == autotune.cache_key(P, 256, 3_250_000, gpu)         # same size bucket
    assert k1 != autotune.cache_key(Q, 256, 3_200_000, gpu)         # other geometry
    assert k1 != autotune.cache_key(P, 64, 3_200_000, gpu)          # other batch size
    assert k1 != autotune.cache_key(P, 256, 3_200_000, "NVIDIA B200")   # other GPU
    # every parameter the tuner does not choose is in the hash; the tuned ones are not
    R = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32, pt_min=0.5)
    assert k1 != autotune.cache_key(R, 256, 3_200_000, gpu)
    S = autotune._with(P, 512, [1, 2, 3, 4, 5, 6], [256, 64, 0, 0, 0, 32])
    assert k1 == autotune.cache_key(S, 256, 3_200_000, gpu)
    path = str(tmp_path / "tune.json")
    autotune.store_cache(path, k1, {"n_phi_bins": 256, "grid_per_sm": [1, 2, 3, 4, 5, 6],
                                    "block_threads": [512, 128, 0, 0, 0, 64]})
    got = autotune.load_cache(path)[k1]
    assert got["grid_per_sm"] == [1, 2, 3, 4, 5, 6]
    assert got["block_threads"] == [512, 128, 0, 0, 0, 64]
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


def test_with_copies_and_sets_fields():
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    Q = autotune._with(P, 1024, [3, 0, 5, 0, 0, 7], [256, 128, 0, 0, 0, 32])
    assert Q.n_phi_bins == 1024 and list(Q.grid_per_sm) == [3, 0, 5, 0, 0, 7]
    assert list(Q.block_threads) == [256, 128, 0, 0, 0, 32]
    assert P.n_phi_bins == 0 and list(P.grid_per_sm) == [0] * 6
    assert list(P.block_threads) == [0] * 6
    assert Q.cos_phi_window == P.cos_phi_window and Q.n_pairs == P.n_pairs


def test_library_accepts_exactly_the_listed_block_sizes():
    """pxr_params_check takes every candidate of BLOCKS and 0, and rejects other sizes and a
    block size on a stage without a block axis (host-side check; no GPU)."""
    P = pxr.params_from(synth.params_barrel_quadruplets(), cut_mode=pxr.CUT_FP32)
    for k in range(autotune.N_STAGES):
        for t in autotune.BLOCKS.get(k, ()):
            block = [0] * 6
            block[k] = t
            pxr.pxr_params_check(autotune._with(P, 0, [0] * 6, block))
        for t in (16, 96, 2048) + ((256,) if k not in autotune.BLOCKS else ()):
            block = [0] * 6
            block[k] = t
            with pytest.raises(pxr.PxrError) as e:
                pxr.pxr_params_check(autotune._with(P, 0, [0] * 6, block))
            assert e.value.code == pxr.EINVAL and "block_threads" in str(e.value)


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
                        fit_mode=pxr.FIT_SPLIT)
    with pxr.Context(device=0, mem_budget_bytes=4 << 30) as ctx:
        cache = str(tmp_path / "tune.json")
        blocks = {0: (256,), 1: (64,), 5: (32,)}
        T, info = autotune.tune_plan(ctx, off, x, y, z, layer, P, reps=1, bins=(64, 1024),
                                     grids=(1, 32), blocks=blocks, cache=cache)
        assert info["trials"] == 2 + 6 * 2 + 3 and info["n_phi_bins"] in (64, 1024)
        assert info["gpu"] and info["key"] == autotune.cache_key(P, len(evs), int(off[-1]),
                                                                 info["gpu"])
        _, again = autotune.tune_plan(ctx, off, x, y, z, layer, P, cache=cache)
        assert again.get("cached") and again["grid_per_sm"] == info["grid_per_sm"]
        assert again["block_threads"] == info["block_threads"]
        # every non-default launch shape at once, against the built-in one
        F = autotune._with(P, 64, [1, 1, 1, 1, 1, 1], [256, 64, 0, 0, 0, 32])
        out = []
        for prm in (P, T, F):
            plan = pxr.Plan(ctx, off, x, y, z, layer, prm, use_graph=True)
            plan.pxr_plan_run()
            out.append([plan.pxr_plan_tracks(e) for e in range(len(evs))])
            plan.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            for k in pxr.TRACK_FIELDS:
                assert np.array_equal(a[k], b[k]), k
