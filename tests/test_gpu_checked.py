"""The checked build (libpxr_checked.so, compiled with PXR_CHECKED): every index that a kernel
reads from another kernel's output, or computes from it (cell, edge and hit indices in the CA
passes, the walk, the selection, the canonical ordering and the fit), is compared with the extent
of its array before the access; a violation sets the event's F_BOUNDS flag and skips the access,
and the host reports PXR_EBOUNDS.  This is the debug form of race and bounds detection where no
sanitizer runs: on the parity workloads the checked library must report no violation and give
the same tracks, bit for bit, as the normal library.

Each library runs in a subprocess of its own (the binding loads one library per process, chosen
by the PXR_CHECKED environment variable).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workloads():
    from paper_2104_06573_gb300 import pxr, synth
    barrel, dense = synth.params_barrel_quadruplets(), synth.params_phase1()
    ev_b = synth.event_barrel(0)
    ev_d = synth.event_phase1(0)
    counts = synth.batch_track_counts(32)
    batch = [synth.make_event(e, counts[e]) for e in range(32)]
    yield "barrel_fp64", barrel, [ev_b], dict(cut_mode=pxr.CUT_FP64)
    yield "barrel_fp32", barrel, [ev_b], dict(cut_mode=pxr.CUT_FP32)
    yield "dense_fp64", dense, [ev_d], dict(cut_mode=pxr.CUT_FP64)
    yield "dense_fp32", dense, [ev_d], dict(cut_mode=pxr.CUT_FP32, fit_mode=pxr.FIT_SPLIT)
    yield "batch32", barrel, batch, dict(cut_mode=pxr.CUT_FP32, fit_mode=pxr.FIT_SPLIT,
                                         n_phi_bins=1024)


def _run(out_path):
    """Reconstruct every workload with the library this process loaded; save the tracks."""
    sys.path.insert(0, ROOT)
    import torch
    from paper_2104_06573_gb300 import pxr
    dev = torch.device("cuda:0")
    res = {"lib": np.array(os.path.basename(pxr.LIB_PATH))}
    with pxr.Context(device=0, mem_budget_bytes=16 << 30) as ctx:
        for name, P, evs, kw in _workloads():
            off = np.zeros(len(evs) + 1, np.uint32)
            off[1:] = np.cumsum([e.n for e in evs])
            cat = lambda k: np.concatenate([getattr(e, k) for e in evs])
            x = torch.from_numpy(cat("x")).to(dev)
            y = torch.from_numpy(cat("y")).to(dev)
            z = torch.from_numpy(cat("z")).to(dev)
            layer = torch.from_numpy(cat("layer").astype(np.uint16).view(np.int16)).to(dev)
            plan = pxr.Plan(ctx, off, x, y, z, layer, pxr.params_from(P, **kw), use_graph=True)
            plan.pxr_plan_run()
            cnt = plan.pxr_plan_counts()
            res[name + "/flags"] = np.asarray(cnt["flags"])
            for e in range(len(evs)):
                t = plan.pxr_plan_tracks(e)
                res[f"{name}/{e}/status"] = np.array(t["status"])
                for k in ("hit_idx", "n_hits", "pt", "phi", "cot_theta", "dxy", "dz", "chi2",
                          "charge"):
                    res[f"{name}/{e}/{k}"] = np.asarray(t[k])
            plan.close()
    np.savez(out_path, **res)


def _reconstruct(tmp_path, checked):
    out = tmp_path / ("checked.npz" if checked else "normal.npz")
    env = dict(os.environ, PXR_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--run", str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_library_exports_the_same_symbols():
    """Host-only: both variants are built and export every declared function."""
    import ctypes as C
    from paper_2104_06573_gb300 import build_lib, pxr
    build_lib.build()
    names = pxr.declared_functions()
    for lib in ("libpxr.so", "libpxr_checked.so"):
        L = C.CDLL(os.path.join(build_lib.OUT, lib))
        missing = [n for n in names if not hasattr(L, n)]
        assert not missing, (lib, missing)


@pytest.mark.gpu
def test_checked_build_finds_no_violation_and_equals_normal(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    chk = _reconstruct(tmp_path, True)
    ref = _reconstruct(tmp_path, False)
    assert str(chk["lib"]) == "libpxr_checked.so" and str(ref["lib"]) == "libpxr.so"
    keys = sorted(k for k in ref if k != "lib")
    assert keys == sorted(k for k in chk if k != "lib")
    for k in keys:
        if k.endswith("/flags"):
            assert not chk[k].any(), (k, chk[k])           # no F_BOUNDS (nor any other flag)
        if k.endswith("/status"):
            assert int(chk[k]) == 0, k
        assert np.array_equal(chk[k], ref[k], equal_nan=True), k


if __name__ == "__main__" and len(sys.argv) == 3 and sys.argv[1] == "--run":
    _run(sys.argv[2])
