"""Host-side checks of the C ABI: the library builds and loads, exports every function that
include/pxr.h declares, its structs have the layout the binding assumes, and the host-only
entry points behave (no GPU needed)."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_06573_gb300 import build_lib, pxr
    build_lib.build()
    return pxr.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2104_06573_gb300 import pxr
    names = pxr.declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(lib, tmp_path):
    from paper_2104_06573_gb300 import pxr
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pxr.h"', "int main(void){"]
    for cname, cls in (("pxr_params", pxr.pxr_params), ("pxr_config", pxr.pxr_config),
                       ("pxr_tracks", pxr.pxr_tracks)):
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _t in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    for cname, cls in (("pxr_params", pxr.pxr_params), ("pxr_config", pxr.pxr_config),
                       ("pxr_tracks", pxr.pxr_tracks)):
        assert table[(cname, "sizeof")] == C.sizeof(cls), cname
        for f, _t in cls._fields_:
            assert table[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_presets_match_workload_definitions(lib):
    from paper_2104_06573_gb300 import pxr, synth
    for preset, ref in ((pxr.PRESET_BARREL, synth.params_barrel_quadruplets()),
                        (pxr.PRESET_PHASE1, synth.params_phase1())):
        got = pxr.pxr_params_init(preset)
        want = pxr.params_from(ref)
        assert bytes(got) == bytes(want), preset


def test_version_and_errors_without_gpu(lib):
    from paper_2104_06573_gb300 import pxr
    assert "sm_103a" in pxr.pxr_version()
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: context creation is covered by the GPU tests")
    with pytest.raises(pxr.PxrError) as ei:
        pxr.Context(device=0)
    assert ei.value.code == pxr.ECUDA


def test_params_validation(lib):
    """Parameter validation runs on the host, before any device work."""
    from paper_2104_06573_gb300 import pxr, synth
    p = pxr.params_from(synth.params_barrel_quadruplets())
    bad = []
    for field, val in (("min_hits", 1), ("max_hits", 7), ("cut_mode", 5), ("fit_mode", 9),
                       ("phi_window", 0.0), ("cos_phi_window", 0.5), ("dca_cut", -1.0),
                       ("n_phi_bins", 17), ("n_layers", 0)):
        q = pxr.pxr_params()
        C.memmove(C.addressof(q), C.addressof(p), C.sizeof(p))
        setattr(q, field, val)
        bad.append(lib.pxr_params_check(C.byref(q)))
    assert all(rc == pxr.EINVAL for rc in bad), bad
    assert lib.pxr_params_check(C.byref(p)) == pxr.OK
    q = pxr.params_from(synth.params_phase1())
    q.pair_outer[0] = q.pair_inner[0]                    # inner == outer
    assert lib.pxr_params_check(C.byref(q)) == pxr.EINVAL
    # layer pairs that form a cycle (3 -> 0 closes 0 -> 1 -> 2 -> 3) have no CA level order
    q = pxr.params_from(synth.params_barrel_quadruplets())
    q.pair_inner[q.n_pairs], q.pair_outer[q.n_pairs] = 3, 0
    q.n_pairs += 1
    assert lib.pxr_params_check(C.byref(q)) == pxr.EINVAL
    for k, v in ((0, 65), (5, 100)):                     # grid caps above 64 CTAs per SM
        q = pxr.params_from(synth.params_barrel_quadruplets())
        q.grid_per_sm[k] = v
        assert lib.pxr_params_check(C.byref(q)) == pxr.EINVAL
    # the optional steps after the fit
    for kw in (dict(pt_min=-1.0), dict(pt_min=float("nan")), dict(chi2_max=-0.5),
               dict(chi2_max=float("inf")), dict(vertexing=True, vtx_min_tracks=1),
               dict(vertexing=True, vtx_gap=0.0), dict(vertexing=True, vtx_gap=float("nan"))):
        q = pxr.params_from(synth.params_barrel_quadruplets(), **kw)
        assert lib.pxr_params_check(C.byref(q)) == pxr.EINVAL, kw
    for field, val in (("clean_shared", 2), ("fit_cov", 2), ("vertexing", 3), ("fit_mode", 5)):
        q = pxr.params_from(synth.params_barrel_quadruplets())
        setattr(q, field, val)
        assert lib.pxr_params_check(C.byref(q)) == pxr.EINVAL, field
    for kw in (dict(pt_min=0.9, chi2_max=10.0, clean_shared=True), dict(fit_cov=True),
               dict(vertexing=True), dict(fit_mode=pxr.FIT_RIEMANN)):
        q = pxr.params_from(synth.params_barrel_quadruplets(), **kw)
        assert lib.pxr_params_check(C.byref(q)) == pxr.OK, kw


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """The product path has no fallback: a missing library raises."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2104_06573_gb300 import pxr\n"
            "pxr.LIB_PATH = %r\n"
            "try:\n    pxr.load()\nexcept RuntimeError as e:\n    print('raised')\n")
    r = subprocess.run([sys.executable, "-c", code % (ROOT, str(tmp_path / "nope.so"))],
                       capture_output=True, text=True)
    assert "raised" in r.stdout, r.stdout + r.stderr
