"""Build of the pxr CUDA library (sm_103a only), in-tree: paper_2104_06573_gb300/_build/libpxr.so,
and its checked variant libpxr_checked.so (compiled with PXR_CHECKED: device-side bounds checks
that set an error flag and skip the access, for debugging and the race/bounds tests).

Each translation unit is compiled by nvcc in parallel (both variants at once), then linked into
one shared library per variant with the CUDA runtime linked statically (no dependence on the
runtime library search path).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpxr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


VARIANTS = (("libpxr.so", "", []), ("libpxr_checked.so", "checked", ["-DPXR_CHECKED"]))


def build(force: bool = False, verbose: bool = False, extra=(), variants=VARIANTS) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "pxr.h"))
    srcs = sources()
    jobs = []                                   # (source, object, flags) of every variant
    libs = []                                   # (library, objects)
    for lib, sub, flags in variants:
        d = os.path.join(OUT, sub) if sub else OUT
        os.makedirs(d, exist_ok=True)
        objs = [os.path.join(d, os.path.basename(s)[:-3] + ".o") for s in srcs]
        jobs += [(s, o, flags) for s, o in zip(srcs, objs)]
        libs.append((os.path.join(OUT, lib), objs))

    def compile_one(job):
        src, obj, flags = job
        if not force and not _stale(obj, [src] + headers):
            return ""
        cmd = [nvcc, *ARCH, *FLAGS, *flags, *extra, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(compile_one, jobs))
    if verbose:
        for l in logs:
            if l:
                print(l)
    for lib, objs in libs:
        if force or _stale(lib, objs):
            tmp = lib + f".{os.getpid()}.tmp"
            cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
