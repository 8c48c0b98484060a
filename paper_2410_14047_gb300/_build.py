"""Builds the CUDA library (sm_103a) in-tree next to this file.

Two variants of the same sources: _libdifuser_im.so (the library) and
_libdifuser_im_bounds.so, compiled with IM_BOUNDS_CHECK: every checked device
index (vertex ids, edge and list offsets, bucket ids, queue entries) is tested
against its range, and a bad one raises an error bit the host reports as
IM_E_STATE instead of touching memory out of range.  The bounds-checked
variant is for tests on small cases; it is slower.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "_libdifuser_im.so")
BOUNDS_LIB = os.path.join(HERE, "_libdifuser_im_bounds.so")
SOURCES = ["im_kernels.cu", "im_frontier.cu", "im_api.cu", "im_noalloc.cu", "im_server.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("im_device.cuh", "im_launch.h", "im_internal.h")] + [
    os.path.join(ROOT, "include", "difuser_im.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-pthread"]
# variant name -> (library path, object directory, extra flags)
VARIANTS = {
    "": (LIB, os.path.join(HERE, "_build"), []),
    "bounds": (BOUNDS_LIB, os.path.join(HERE, "_build_bounds"), ["-DIM_BOUNDS_CHECK"]),
}


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps)


def build_variants(variants=("",), force: bool = False, verbose: bool = False) -> list:
    """Compile every translation unit of the stale variants in parallel, then
    link each variant's shared library."""
    todo = [v for v in variants if force or _stale(VARIANTS[v][0])]
    procs = []
    for v in todo:
        lib, objdir, extra = VARIANTS[v]
        os.makedirs(objdir, exist_ok=True)
        for s in SOURCES:
            obj = os.path.join(objdir, s.replace(".cu", ".o"))
            cmd = [NVCC, *FLAGS, *extra, "-c", os.path.join(CSRC, s), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
    for v in todo:
        lib, objdir, _ = VARIANTS[v]
        objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler", "-pthread", "-o",
               tmp, *objs]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
        os.replace(tmp, lib)
    return [VARIANTS[v][0] for v in variants]


def build(force: bool = False, verbose: bool = False) -> str:
    """The library itself (the normal variant)."""
    return build_variants(("",), force, verbose)[0]


def build_bounds(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checked variant."""
    return build_variants(("bounds",), force, verbose)[0]


if __name__ == "__main__":
    print(build_variants(("", "bounds"), force="--force" in sys.argv, verbose=True))
