"""Build the sm_103a TENO-AA shared library in-tree with nvcc.

Every translation unit is compiled in parallel (one -gencode, no FMA
contraction: the arithmetic order of each expression is fixed by the source),
then linked into paper_2109_14340_gb300/_build/libteno_gb300.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libteno_gb300.so")
DEBUG_LIB = os.path.join(BUILD, "libteno_gb300_debug.so")   # -DTENO_DEBUG_BOUNDS
PROBE_LIB = os.path.join(BUILD, "libteno_probe.so")
PROBE_SRC = os.path.join(PKG, "probe", "fp64_probe.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _nvcc() -> str:
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nv):
        raise RuntimeError("nvcc not found: the TENO-AA CUDA library cannot be built")
    return nv


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime():
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC)
          if f.endswith((".cu", ".cuh", ".h"))]
    ts.append(os.path.getmtime(os.path.join(ROOT, "include", "teno.h")))
    ts.append(os.path.getmtime(__file__))
    return max(ts)


def build_probe(force: bool = False) -> str:
    """The FP64 peak probe library (measurement only, not the product path)."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(PROBE_LIB) and \
            os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    tmp = PROBE_LIB + ".%d.tmp" % os.getpid()
    cmd = [_nvcc()] + ARCH + FLAGS + ["-shared", PROBE_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for the probe:\n%s" % r.stderr)
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libteno_gb300.so, or with debug=True the bounds-checked
    libteno_gb300_debug.so (the same sources with -DTENO_DEBUG_BOUNDS)."""
    lib = DEBUG_LIB if debug else LIB
    odir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(odir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    nv = _nvcc()
    objs = []
    extra = ["-DTENO_DEBUG_BOUNDS"] if debug else []

    def compile_one(src):
        obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
        cmd = [nv] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_probe(force=True))
