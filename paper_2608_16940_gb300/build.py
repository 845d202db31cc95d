"""Build libqsa.so in-tree for sm_103a with nvcc (no cmake).

Every translation unit under csrc/ is compiled in parallel into _build/ and
linked into paper_2608_16940_gb300/libqsa.so.  Rebuilds only what changed.
With --debug-bounds (debug_bounds=True) the same sources are compiled with
-DQSA_DEBUG_BOUNDS into _build_dbg/ and linked into libqsa_debug.so: the
state accesses of the main kernels are bounds-checked (qsa_bounds.cuh).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libqsa.so")
LIB_DEBUG = os.path.join(PKG, "libqsa_debug.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _headers_mtime() -> float:
    hs = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
          glob.glob(os.path.join(INCLUDE, "*.h")))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, obj: str, extra) -> None:
    cmd = [_nvcc()] + ARCH + COMMON + list(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")


def build(verbose: bool = False, extra=(), debug_bounds: bool = False) -> str:
    build_dir, lib = (BUILD + "_dbg", LIB_DEBUG) if debug_bounds else (BUILD, LIB)
    extra = list(extra) + (["-DQSA_DEBUG_BOUNDS"] if debug_bounds else [])
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = _headers_mtime()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s) + ".o")
        objs.append(o)
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append((s, o))
    if jobs:
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            list(ex.map(lambda so: _compile(so[0], so[1], extra), jobs))
    if jobs or not os.path.exists(lib):
        cmd = [_nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", lib] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(f"built {lib} ({len(jobs)} units recompiled)")
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    dbg = "--debug-bounds" in args
    build(verbose=True, extra=[a for a in args if a != "--debug-bounds"], debug_bounds=dbg)
