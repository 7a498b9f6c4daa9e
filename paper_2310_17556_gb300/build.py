"""Build libdfs.so in-tree with nvcc for sm_103a (GB300).

Every .cu file under csrc/ is compiled to an object in parallel, then linked into
``paper_2310_17556_gb300/libdfs.so``.  ``--debug-bounds`` builds the same sources with
-DDFS_DEBUG_BOUNDS (device index checks that record DFS_ERR_BOUNDS instead of faulting) into
``libdfs_debug.so``, in its own object folder; the binding loads it when the environment variable
DFS_DEBUG_BOUNDS is set to 1.  No CMake, no torch extension machinery: the C ABI
in include/dfs.h is the boundary, and the Python binding loads the library with ctypes.

    python -m paper_2310_17556_gb300.build [--force] [--debug-bounds]
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdfs.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libdfs_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdfs")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, debug_bounds: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source and link libdfs.so (libdfs_debug.so with debug_bounds); returns
    the library path."""
    lib, build_dir = (LIB_DEBUG, BUILD_DEBUG) if debug_bounds else (LIB, BUILD)
    os.makedirs(build_dir, exist_ok=True)
    deps = _deps() + [os.path.abspath(__file__)]
    if not force and not _stale(lib, deps):
        return lib
    extra = ["-DDFS_DEBUG_BOUNDS"] if debug_bounds else []
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--debug-bounds", action="store_true")
    a = ap.parse_args()
    build(force=a.force, debug_bounds=a.debug_bounds, verbose=True)
    sys.exit(0)
