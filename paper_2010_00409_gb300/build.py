"""Build the CUDA library libpsatd.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit under csrc/ compiles in parallel; the objects link into
paper_2010_00409_gb300/libpsatd.so with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build", "psatd")
LIB = os.path.join(HERE, "libpsatd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-O3"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stamp() -> str:
    h = hashlib.sha256()
    for f in _sources() + _headers() + [__file__]:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _compile(src: str, extra, bdir: str = BUILD) -> str:
    obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


DEBUG_LIB = os.path.join(HERE, "libpsatd_debug.so")


def build_library(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile csrc/*.cu and link libpsatd.so; skipped when sources are unchanged.

    debug=True builds libpsatd_debug.so with -DPSATD_DEBUG: every instrumented
    global index is bounds-checked (psatd_debug_bounds_report)."""
    lib = DEBUG_LIB if debug else LIB
    bdir = BUILD + ("_debug" if debug else "")
    extra = tuple(extra) + (("-DPSATD_DEBUG",) if debug else ())
    os.makedirs(bdir, exist_ok=True)
    stamp_file = os.path.join(bdir, "stamp")
    stamp = _stamp() + repr(tuple(extra))
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        if open(stamp_file).read() == stamp:
            return lib
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, bdir), srcs))
    LIB_ = lib
    tmp = LIB_ + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB_)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    if verbose:
        print("built", LIB_, file=sys.stderr)
    return LIB_


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv)
