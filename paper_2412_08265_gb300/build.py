"""Compile the CUDA library (sm_103a) in-tree: paper_2412_08265_gb300/_lib/librubix.so.

Each translation unit is compiled by its own nvcc process (in parallel) and the
objects are linked into one shared library with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "librubix.so")
# the bounds-checking build (RUBIX_DEBUG=1): computed shared-memory and record
# indices are checked against their buffers and reported in the device error
# word (kErrBounds) instead of faulting; built on request by the tests only
DEBUG_LIBDIR = os.path.join(HERE, "_lib_debug")
DEBUG_LIB = os.path.join(DEBUG_LIBDIR, "librubix.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["api.cu", "engine.cu", "serve.cu", "sort.cu", "setup.cu", "deposit.cu", "rows.cu", "psf_lsf.cu", "adjoint.cu", "adjoint_tiles.cu", "noalloc.cu", "selftest.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is compiled without floating-point contraction: the orientation
# matrix and the key coordinates are defined with every product and sum
# rounded once (no fused multiply-add), on x86 and Arm hosts alike.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _digest(extra=()) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "rubix.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile the library (debug=True: the bounds-checking build, in its own
    directory) and return the path of the shared object."""
    libdir, lib = (DEBUG_LIBDIR, DEBUG_LIB) if debug else (LIBDIR, LIB)
    extra = ["-DRUBIX_DEBUG=1"] if debug else []
    os.makedirs(libdir, exist_ok=True)
    stamp = os.path.join(libdir, "build.stamp")
    dig = _digest(extra)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == dig:
        return lib
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(libdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
