"""Compiles the CUDA library liblsmc.so in-tree (sm_103a only).

Each translation unit of csrc/ is compiled by nvcc in parallel, then linked
into paper_2206_03719_gb300/_build/liblsmc.so with the CUDA runtime linked
statically.  No cmake, no torch extension machinery.

build(checked=True) makes the checked build instead, in _build_checked/:
the same sources compiled with LSMC_CHECKED, whose kernels test every
global-memory access against the byte ranges of their launch and record
the first one outside them (lsmc_check_report) -- the library's own bounds
checker, for tests on small cases.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
BUILD_DIR = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblsmc.so")
CHECKED_DIR = os.path.join(_HERE, "_build_checked")
CHECKED_LIB_PATH = os.path.join(CHECKED_DIR, "liblsmc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-I" + _INCLUDE, "-I" + _CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblsmc.so")


def _sources():
    return sorted(glob.glob(os.path.join(_CSRC, "*.cu")) + glob.glob(os.path.join(_CSRC, "*.cpp")))


def _fingerprint(flags) -> str:
    h = hashlib.sha256()
    files = _sources() + sorted(glob.glob(os.path.join(_CSRC, "*.h")) +
                                glob.glob(os.path.join(_CSRC, "*.cuh")) +
                                glob.glob(os.path.join(_INCLUDE, "*.h")))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile liblsmc.so (or its checked build) if missing or stale; returns
    its path."""
    build_dir, lib_path = (CHECKED_DIR, CHECKED_LIB_PATH) if checked else (BUILD_DIR, LIB_PATH)
    flags = NVCC_FLAGS + (["-DLSMC_CHECKED"] if checked else [])
    fp = _fingerprint(flags)
    stamp = os.path.join(build_dir, "liblsmc.fingerprint")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(fp)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
