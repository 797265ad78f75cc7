"""Build the CUDA library ``liblz.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` is compiled to an object in parallel (one ``-gencode``,
``-lineinfo``), then linked into ``paper_2304_07342_gb300/liblz.so`` against
the shared CUDA runtime.  Rebuilds only when a source or header is newer
than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblz.so")
# the bounds-checked variant (-DLZ_CHECKED: computed shared/global indices
# checked, violations reported as LZ_ERR_INTERNAL), built only on request
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "liblz_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.h")) +
            [os.path.join(ROOT, "include", "lz.h"), __file__])


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD_CHECKED if checked else BUILD
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        log = obj + ".log"
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DLZ_CHECKED"] if checked else []), "-Xptxas", "-v",
               "-c", src, "-o", obj]
        procs.append((src, log, subprocess.Popen(
            cmd, stdout=open(log, "w"), stderr=subprocess.STDOUT)))
    failed = []
    for src, log, p in procs:
        if p.wait() != 0:
            failed.append((src, open(log).read()))
    if failed:
        msg = "\n".join(f"--- {s}\n{l}" for s, l in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    if verbose:
        for _, log, _ in procs:
            sys.stdout.write(open(log).read())
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
