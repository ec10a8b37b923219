"""Build of the in-tree CUDA library libeptv.so (sm_103a) with nvcc.

The library has a plain C ABI (include/eptv.h); no torch headers are involved, so it
is compiled directly with nvcc rather than as a torch extension."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libeptv.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(PKG, "csrc", "*.cuh"))) + \
        [os.path.join(ROOT, "include", "eptv.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps())


def _compile(args):
    subprocess.check_call(args)


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compiles every csrc/*.cu to an object in _build/ (in parallel: the translation units
    share no device code) and links them into libeptv.so."""
    if not force and up_to_date():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    obj_dir = os.path.join(PKG, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc")]
    if extra:
        flags += list(extra)
    tag = f".{os.getpid()}"
    jobs, objs = [], []
    for src in sources():
        obj = os.path.join(obj_dir, os.path.splitext(os.path.basename(src))[0] + tag + ".o")
        objs.append(obj)
        jobs.append([nvcc, *flags, "-c", src, "-o", obj])
    if verbose:
        for j in jobs:
            print(" ".join(j), file=sys.stderr)
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    try:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(_compile, jobs))
        tmp = LIB + f"{tag}.tmp"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
