"""Build libperm.so in-tree with nvcc for sm_103a (no CMake, no torch extension machinery).

Each ``csrc/*.cu`` file is compiled to an object in parallel, then linked into
``paper_2510_03421_gb300/libperm.so`` with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libperm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _digest(path: str, extra: str) -> str:
    h = hashlib.sha1(extra.encode())
    with open(path, "rb") as f:
        h.update(f.read())
    for hp in _headers():
        with open(hp, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _compile(src: str, extra_flags) -> str:
    flags = NVCC_FLAGS + ARCH + list(extra_flags)
    key = _digest(src, " ".join(flags) + os.uname().machine)
    obj = os.path.join(BUILD, "%s.%s.o" % (os.path.basename(src)[:-3], key))
    if not os.path.exists(obj):
        tmp = obj + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc()] + flags + ["-c", src, "-o", tmp])
        os.replace(tmp, obj)
    return obj


def build(verbose: bool = False, extra_flags=(), jobs: int | None = None) -> str:
    """Compile every CUDA source and link libperm.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra_flags), srcs))
    for old in glob.glob(os.path.join(BUILD, "*.o")):  # objects of earlier source versions
        if old not in objs:
            os.remove(old)
    stamp = hashlib.sha1("".join(objs).encode()).hexdigest()[:16]
    stamp_file = os.path.join(BUILD, "libperm.stamp")
    if os.path.exists(LIB) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
