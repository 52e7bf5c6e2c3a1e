"""Builds the in-tree CUDA library libmhd_b300.so for sm_103a with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmhd_b300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared"]
LIBS = ["-lcufft"]  # the FFT of the magnetic spectrum (a plain library transform)


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


COMPILE_FLAGS = [f for f in NVCC_FLAGS if f != "-shared"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ (one nvcc per file, in parallel) and link
    them into one shared library (atomic replace)."""
    if not force and not stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(CSRC, os.path.basename(src)[:-3] + tag + ".o") for src in sources()]
    cmds = [["nvcc", *COMPILE_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj] for src, obj in zip(sources(), objs)]
    link = ["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", LIB + tag, *objs, *LIBS]
    try:
        with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
            for cmd in cmds:
                if verbose:
                    print(" ".join(cmd))
            for f in [ex.submit(subprocess.check_call, cmd) for cmd in cmds]:
                f.result()
        if verbose:
            print(" ".join(link))
        subprocess.check_call(link)
        os.replace(LIB + tag, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
