"""Build libdhrs.so (all CUDA sources, sm_103a) in-tree with nvcc, and the
bounds-checked debug build libdhrs_debug.so (DHR_DEBUG).

    python -m paper_2406_06963_b300.build [--force] [--debug | --all]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libdhrs.so")
LIB_DEBUG = os.path.join(HERE, "libdhrs_debug.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
         "-Xptxas", "-warn-spills", "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "dhrs.h"), __file__]


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build the release library (or, with debug, the DHR_DEBUG one) unless it
    is newer than every source."""
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(f) <= t for f in _inputs()):
            return lib
    cmd = ["nvcc", *ARCH, *FLAGS, *(["-DDHR_DEBUG"] if debug else []), *sources(), "-o", lib]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    return lib


if __name__ == "__main__":
    force, verbose = "--force" in sys.argv, "-v" in sys.argv
    if "--all" in sys.argv:
        print(build(force, verbose))
        print(build(force, verbose, debug=True))
    else:
        print(build(force, verbose, debug="--debug" in sys.argv))
