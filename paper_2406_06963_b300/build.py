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
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
         "-Xptxas", "-warn-spills", "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]
OBJ_DIR = os.path.join(HERE, "_build")   # per-source objects (git-ignored)


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
    # every source compiles to its own object in parallel (each translation
    # unit carries its own device code), then one link
    from concurrent.futures import ThreadPoolExecutor
    tag = "debug" if debug else "release"
    os.makedirs(OBJ_DIR, exist_ok=True)
    extra = (["-DDHR_DEBUG"] if debug else []) + (["-Xptxas=-v"] if verbose else [])
    objs = [os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + "." + tag + ".o") for src in sources()]

    def compile_one(src_obj):
        src, obj = src_obj
        return subprocess.run(["nvcc", *ARCH, *FLAGS, *extra, "-c", src, "-o", obj], capture_output=True, text=True)

    with ThreadPoolExecutor(max_workers=max(1, min(len(objs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, zip(sources(), objs)))
    for src, r in zip(sources(), results):
        if r.stdout or r.stderr:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise subprocess.CalledProcessError(r.returncode, "nvcc " + src)
    subprocess.run(["nvcc", *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", lib], check=True)
    return lib


if __name__ == "__main__":
    force, verbose = "--force" in sys.argv, "-v" in sys.argv
    if "--all" in sys.argv:
        print(build(force, verbose))
        print(build(force, verbose, debug=True))
    else:
        print(build(force, verbose, debug="--debug" in sys.argv))
