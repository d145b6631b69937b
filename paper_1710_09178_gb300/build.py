"""Build liblqcd.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
paper_1710_09178_gb300/liblqcd.so.  No cmake, no setuptools: plain nvcc and g++.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblqcd.so")
# the debug build: every computed neighbour address checked on the device (csrc/bounds.h)
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "liblqcd_debug.so")

CU_SOURCES = ["capi.cu", "pack.cu", "dslash.cu", "solver.cu", "mrhs.cu", "force.cu", "trajectory.cu", "batch.cu", "noalloc.cu", "df64.cu"]
CPP_SOURCES = ["rational.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-I" + INCLUDE]


def nvcc_path() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblqcd.so")
    return p


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lqcd.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile and link liblqcd.so (debug=True: liblqcd_debug.so, with the device-side neighbour-index
    checks); returns its path.  Skips the work when up to date."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and not ptxas_info and not _sources_newer_than(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = nvcc_path()
    defs = ["-DLQCD_DEBUG_BOUNDS"] if debug else []
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(bdir, src + ".o")
        extra = ["-Xptxas", "-v"] if ptxas_info else []
        jobs.append([nvcc, *ARCH, *NVCC_FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(bdir, src + ".o")
        jobs.append(["g++", *CXX_FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(os.cpu_count() or 8, len(jobs))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o, file=sys.stderr)
    objs = [os.path.join(bdir, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    tmp = lib + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug="--debug" in sys.argv))
