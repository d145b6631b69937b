"""Build the C++ oracle (test infrastructure) into two shared libraries beside its source.

  liborc.so      one core (no OpenMP)
  liborc_omp.so  the same source with OpenMP over the site loops

Plain g++ (C++17, -O2, no -march flags, no floating-point contraction), so the x86 and Arm
builds compute the same operations in the same order.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIBS = {"serial": os.path.join(HERE, "liborc.so"), "omp": os.path.join(HERE, "liborc_omp.so")}
FLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _stale(lib: str) -> bool:
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(SRC), os.path.getmtime(__file__))


def build(force: bool = False) -> dict:
    """Compile both libraries when missing or older than the source; returns their paths."""
    for kind, lib in LIBS.items():
        if not force and not _stale(lib):
            continue
        extra = ["-fopenmp"] if kind == "omp" else ["-Wno-unknown-pragmas"]
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run(["g++", *FLAGS, *extra, SRC, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, lib)
    return dict(LIBS)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
