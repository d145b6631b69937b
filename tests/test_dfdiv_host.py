"""The double-FP32 division used by the solver's scalar steps (csrc/dfdiv.h, Dekker's method) on the
host: the header compiles as plain C++ and, built without contraction (the device's IEEE FP32 operations
one rounding each), its quotients of seeded random pairs lie within 2^-44 of the exact quotient and exact
quotients stay exact (tests/native/dfdiv_main.cpp)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1710_09178_gb300", "csrc")


def test_double_fp32_division_on_host(tmp_path):
    exe = tmp_path / "dfdiv"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-Wall", "-Wextra", "-Werror", "-I" + CSRC,
                        os.path.join(ROOT, "tests", "native", "dfdiv_main.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
