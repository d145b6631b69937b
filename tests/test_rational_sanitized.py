"""Host sanitizers on the native rational-approximation code (Appendix): csrc/rational.cpp and a
driver (tests/native/rational_sanitized_main.cpp) built with AddressSanitizer and
UndefinedBehaviorSanitizer, any report fatal.  The driver computes the approximations of every
workload, checks signs and error bounds and the argument errors."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAGS = ["-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
         "-fno-omit-frame-pointer"]


def test_rational_code_is_clean_under_asan_and_ubsan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "rational_sanitized")
    build = subprocess.run([gxx, *FLAGS, "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "native", "rational_sanitized_main.cpp"),
                            os.path.join(ROOT, "paper_1710_09178_gb300", "csrc", "rational.cpp"), "-o", exe],
                           capture_output=True, text=True, timeout=300)
    if build.returncode != 0 and "sanitize" in build.stderr and "cannot find" in build.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "ALL OK" in run.stdout
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
