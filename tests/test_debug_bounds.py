"""The debug build's device-side neighbour-index checks.

CPU: the predicate the checks use (csrc/bounds.h) rejects every address outside the lattice and
accepts every address inside it (tests/native/bounds_main.cpp compiled with g++); the release
library reports that it has no checks.  GPU: the debug build (liblqcd_debug.so) runs the
half-lattice hop in every link format, the A-apply and converged shifted-CG solves (main solve,
double-FP32 checks, multi-RHS refinement) and the fermion force on valid lattices, with results
equal to the release build's and an error word that stays 0.  No GPU run is given a bad geometry:
out-of-range addresses are exercised on the host only.
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1710_09178_gb300", "csrc")


def test_bounds_predicate_on_host(tmp_path):
    exe = tmp_path / "bounds"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror", "-I" + CSRC,
                        os.path.join(ROOT, "tests", "native", "bounds_main.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_release_library_has_no_bounds_word():
    import ctypes

    import paper_1710_09178_gb300 as lq

    lib = lq.load_library()
    h = ctypes.c_void_p()
    assert lib.lqcd_create(ctypes.byref(h), (ctypes.c_int * 4)(4, 4, 4, 4), 0.1, None) == lq.LQCD_OK
    w = ctypes.c_uint(7)
    assert lib.lqcd_bounds_word(h, ctypes.byref(w)) == lq.LQCD_ERR_STATE and w.value == 0
    assert b"debug build" in lib.lqcd_last_error(h)
    assert lib.lqcd_destroy(h) == lq.LQCD_OK


@pytest.mark.gpu
@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((10, 6, 4, 6), 0.05), ((16, 16, 16, 8), 0.05)])
def test_debug_build_runs_clean_on_valid_lattices(dims, mass):
    import ctypes

    import torch

    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import build, inputs

    build.build(debug=True)
    dbg = lq.load_debug_library()
    U = torch.from_numpy(inputs.gauge_field(dims, seed=21)).cuda()
    psi = torch.from_numpy(inputs.gaussian_vector(dims, 22)).cuda()
    c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * mass ** 2, 16 + 4 * mass ** 2, 8)
    outs = {}
    for name, lib in (("release", lq.load_library()), ("debug", dbg)):
        ctx = lq.Context(dims, mass, lib=lib)
        ctx.set_gauge(U)
        got = []
        for prec in (lq.FP64, lq.FP32, lq.FP32_R12, lq.FP32_R8, lq.FP32_L16, lq.DF64):
            vin, vout, vq = ctx.new_vector(prec), ctx.new_vector(prec), ctx.new_vector(prec)
            ctx.pack(vin, prec, psi)
            lq.dslash_eo(ctx, vout, vin, 1, prec)
            ctx.apply_A(vq, vin, 0.3, prec)
            got += [vout.clone(), vq.clone()]
        for prec in (lq.FP32, lq.FP64):
            xs = [torch.empty_like(psi) for _ in poles]
            rc, st = lq.mshift_cg(ctx, poles, res, c0, psi, xs, None, tol=1e-10, prec=prec)
            assert rc == 0
            got += [x.clone() for x in xs]
        Fa = torch.empty((int(np.prod(dims)), 4, 8), dtype=torch.float64, device="cuda")
        rc, S, _ = lq.fermion_force(ctx, poles, res, c0, psi, Falg=Fa, tol=1e-10, prec=lq.FP64)
        assert rc == 0
        got.append(Fa.clone())
        if name == "debug":
            word = ctypes.c_uint(123)
            assert dbg.lqcd_bounds_word(ctx.handle, ctypes.byref(word)) == lq.LQCD_OK
            assert word.value == 0
        torch.cuda.synchronize()
        outs[name] = got
        ctx.close()
    # the checks change no result
    for a, b in zip(outs["release"], outs["debug"]):
        assert torch.equal(a, b)
