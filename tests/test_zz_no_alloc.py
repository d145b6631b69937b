"""lqcd_apply_A_noalloc: the allocation-free variant of lqcd_apply_A.

It exists for callers that must not allocate device memory when they call it (memory
owned by a framework allocator or a fixed budget, or loops that cannot afford the device
synchronisation of cudaMalloc/cudaFree).  Its scratch is a static array inside the
library.  The tests call it through the C ABI and compare it with lqcd_apply_A, which
allocates its scratch, on two calls in a row (the second call reuses the array the
first one left behind) in every precision it accepts; compare its 12-real result with the
oracle's A at 16^3 x 8; run it with 8 threads per site on the largest lattice class its
scratch admits; and check that an oversized lattice and an unsupported precision are refused.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64, FP32, FP32_R12, FP32_R8, FP32_L16, DF64 = 0, 1, 2, 4, 5, 6
OPT_DSLASH_TPS = 5


def _setup(dims, mass):
    import torch

    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import build, inputs

    build.build()
    ctx = lq.Context(dims, mass)
    ctx.set_gauge(torch.from_numpy(inputs.gauge_field(dims, seed=12)).cuda())
    return lq, ctx, inputs


@pytest.mark.parametrize("dims", [(10, 6, 4, 6), (16, 16, 16, 8)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 2e-6), (FP32_R12, 2e-6), (FP32_R8, 2e-6),
                                      (FP32_L16, 2e-6)])
def test_noalloc_matches_apply_A_on_two_calls(dims, prec, tol):
    import torch

    lq, ctx, inputs = _setup(dims, 0.05)
    lib = lq.load_library()
    for call, (seed, sigma) in enumerate([(51, 0.0), (52, 0.37)]):
        psi = torch.from_numpy(inputs.gaussian_vector(dims, seed)).cuda()
        p = ctx.new_vector(prec)
        ctx.pack(p, prec, psi)
        q_ref = ctx.new_vector(prec)
        q_new = ctx.new_vector(prec)
        q_new.fill_(0xFF)  # NaN pattern: every element must be written
        pq_ref = ctx.apply_A(q_ref, p, sigma, prec, want_dot=True)
        pq_new = ctypes.c_double(0.0)
        rc = lib.lqcd_apply_A_noalloc(ctx.handle, q_new.data_ptr(), p.data_ptr(), sigma, prec, ctypes.byref(pq_new))
        assert rc == 0, lib.lqcd_last_error(ctx.handle)
        a = torch.empty_like(psi)
        b = torch.empty_like(psi)
        ctx.unpack(a, q_ref, prec)
        ctx.unpack(b, q_new, prec)
        torch.cuda.synchronize()
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(a)), f"call {call}"
        assert abs(pq_new.value - pq_ref) <= tol * abs(pq_ref), f"call {call}"


def test_noalloc_refuses_lattice_beyond_static_scratch():
    import torch

    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import build

    build.build()
    lib = lq.load_library()
    ctx = lq.Context((32, 32, 32, 12), 0.05)  # V/2 = 196608 > 170661: FP64 temporary does not fit
    q = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = lib.lqcd_apply_A_noalloc(ctx.handle, q.data_ptr(), p.data_ptr(), 0.0, FP64, None)
    assert rc == lq.LQCD_ERR_ARG
    assert b"static scratch" in lib.lqcd_last_error(ctx.handle)


def test_noalloc_r12_matches_oracle_16c8():
    # 12-real FP32 links, element by element against the FP64 oracle's (A + sigma) p (Section 3.2)
    import torch

    from oracle import staggered

    dims, mass, sigma = (16, 16, 16, 8), 0.05, 0.21
    lq, ctx, inputs = _setup(dims, mass)
    lib = lq.load_library()
    U = inputs.gauge_field(dims, seed=12)
    psi = inputs.gaussian_vector(dims, 61)
    p = ctx.new_vector(FP32_R12)
    ctx.pack(p, FP32_R12, torch.from_numpy(psi).cuda())
    q = ctx.new_vector(FP32_R12)
    pq = ctypes.c_double(0.0)
    rc = lib.lqcd_apply_A_noalloc(ctx.handle, q.data_ptr(), p.data_ptr(), sigma, FP32_R12, ctypes.byref(pq))
    assert rc == 0, lib.lqcd_last_error(ctx.handle)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    ctx.unpack(out, q, FP32_R12)
    got = out.cpu().numpy()
    # the oracle sees the FP32-rounded input the kernel sees
    psi32 = psi.real.astype(np.float32).astype(np.float64) + 1j * psi.imag.astype(np.float32).astype(np.float64)
    ref = staggered.A_apply(U, psi32, mass, dims, sigma)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    dot = float(np.real(np.vdot(psi32, ref)))
    assert abs(pq.value - dot) <= 2e-6 * abs(dot)


def test_noalloc_eight_threads_per_site_at_40c8():
    # 40^3 x 8 (V/2 = 256000) in FP32 with 8 threads per output site: 16000 thread blocks, all with
    # a partial-sum slot of the static scratch; the result equals lqcd_apply_A's
    import torch

    dims = (40, 40, 40, 8)
    lq, ctx, inputs = _setup(dims, 0.02)
    lib = lq.load_library()
    ctx.set_option(OPT_DSLASH_TPS, 8)
    psi = torch.from_numpy(inputs.gaussian_vector(dims, 71)).cuda()
    p = ctx.new_vector(FP32)
    ctx.pack(p, FP32, psi)
    q_ref, q_new = ctx.new_vector(FP32), ctx.new_vector(FP32)
    pq_ref = ctx.apply_A(q_ref, p, 0.0, FP32, want_dot=True)
    pq_new = ctypes.c_double(0.0)
    rc = lib.lqcd_apply_A_noalloc(ctx.handle, q_new.data_ptr(), p.data_ptr(), 0.0, FP32, ctypes.byref(pq_new))
    assert rc == 0, lib.lqcd_last_error(ctx.handle)
    torch.cuda.synchronize()
    assert torch.equal(q_ref, q_new)
    assert pq_new.value == pq_ref


def test_noalloc_refuses_double_fp32():
    import torch

    lq, ctx, inputs = _setup((4, 4, 4, 4), 0.1)
    lib = lq.load_library()
    q = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = lib.lqcd_apply_A_noalloc(ctx.handle, q.data_ptr(), p.data_ptr(), 0.0, DF64, None)
    assert rc == lq.LQCD_ERR_ARG
    assert b"LQCD_FP32_L16" in lib.lqcd_last_error(ctx.handle)
