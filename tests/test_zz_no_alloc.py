"""lqcd_apply_A_noalloc: the allocation-free variant of lqcd_apply_A.

It exists for callers that must not allocate device memory when they call it (memory
owned by a framework allocator or a fixed budget, or loops that cannot afford the device
synchronisation of cudaMalloc/cudaFree).  Its scratch is a static array inside the
library.  The tests call it through the C ABI and compare it with lqcd_apply_A, which
allocates its scratch, on two calls in a row (the second call reuses the array the
first one left behind), and check that an oversized lattice is refused.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


def _setup(dims, mass):
    import torch

    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import build, inputs

    build.build()
    ctx = lq.Context(dims, mass)
    ctx.set_gauge(torch.from_numpy(inputs.gauge_field(dims, seed=12)).cuda())
    return lq, ctx, inputs


@pytest.mark.parametrize("dims", [(10, 6, 4, 6), (16, 16, 16, 8)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 2e-6)])
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
    ctx = lq.Context((32, 32, 32, 12), 0.05)  # V/2 = 196608 > 173392: FP64 temporary does not fit
    q = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = lib.lqcd_apply_A_noalloc(ctx.handle, q.data_ptr(), p.data_ptr(), 0.0, FP64, None)
    assert rc == lq.LQCD_ERR_ARG
    assert b"static scratch" in lib.lqcd_last_error(ctx.handle)
