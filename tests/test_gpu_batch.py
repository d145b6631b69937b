"""mshift_cg_batch (independent problems solved concurrently) and lqcd_autotune.

Bars: every problem's outputs are bit-identical to a stand-alone mshift_cg call on the same
context (the reductions are deterministic); statuses are OK; the oracle's FP64 true residual of
the batched solutions is <= tol; the autotuned Dslash still matches the oracle.
"""
import numpy as np
import pytest

from gpu_util import make_context, rel_max, to_dev, gpu_dslash
from oracle import rational, solvers, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_batch_equals_individual_solves():
    import torch

    import paper_1710_09178_gb300 as lq

    lattices = [((4, 4, 4, 4), 0.1), ((10, 6, 4, 6), 0.05), ((8, 8, 8, 8), 0.02)]
    problems, owners, data = [], [], []
    for li, (dims, mass) in enumerate(lattices):
        owner, U = make_context(dims, mass, gauge_seed=50 + li)
        owners.append(owner)
        c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
        for f in range(2):
            ctx = lq.Context(dims, mass)
            ctx.share_gauge(owner)
            b = inputs.gaussian_vector(dims, 60 + 2 * li + f)
            bd = to_dev(b)
            xs = [torch.empty_like(bd) for _ in poles]
            y = torch.empty_like(bd)
            problems.append(dict(ctx=ctx, shifts=poles, residues=res, c0=c0, b=bd, xs=xs, y=y, tol=1e-10,
                                 prec=lq.FP32))
            data.append((dims, mass, U, b, poles))
    rc, st, stats = lq.mshift_cg_batch(problems, nthreads=4)
    torch.cuda.synchronize()
    assert rc == 0 and all(s == 0 for s in st)
    batched = [([x.cpu().numpy() for x in p["xs"]], p["y"].cpu().numpy()) for p in problems]
    # stand-alone solves on the same contexts give the same bits
    for p, (bx, by) in zip(problems, batched):
        rc1, _ = lq.mshift_cg(p["ctx"], p["shifts"], p["residues"], p["c0"], p["b"], p["xs"], p["y"], tol=1e-10,
                              prec=lq.FP32)
        torch.cuda.synchronize()
        assert rc1 == 0
        assert all(np.array_equal(x.cpu().numpy(), a) for x, a in zip(p["xs"], bx))
        assert np.array_equal(p["y"].cpu().numpy(), by)
    # the oracle's FP64 true residual of one batched problem per lattice
    for k in (0, 2, 4):
        dims, mass, U, b, poles = data[k]
        tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, batched[k][0], poles)
        assert np.all(tr <= 1.001e-10)


def test_batch_rejects_shared_context():
    import torch

    import paper_1710_09178_gb300 as lq

    ctx, U = make_context((4, 4, 4, 4), 0.1)
    b = to_dev(inputs.gaussian_vector((4, 4, 4, 4), 3))
    p = dict(ctx=ctx, shifts=[0.1], residues=[1.0], b=b)
    rc, st, _ = lq.mshift_cg_batch([p, dict(p)], raise_on_error=False)
    assert rc == lq.LQCD_ERR_ARG


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 16, 8)])
def test_autotune_keeps_parity(dims):
    import paper_1710_09178_gb300 as lq

    ctx, U = make_context(dims, 0.05, gauge_seed=70)
    best = ctx.autotune(lq.FP32)
    assert best in (1, 2, 4, 8)
    psi = inputs.gaussian_vector(dims, 71)
    for p in (0, 1):
        assert rel_max(gpu_dslash(ctx, psi, p, lq.FP32), staggered.dslash_eo(U, psi, dims, p)) < 2e-6
