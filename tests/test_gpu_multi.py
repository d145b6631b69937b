"""mshift_cg_multi: the shifted CG of several right-hand sides of one lattice at once (the
pseudofermions of one gauge field in the batched workload; the paper solves one source at a time).

Bars: every system's solutions, y and statistics equal those of mshift_cg on that source alone,
bit for bit (the systems run the same arithmetic; they only share kernel launches and, in the FP32
iterations, the link loads of the Dslash; after the solve their checks and refinement run jointly
when every (system, shift) pair fits the refinement's 64 slots, else system by system: 4 x 17), in
every FP32 Krylov mode, with and without the double-FP32 first phase and with and without CUDA graphs; the oracle's FP64 true residual of every
returned x_k is at most tol; unsupported modes and bad arguments are refused.
"""
import numpy as np
import pytest

from gpu_util import make_context, rel_norm, to_dev
from oracle import rational, solvers, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32, FP32_R12, FP16FIX, FP32_R8, FP32_L16, DF64 = 0, 1, 2, 3, 4, 5, 6


def _solve_single(lq, ctx, b, poles, res, c0, prec):
    import torch

    xs = [torch.empty_like(b) for _ in poles]
    y = torch.empty_like(b)
    rc, st = lq.mshift_cg(ctx, poles, res, c0, b, xs, y, tol=1e-10, prec=prec)
    torch.cuda.synchronize()
    return rc, st, [x.clone() for x in xs], y.clone()


def _solve_multi(lq, ctx, bs, poles, res, c0, prec):
    import torch

    xs = [[torch.empty_like(b) for _ in poles] for b in bs]
    ys = [torch.empty_like(b) for b in bs]
    rc, sts = lq.mshift_cg_multi(ctx, poles, res, c0, bs, xs, ys, tol=1e-10, prec=prec)
    torch.cuda.synchronize()
    return rc, sts, xs, ys


KEYS = ("iterations", "reliable_updates", "refine_iterations", "refined_shifts", "refine_rounds", "shift_iterations",
        "df_iterations", "true_residual")


@pytest.mark.parametrize("dims,mass,npoles,nrhs", [((10, 6, 4, 6), 0.05, 12, 2), ((16, 16, 16, 8), 0.05, 14, 4),
                                                   ((8, 8, 8, 4), 0.02, 12, 3), ((8, 8, 8, 4), 0.02, 17, 4)])
@pytest.mark.parametrize("prec", [FP32, FP32_R12, FP16FIX, FP32_L16])
def test_multi_equals_single_solves(dims, mass, npoles, nrhs, prec):
    import paper_1710_09178_gb300 as lq

    ctx, U = make_context(dims, mass, gauge_seed=31)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(npoles, 4 * mass ** 2, 16 + 4 * mass ** 2)
    bs = [to_dev(inputs.gaussian_vector(dims, 40 + s)) for s in range(nrhs)]
    single = [_solve_single(lq, ctx, b, poles, res, c0, prec) for b in bs]
    rc, sts, xs, ys = _solve_multi(lq, ctx, bs, poles, res, c0, prec)
    assert rc == 0
    for s in range(nrhs):
        rc1, st1, xs1, y1 = single[s]
        assert rc1 == 0
        for k in KEYS:
            assert sts[s][k] == st1[k], (s, k, sts[s][k], st1[k])
        for a, c in zip(xs[s], xs1):
            assert np.array_equal(a.cpu().numpy(), c.cpu().numpy())
        assert np.array_equal(ys[s].cpu().numpy(), y1.cpu().numpy())


@pytest.mark.parametrize("switch,graph", [(0.0, 1), (1e-3, 0), (0.0, 0)])
def test_multi_equals_single_without_schedule_or_graphs(switch, graph):
    # FP32 from the start (no double-FP32 phase) and/or plain launches polled by the host
    import paper_1710_09178_gb300 as lq

    dims, mass = (10, 6, 4, 6), 0.05
    ctx, U = make_context(dims, mass, gauge_seed=33)
    ctx.set_option(lq.OPT_DF_SWITCH, switch)
    ctx.set_option(lq.OPT_USE_GRAPH, graph)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    bs = [to_dev(inputs.gaussian_vector(dims, 50 + s)) for s in range(4)]
    single = [_solve_single(lq, ctx, b, poles, res, c0, FP32) for b in bs]
    rc, sts, xs, ys = _solve_multi(lq, ctx, bs, poles, res, c0, FP32)
    assert rc == 0
    for s in range(4):
        assert sts[s]["iterations"] == single[s][1]["iterations"]
        for a, c in zip(xs[s], single[s][2]):
            assert np.array_equal(a.cpu().numpy(), c.cpu().numpy())


def test_multi_certified_by_oracle():
    # four Gaussian sources of the 16^3 x 4 batch lattice, 12-pole x^{-1/2} at m = 0.02
    import paper_1710_09178_gb300 as lq

    dims, mass = (16, 16, 16, 4), 0.02
    ctx, U = make_context(dims, mass, gauge_seed=35)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    bh = [inputs.gaussian_vector(dims, 60 + s) for s in range(4)]
    rc, sts, xs, ys = _solve_multi(lq, ctx, [to_dev(b) for b in bh], poles, res, c0, FP32)
    assert rc == 0
    A = lambda v, s: staggered.A_apply(U, v, mass, dims, s)
    for s in range(4):
        xh = [x.cpu().numpy() for x in xs[s]]
        tr = solvers.true_residuals(A, bh[s], xh, poles)
        assert np.all(tr <= 1e-10), (s, tr)
        assert rel_norm(ys[s].cpu().numpy(), solvers.rational_apply(bh[s], xh, c0, res)) < 1e-13


def test_multi_of_one_equals_mshift_cg_and_partial_outputs():
    import torch

    import paper_1710_09178_gb300 as lq

    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U = make_context(dims, mass)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(8, 4 * mass ** 2, 16 + 4 * mass ** 2)
    b = to_dev(inputs.gaussian_vector(dims, 70))
    rc1, st1, xs1, y1 = _solve_single(lq, ctx, b, poles, res, c0, FP32)
    rc, sts, xs, ys = _solve_multi(lq, ctx, [b], poles, res, c0, FP32)
    assert rc == rc1 == 0 and sts[0]["iterations"] == st1["iterations"]
    assert all(torch.equal(a, c) for a, c in zip(xs[0], xs1)) and torch.equal(ys[0], y1)
    # x outputs of one system only, y of the other only
    b2 = to_dev(inputs.gaussian_vector(dims, 71))
    xs2 = [torch.empty_like(b) for _ in poles]
    y2 = torch.empty_like(b)
    rc, sts = lq.mshift_cg_multi(ctx, poles, res, c0, [b, b2], [xs2, None], [None, y2], prec=FP32)
    torch.cuda.synchronize()
    assert rc == 0
    assert all(torch.equal(a, c) for a, c in zip(xs2, xs1))
    _, _, _, y2ref = _solve_single(lq, ctx, b2, poles, res, c0, FP32)
    assert torch.equal(y2, y2ref)


def test_multi_rejects_bad_arguments():
    import paper_1710_09178_gb300 as lq

    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U = make_context(dims, mass)
    b1, b2 = to_dev(inputs.gaussian_vector(dims, 80)), to_dev(inputs.gaussian_vector(dims, 81))
    for prec in (FP64, DF64):  # several right-hand sides need an FP32 Krylov mode
        rc, _ = lq.mshift_cg_multi(ctx, [0.1, 0.2], [1.0, 1.0], 0.0, [b1, b2], prec=prec, raise_on_error=False)
        assert rc == lq.LQCD_ERR_ARG
    rc, _ = lq.mshift_cg_multi(ctx, [0.1], [1.0], 0.0, [b1] * 5, prec=FP32, raise_on_error=False)
    assert rc == lq.LQCD_ERR_ARG
    rc, _ = lq.mshift_cg_multi(ctx, [0.1], [1.0], 0.0, [b1, b1], prec=FP32, raise_on_error=False)
    assert rc == lq.LQCD_ERR_ARG
    ctx.set_option(lq.OPT_DF_RESID, 0)
    rc, _ = lq.mshift_cg_multi(ctx, [0.1], [1.0], 0.0, [b1, b2], prec=FP32, raise_on_error=False)
    assert rc == lq.LQCD_ERR_ARG
    # the context stays usable
    ctx.set_option(lq.OPT_DF_RESID, 1)
    rc, _ = lq.mshift_cg_multi(ctx, [0.1], [1.0], 0.0, [b1, b2], prec=FP32, raise_on_error=False)
    assert rc == 0


@pytest.mark.parametrize("refine", [0, 1])
def test_multi_joint_and_fallback_post_solve(refine):
    # After the solve the systems' checks and refinement run jointly; a zero source among them sends
    # the call down the system-by-system path.  Either way, with and without refinement, every system
    # equals its own mshift_cg bit for bit.
    import torch

    import paper_1710_09178_gb300 as lq

    dims, mass = (8, 8, 8, 4), 0.02
    ctx, U = make_context(dims, mass, gauge_seed=37)
    ctx.set_option(lq.OPT_REFINE, refine)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    b1, b2 = to_dev(inputs.gaussian_vector(dims, 90)), to_dev(inputs.gaussian_vector(dims, 91))
    for bs in ([b1, b2], [b1, torch.zeros_like(b1), b2]):
        single = []
        for b in bs:
            xs1 = [torch.empty_like(b) for _ in poles]
            y1 = torch.empty_like(b)
            rc1, st1 = lq.mshift_cg(ctx, poles, res, c0, b, xs1, y1, tol=1e-10, prec=FP32, raise_on_error=False)
            single.append((rc1, st1, xs1, y1))
        xs = [[torch.empty_like(b) for _ in poles] for b in bs]
        ys = [torch.empty_like(b) for b in bs]
        rc, sts = lq.mshift_cg_multi(ctx, poles, res, c0, bs, xs, ys, tol=1e-10, prec=FP32, raise_on_error=False)
        torch.cuda.synchronize()
        assert rc == next((x[0] for x in single if x[0] != 0), 0)  # the first system that is not OK
        if refine:
            assert rc == 0
        for s in range(len(bs)):
            for k in KEYS:
                assert sts[s][k] == single[s][1][k], (len(bs), s, k)
            for a, c in zip(xs[s], single[s][2]):
                assert torch.equal(a, c)
            assert torch.equal(ys[s], single[s][3])
