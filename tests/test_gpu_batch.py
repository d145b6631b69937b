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
    tps, bs, order = ctx.autotune_shape(lq.FP32)
    assert tps in (1, 2, 4, 8) and bs in (64, 128) and order in (0, 1)
    psi = inputs.gaussian_vector(dims, 71)
    for p in (0, 1):
        assert rel_max(gpu_dslash(ctx, psi, p, lq.FP32), staggered.dslash_eo(U, psi, dims, p)) < 2e-6


@pytest.mark.parametrize("prec", [1, 2, 4, 5])  # FP32, 12-real, 8-real, 16-bit links
def test_every_launch_shape_matches_oracle(prec):
    # threads per site x threads per block x block-to-site order: the half-Dslash against the oracle
    # (element by element, ragged 10x6x4x6 lattice: V/2 = 720 sites, not a multiple of any block), the
    # A-apply's dot product, and a converged mixed solve certified by the oracle's FP64 true residual
    import itertools

    import paper_1710_09178_gb300 as lq
    from gpu_util import gpu_apply_A, gpu_mshift
    from oracle import linkcomp, rational, solvers

    dims, mass = (10, 6, 4, 6), 0.05
    ctx, U = make_context(dims, mass, gauge_seed=72)
    Ur = linkcomp.decode_l16(linkcomp.encode_l16(U.reshape(-1, 3, 3))).reshape(U.shape) if prec == 5 else U
    psi = inputs.gaussian_vector(dims, 73)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(8, 4 * mass ** 2, 16 + 4 * mass ** 2)
    tol = 1e-4 if prec == 4 else 2e-6
    for tps, bs, order in itertools.product((1, 2, 4, 8), (64, 128), (0, 1)):
        ctx.set_option(lq.OPT_DSLASH_TPS, tps)
        ctx.set_option(lq.OPT_DSLASH_BS, bs)
        ctx.set_option(lq.OPT_DSLASH_ORDER, order)
        for p in (0, 1):
            got = gpu_dslash(ctx, psi, p, prec)
            assert rel_max(got, staggered.dslash_eo(Ur, psi, dims, p)) < tol, (tps, bs, order, p)
        q, pq = gpu_apply_A(ctx, psi, 0.2, prec)
        ref = staggered.A_apply(Ur, psi, mass, dims, 0.2)
        assert abs(pq - np.real(np.vdot(psi, ref))) <= tol * abs(pq), (tps, bs, order)
        if (tps, bs, order) in ((8, 64, 1), (2, 128, 1)):
            rc, st, xs, _ = gpu_mshift(ctx, psi, poles, prec=prec)
            assert rc == 0
            tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), psi, xs, poles)
            assert np.all(tr <= 1e-10)


@pytest.mark.parametrize("prec", [0, 1, 2, 4, 5])  # FP64, FP32, 12-real, 8-real, 16-bit links
def test_dslash_batch_equals_single_launches_and_oracle(prec):
    # five lattices of different sizes (one with a ragged last chunk: V/2 = 720), both parities:
    # the persistent batched launch gives the bits of one dslash_eo per lattice, and those match
    # the oracle (16-bit links: on the oracle-decoded links)
    import torch

    import paper_1710_09178_gb300 as lq
    from oracle import linkcomp

    lattices = [(4, 4, 4, 4), (10, 6, 4, 6), (8, 8, 8, 8), (16, 16, 16, 4), (2, 2, 2, 2)]
    ctxs, ins, outs, refs, pars = [], [], [], [], []
    for li, dims in enumerate(lattices):
        ctx, U = make_context(dims, 0.05, gauge_seed=80 + li)
        psi = inputs.gaussian_vector(dims, 90 + li)
        p = li & 1
        vin = ctx.new_vector(prec)
        ctx.pack(vin, prec, to_dev(psi))
        ctxs.append(ctx)
        ins.append(vin)
        outs.append(ctx.new_vector(prec))
        pars.append(p)
        Ur = linkcomp.decode_l16(linkcomp.encode_l16(U.reshape(-1, 3, 3))).reshape(U.shape) if prec == 5 else U
        refs.append(staggered.dslash_eo(Ur, psi, dims, p))
    lq.dslash_eo_batch(ctxs, outs, ins, pars, prec)
    torch.cuda.synchronize()
    for ctx, vin, vout, p, ref in zip(ctxs, ins, outs, pars, refs):
        single = ctx.new_vector(prec)
        lq.dslash_eo(ctx, single, vin, p, prec)
        torch.cuda.synchronize()
        assert torch.equal(single, vout)
        got = torch.empty(ctx.Vh, 3, dtype=torch.complex128, device="cuda")
        ctx.unpack(got, vout, prec)
        got = got.cpu().numpy()
        tol = 1e-12 if prec == 0 else (1e-4 if prec == 4 else 2e-6)
        assert rel_max(got, ref) < tol


def test_dslash_batch_rejects_bad_arguments():
    import paper_1710_09178_gb300 as lq

    ctx, _ = make_context((4, 4, 4, 4), 0.1)
    v, w = ctx.new_vector(lq.FP32), ctx.new_vector(lq.FP32)
    for args in (([ctx], [v], [v], [0], lq.FP32), ([ctx], [w], [v], [2], lq.FP32), ([ctx], [w], [v], [0], lq.DF64),
                 ([ctx], [w], [v], [0], lq.FP16FIX)):
        with pytest.raises(lq.LqcdError):
            lq.dslash_eo_batch(*args)
    bare = lq.Context((4, 4, 4, 4), 0.1)
    with pytest.raises(lq.LqcdError):
        lq.dslash_eo_batch([ctx, bare], [w, v], [v, w], [0, 1], lq.FP32)
    with pytest.raises(lq.LqcdError):
        lq.dslash_eo_batch([ctx] * (lq.MAX_BATCH + 1), [w] * (lq.MAX_BATCH + 1), [v] * (lq.MAX_BATCH + 1),
                           [0] * (lq.MAX_BATCH + 1), lq.FP32)


def test_dslash_batch_of_many_lattices_in_one_launch_and_under_capture():
    # 70 lattices (more than one parameter block holds): one persistent launch from the uploaded
    # descriptor table; a new set of descriptors first met inside a CUDA-graph capture takes the
    # parameter-block launches instead.  Both give the bits of one dslash_eo per lattice.
    import torch

    import paper_1710_09178_gb300 as lq

    sizes = [(4, 4, 4, 4), (6, 4, 2, 4), (8, 4, 4, 2), (2, 2, 2, 2), (10, 6, 4, 6)]
    ctxs, ins, outs, pars = [], [], [], []
    for li in range(70):
        dims = sizes[li % len(sizes)]
        ctx, _ = make_context(dims, 0.05, gauge_seed=100 + li % 7)
        vin = ctx.new_vector(lq.FP32)
        ctx.pack(vin, lq.FP32, to_dev(inputs.gaussian_vector(dims, 200 + li)))
        ctxs.append(ctx)
        ins.append(vin)
        outs.append(ctx.new_vector(lq.FP32))
        pars.append((li // 3) & 1)
    launches = ctxs[0].launch_count()
    lq.dslash_eo_batch(ctxs, outs, ins, pars, lq.FP32)
    torch.cuda.synchronize()
    assert ctxs[0].launch_count() - launches == 1
    singles = []
    for ctx, vin, vout, p in zip(ctxs, ins, outs, pars):
        single = ctx.new_vector(lq.FP32)
        lq.dslash_eo(ctx, single, vin, p, lq.FP32)
        torch.cuda.synchronize()
        assert torch.equal(single, vout)
        singles.append(single)
    # the other parity, first met during a capture on the contexts' stream
    s = torch.cuda.Stream()
    for c in ctxs:
        c.set_stream(s.cuda_stream)
    outs2 = [c.new_vector(lq.FP32) for c in ctxs]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        lq.dslash_eo_batch(ctxs, outs2, ins, [1 - p for p in pars], lq.FP32)
    g.replay()
    torch.cuda.synchronize()
    for ctx, vin, vout, p in zip(ctxs, ins, outs2, pars):
        single = ctx.new_vector(lq.FP32)
        lq.dslash_eo(ctx, single, vin, 1 - p, lq.FP32)
        torch.cuda.synchronize()
        assert torch.equal(single, vout)


def test_batch_of_multi_rhs_problems_equals_single_solves():
    # one problem per lattice with its four sources solved together (mshift_cg_multi), the problems
    # run concurrently by mshift_cg_batch: every source's solutions and y equal its stand-alone
    # mshift_cg solve bit for bit
    import torch

    import paper_1710_09178_gb300 as lq

    lattices = [((4, 4, 4, 4), 0.1), ((10, 6, 4, 6), 0.05), ((8, 8, 8, 4), 0.02), ((12, 12, 12, 4), 0.05)]
    problems = []
    for li, (dims, mass) in enumerate(lattices):
        ctx, U = make_context(dims, mass, gauge_seed=150 + li)
        c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
        bs = [to_dev(inputs.gaussian_vector(dims, 160 + 4 * li + f)) for f in range(4)]
        xss = [[torch.empty_like(b) for _ in poles] for b in bs]
        ys = [torch.empty_like(b) for b in bs]
        problems.append(dict(ctx=ctx, shifts=poles, residues=res, c0=c0, bs=bs, xss=xss, ys=ys, tol=1e-10,
                             prec=lq.FP32))
    rc, st, stats = lq.mshift_cg_batch(problems, nthreads=4)
    torch.cuda.synchronize()
    assert rc == 0 and all(s == 0 for s in st)
    for p, sts in zip(problems, stats):
        assert len(sts) == 4
        for f in range(4):
            xs = [torch.empty_like(p["bs"][f]) for _ in p["shifts"]]
            y = torch.empty_like(p["bs"][f])
            rc1, st1 = lq.mshift_cg(p["ctx"], p["shifts"], p["residues"], p["c0"], p["bs"][f], xs, y, tol=1e-10,
                                    prec=lq.FP32)
            torch.cuda.synchronize()
            assert rc1 == 0 and st1["iterations"] == sts[f]["iterations"]
            assert all(torch.equal(a, c) for a, c in zip(xs, p["xss"][f]))
            assert torch.equal(y, p["ys"][f])
