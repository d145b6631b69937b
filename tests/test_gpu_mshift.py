"""GPU parity of the shifted CG (Section 4, ref. [mcg]) and the rational application (Eq. ratapprx).

Bars:
  - FP64, fixed iteration count (no shift stopped): every x_k within 1e-12 relative of
    the oracle run for the same number of iterations (the two differ only in the
    summation order of the dot products and in when the x_k, p_k updates are applied);
    double-FP32 (~48-bit arithmetic) within 1e-11;
  - FP64 without refinement, converged: the same stopping iteration for every shift as
    the oracle, and every x_k within 1e-12 relative of the oracle's, or within 4 times the
    difference between the numpy and the C++ oracle where those two (which differ only in the
    order of their sums) already disagree by more: near convergence CG amplifies rounding
    (4^4: the two oracles differ by 6e-12 after 102 iterations);
  - converged solves, every precision: the FP64 true residual |b - (A+d_k)x_k|/|b|
    computed by the oracle is <= the requested 1e-10 for every shift, and x_k is within
    kappa_k * 2e-10 of the oracle's converged solution (kappa_k bounds the condition number);
  - y = c0 b + sum c_k x_k within the same bound of the oracle's y.
"""
import numpy as np
import pytest

from gpu_util import gpu_mshift, make_context, rel_norm
from oracle import rational, solvers, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32, FP32_R12, FP16FIX, FP32_R8, FP32_L16, DF64 = 0, 1, 2, 3, 4, 5, 6


def _problem(dims, mass, npoles, gseed, vseed):
    ctx, U = make_context(dims, mass, gauge_seed=gseed)
    b = inputs.gaussian_vector(dims, vseed)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(npoles, 4 * mass ** 2, 16 + 4 * mass ** 2)
    return ctx, U, b, c0, res, poles


@pytest.mark.parametrize("prec", [FP64, DF64])
@pytest.mark.parametrize("dims,iters", [((4, 4, 4, 4), 25), ((10, 6, 4, 6), 37), ((16, 16, 16, 8), 20)])
def test_fp64_fixed_iterations_match_oracle(dims, iters, prec):
    # FP64 and double-FP32 (~48-bit) recurrences against the oracle for the same iteration count
    import paper_1710_09178_gb300 as lq

    mass = 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 12, 1, 2)
    ctx.set_option(lq.OPT_REFINE, 0)
    rc, st, xs, _ = gpu_mshift(ctx, b, poles, tol=1e-300, maxiter=iters, prec=prec)
    assert rc == lq.LQCD_ERR_NOT_CONVERGED and st["iterations"] == iters
    oxs, info = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, poles.min()), b, poles,
                                      fixed_iters=iters)
    bar = 1e-12 if prec == FP64 else 1e-11
    for x, ox in zip(xs, oxs):
        assert rel_norm(x, ox) < bar


def test_fp64_fixed_iterations_match_oracle_32c8():
    # the bench workload (32^3 x 8, m 0.02, 16-pole x^{-1/2}, gauge seed 5, source seed 6) in FP64
    # for 20 iterations with no shift stopped, against the C++ oracle's 20 iterations: 1e-12
    import paper_1710_09178_gb300 as lq
    from oracle import cpp_oracle

    dims, mass, iters = (32, 32, 32, 8), 0.02, 20
    ctx, U = make_context(dims, mass, gauge_seed=5)
    b = inputs.gaussian_vector(dims, 6)
    c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * mass ** 2, 16 + 4 * mass ** 2, 16)
    ctx.set_option(lq.OPT_REFINE, 0)
    rc, st, xs, _ = gpu_mshift(ctx, b, poles, tol=1e-300, maxiter=iters, prec=FP64)
    assert rc == lq.LQCD_ERR_NOT_CONVERGED and st["iterations"] == iters
    oxs, _ = cpp_oracle.load(threaded=True).lattice(dims, U, mass).multishift_cg(b, poles, fixed_iters=iters)
    for x, ox in zip(xs, oxs):
        assert rel_norm(x, ox) < 1e-12


def _check_converged(ctx, U, b, dims, mass, c0, res, poles, prec, tol=1e-10):
    import paper_1710_09178_gb300 as lq

    rc, st, xs, y = gpu_mshift(ctx, b, poles, res, c0, tol=tol, prec=prec, want_y=True)
    assert rc == lq.LQCD_OK, st
    tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, poles)
    assert np.all(tr <= tol * 1.001), tr
    assert np.allclose(tr, st["true_residual"], rtol=1e-3, atol=1e-14)
    return st, xs, y


@pytest.mark.parametrize("prec", [FP64, FP32, FP32_R12, FP16FIX, FP32_R8, FP32_L16, DF64])
def test_converged_solve_matches_oracle_4444(prec):
    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U, b, c0, res, poles = _problem(dims, mass, 12, 1, 2)
    st, xs, y = _check_converged(ctx, U, b, dims, mass, c0, res, poles, prec)
    oxs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, poles.min()), b, poles, tol=1e-12)
    lmin = 4 * mass ** 2
    for x, ox, s in zip(xs, oxs, poles):
        kappa = (16 + lmin + s) / (lmin + s)
        assert rel_norm(x, ox) <= kappa * 2e-10
    oy = solvers.rational_apply(b, oxs, c0, res)
    assert rel_norm(y, oy) <= (16 / lmin) * 2e-10


@pytest.mark.parametrize("prec", [FP64, FP32, FP32_R12, FP16FIX, FP32_R8, FP32_L16, DF64])
def test_converged_solve_16c8(prec):
    dims, mass = (16, 16, 16, 8), 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 14, 3, 4)
    st, xs, y = _check_converged(ctx, U, b, dims, mass, c0, res, poles, prec)
    assert st["iterations"] > 10
    if prec == DF64:
        # ~48-bit recurrences: the iterated residuals stay true, nothing to update or refine
        assert st["reliable_updates"] == 0 and st["refine_iterations"] == 0
    elif prec != FP64:
        assert st["reliable_updates"] >= st["iterations"] // 100 - 1


def test_ragged_lattice_and_unsorted_duplicate_shifts():
    dims, mass = (10, 6, 4, 6), 0.05
    ctx, U = make_context(dims, mass, gauge_seed=6)
    b = inputs.gaussian_vector(dims, 7)
    shifts = np.array([0.3, 0.0, 0.3, 2.5, 0.001])
    for prec in (FP64, FP32):
        rc, st, xs, _ = gpu_mshift(ctx, b, shifts, tol=1e-10, prec=prec)
        assert rc == 0
        tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, shifts)
        assert np.all(tr <= 1.001e-10)
        assert rel_norm(xs[0], xs[2]) < 1e-9


def test_single_shift_and_zero_source():
    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U = make_context(dims, mass)
    b = np.zeros((128, 3), dtype=np.complex128)
    rc, st, xs, y = gpu_mshift(ctx, b, [0.01, 0.2], [1.0, 2.0], 0.5, prec=FP32, want_y=True)
    assert rc == 0 and all(np.all(x == 0) for x in xs) and np.all(y == 0)
    b = inputs.gaussian_vector(dims, 9)
    rc, st, xs, _ = gpu_mshift(ctx, b, [0.0], prec=FP32)
    assert rc == 0
    xc, _ = solvers.cg(lambda v: staggered.A_apply(U, v, mass, dims), b, tol=1e-12)
    assert rel_norm(xs[0], xc) < (16 / 0.04) * 2e-10


def test_maxiter_and_nonfinite_status():
    import paper_1710_09178_gb300 as lq

    dims, mass = (4, 4, 4, 4), 0.01
    ctx, U = make_context(dims, mass)
    b = inputs.gaussian_vector(dims, 10)
    ctx.set_option(lq.OPT_REFINE, 0)
    rc, st, xs, _ = gpu_mshift(ctx, b, [0.0, 0.1], maxiter=3, prec=FP32)
    assert rc == lq.LQCD_ERR_NOT_CONVERGED and st["iterations"] == 3
    b2 = b.copy()
    b2[5, 1] = np.nan
    rc, st, xs, _ = gpu_mshift(ctx, b2, [0.0, 0.1], prec=FP32)
    assert rc == lq.LQCD_ERR_NONFINITE
    # the context stays usable after an error
    ctx.set_option(lq.OPT_REFINE, 1)
    rc, st, xs, _ = gpu_mshift(ctx, b, [0.0, 0.1], prec=FP32)
    assert rc == 0


def test_no_graph_path_matches_graph_path():
    import paper_1710_09178_gb300 as lq

    dims, mass = (10, 6, 4, 6), 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 12, 2, 3)
    ctx.set_option(lq.OPT_REFINE, 0)
    _, st1, xs1, _ = gpu_mshift(ctx, b, poles, tol=1e-300, maxiter=33, prec=FP32)
    ctx.set_option(lq.OPT_USE_GRAPH, 0)
    ctx.set_option(lq.OPT_REFINE, 0)
    _, st2, xs2, _ = gpu_mshift(ctx, b, poles, tol=1e-300, maxiter=33, prec=FP32)
    for a, c in zip(xs1, xs2):
        assert np.array_equal(a, c)  # deterministic reductions: identical bits


@pytest.mark.parametrize("tps,bs,order", [(1, 64, 1), (2, 128, 0), (4, 64, 0), (8, 128, 1)])
def test_converged_solve_every_launch_shape(tps, bs, order):
    # The FP32 Dslash's launch shape (threads per site, threads per block, block-to-site order) changes
    # the per-site sums (threads per site) and the block partials the update kernels sum (their count
    # and grouping); whatever the shape, every shift is certified by the oracle at 1e-10 and the
    # reported residuals are the oracle's.
    import paper_1710_09178_gb300 as lq

    dims, mass = (10, 6, 4, 6), 0.02
    ctx, U, b, c0, res, poles = _problem(dims, mass, 12, 11, 12)
    ctx.set_option(lq.OPT_DSLASH_TPS, tps)
    ctx.set_option(lq.OPT_DSLASH_BS, bs)
    ctx.set_option(lq.OPT_DSLASH_ORDER, order)
    for prec in (FP32, FP32_R12):
        st, xs, y = _check_converged(ctx, U, b, dims, mass, c0, res, poles, prec)
        assert st["iterations"] > 10


@pytest.mark.parametrize("dims,mass,npoles", [((10, 6, 4, 6), 0.05, 12), ((16, 16, 16, 8), 0.05, 14)])
def test_reported_true_residuals_match_oracle(dims, mass, npoles):
    # The mixed modes compute reliable updates and true residuals in double-FP32 (~48-bit) instead
    # of FP64.  The residual norms they report must be the oracle's FP64 residuals of the returned
    # solutions: at convergence (b - (A + d_k) x_k cancels to 1e-10 of |b|) within 1e-12 + 0.2 %,
    # and on an unconverged iterate within 1e-7 relative (the residual vector is rounded to FP32
    # before its norm is taken) plus 1e-13 absolute: the 15 iterations of the unconverged case run
    # in the double-FP32 first phase of the precision schedule, which leaves the large shifts with
    # residuals near 1e-12, where the double-FP32 residual's cancellation floor decides.
    import paper_1710_09178_gb300 as lq

    ctx, U, b, c0, res, poles = _problem(dims, mass, npoles, 3, 4)
    A = lambda v, s: staggered.A_apply(U, v, mass, dims, s)
    for prec in (FP32, FP16FIX, FP32_L16):
        rc, st, xs, _ = gpu_mshift(ctx, b, poles, prec=prec)
        assert rc == 0
        tr = solvers.true_residuals(A, b, xs, poles)
        rep = np.array(st["true_residual"][: len(poles)])
        assert np.all(np.abs(rep - tr) <= 1e-12 + 2e-3 * tr), (rep, tr)
    for switch in (1e-3, 0.0):  # with and without the double-FP32 first phase
        ctx.set_option(lq.OPT_DF_SWITCH, switch)
        ctx.set_option(lq.OPT_REFINE, 0)
        rc, st, xs, _ = gpu_mshift(ctx, b, poles, maxiter=15, prec=FP32)
        assert rc == lq.LQCD_ERR_NOT_CONVERGED
        tr = solvers.true_residuals(A, b, xs, poles)
        rep = np.array(st["true_residual"][: len(poles)])
        assert np.all(np.abs(rep - tr) <= 1e-13 + 1e-7 * tr), (switch, rep, tr)


def test_double_fp32_and_fp64_residual_paths_agree():
    # the same mixed solve with its residuals in double-FP32 and in FP64: the reliable updates
    # round differently in the last FP32 bit, so iteration counts may differ by a step or two;
    # solutions equal to well within the tolerance
    import paper_1710_09178_gb300 as lq

    dims, mass = (16, 16, 16, 8), 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 14, 3, 4)
    rc1, st1, xs1, _ = gpu_mshift(ctx, b, poles, prec=FP32)
    ctx.set_option(lq.OPT_DF_RESID, 0)
    rc2, st2, xs2, _ = gpu_mshift(ctx, b, poles, prec=FP32)
    assert rc1 == rc2 == 0
    assert abs(st1["iterations"] - st2["iterations"]) <= 2
    for x1, x2, s in zip(xs1, xs2, poles):
        kappa = (16 + 4 * mass ** 2 + s) / (4 * mass ** 2 + s)
        assert rel_norm(x1, x2) <= kappa * 2e-10


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_programmatic_dependent_launch_matches_plain_launches(prec):
    # the same graphs captured with and without programmatic dependencies between their kernels,
    # refinement (its own multi-RHS graph) included: identical bits
    import paper_1710_09178_gb300 as lq

    dims, mass = (16, 16, 16, 8), 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 14, 3, 4)
    rc1, st1, xs1, y1 = gpu_mshift(ctx, b, poles, res, c0, prec=prec, want_y=True)
    ctx.set_option(lq.OPT_PDL, 0)
    rc2, st2, xs2, y2 = gpu_mshift(ctx, b, poles, res, c0, prec=prec, want_y=True)
    assert rc1 == rc2 == 0
    assert st1["iterations"] == st2["iterations"] and st1["refine_iterations"] == st2["refine_iterations"]
    for a, c in zip(xs1, xs2):
        assert np.array_equal(a, c)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("dims,mass,npoles", [((4, 4, 4, 4), 0.1, 12), ((16, 16, 16, 8), 0.05, 14)])
def test_fp64_unrefined_solve_matches_oracle_with_same_stopping_rule(dims, mass, npoles):
    # No refinement: every shift stops on |zeta_k| |r| <= tol |b| exactly as in the oracle, and
    # the solutions must agree to the accuracy the two recurrences share (shifts stop in the same
    # iteration; only the summation order of the dot products differs).
    import paper_1710_09178_gb300 as lq

    ctx, U, b, c0, res, poles = _problem(dims, mass, npoles, 3, 4)
    ctx.set_option(lq.OPT_REFINE, 0)
    rc, st, xs, _ = gpu_mshift(ctx, b, poles, tol=1e-10, prec=FP64)
    oxs, info = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, poles.min()), b, poles,
                                      tol=1e-10)
    assert st["iterations"] == info["iterations"]
    assert st["shift_iterations"] == info["shift_iterations"]  # every shift stopped in the same iteration
    # rounding-order spread: the C++ oracle's solve against the numpy oracle's
    from oracle import cpp_oracle

    cxs, cinfo = cpp_oracle.load(threaded=False).lattice(dims, U, mass).multishift_cg(b, poles, tol=1e-10)
    spread = max(rel_norm(c, o) for c, o in zip(cxs, oxs)) if cinfo["iterations"] == info["iterations"] else 0.0
    bar = max(1e-12, 4 * spread)
    for x, ox in zip(xs, oxs):
        assert rel_norm(x, ox) < bar, (rel_norm(x, ox), spread)
    otr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, oxs, poles)
    assert np.allclose(st["true_residual"], otr, rtol=0.1, atol=1e-12)  # near tol the residuals differ at rounding level


@pytest.fixture(scope="module")
def oracle_32c8():
    """The C++ oracle's lattice for the bench workload (32^3 x 8, m 0.02, gauge seed 5) and its own
    converged 16-pole x^{-1/2} and x^{1/4} solves of source seed 6, with the library's coefficients."""
    import paper_1710_09178_gb300 as lq
    from oracle import cpp_oracle

    dims, mass = (32, 32, 32, 8), 0.02
    from gpu_util import seeded_gauge

    U = seeded_gauge(dims, 5)
    b = inputs.gaussian_vector(dims, 6)
    lat = cpp_oracle.load(threaded=True).lattice(dims, U, mass)
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    out = {}
    for power in (-0.5, 0.25):
        c0, res, poles, _ = lq.rational_coeffs(power, lo, hi, 16)
        oxs, _ = lat.multishift_cg(b, poles, tol=1e-10)
        out[power] = (c0, res, poles, oxs)
    return dims, mass, U, b, lat, out


@pytest.mark.parametrize("prec,power", [(FP32, -0.5), (DF64, -0.5), (FP64, -0.5), (FP32, 0.25)])
def test_full_size_32c8_solve_certified_by_oracle(oracle_32c8, prec, power):
    # the benchmark's workload and launch configuration (32^3 x 8, m 0.02, 16-pole x^{-1/2} on
    # [4m^2, 16 + 4m^2] from lqcd_rational_coeffs, gauge seed 5, source seed 6, default options; and
    # the heatbath's x^{1/4}): the oracle's FP64 true residual of every returned x_k is at most tol and
    # equals the one the solve reports; every x_k is within 2 kappa_k tol of the oracle's own solve
    # (kappa_k = (16 + 4m^2 + d_k) / (4m^2 + d_k) bounds the condition number of A + d_k); the returned
    # y is the oracle's c0 b + sum_k c_k x_k of the returned x_k
    dims, mass, U, b, lat, orc = oracle_32c8
    c0, res, poles, oxs = orc[power]
    ctx, _ = make_context(dims, mass, gauge_seed=5)
    rc, st, xs, y = gpu_mshift(ctx, b, poles, res, c0, prec=prec, want_y=True)
    assert rc == 0
    tr = lat.true_residuals(b, xs, poles)
    assert np.all(tr <= 1e-10), tr
    rep = np.array(st["true_residual"][: len(poles)])
    assert np.all(np.abs(rep - tr) <= 1e-12 + 2e-3 * tr), (rep, tr)
    lmin = 4 * mass ** 2
    for x, ox, s in zip(xs, oxs, poles):
        assert rel_norm(x, ox) <= 2 * (16 + lmin + s) / (lmin + s) * 1e-10
    yo = solvers.rational_apply(b, xs, c0, res)
    assert rel_norm(y, yo) < 1e-13


def test_lattice_beyond_l2_40c8():
    # 40^3 x 8: the FP32 links (147 MB) no longer fit in the 126 MB L2, so the solve streams them
    # from HBM every half-Dslash.  8-pole x^{-1/2}, mixed precision; every shift certified by the
    # oracle's FP64 true residual
    dims, mass = (40, 40, 40, 8), 0.05
    ctx, U = make_context(dims, mass, gauge_seed=71)
    b = inputs.gaussian_vector(dims, 72)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(8, 4 * mass ** 2, 16 + 4 * mass ** 2)
    rc, st, xs, _ = gpu_mshift(ctx, b, poles, res, c0, prec=FP32)
    assert rc == 0
    tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, poles)
    assert np.all(tr <= 1e-10), tr


@pytest.mark.parametrize("prec", [FP32, FP32_R12, FP16FIX])
def test_precision_schedule_certified_and_shortens_refinement(prec):
    # The mixed modes start in double-FP32 and change to FP32 at the first window end with
    # |r| <= 1e-3 |b| (LQCD_OPT_DF_SWITCH): every shift certified by the oracle's FP64 true residual,
    # the x_k within the kappa_k tol bound of the oracle's, fewer refinement iterations than the same
    # solve in FP32 from the start, and the same base iteration count
    import paper_1710_09178_gb300 as lq

    dims, mass = (16, 16, 16, 8), 0.05
    ctx, U, b, c0, res, poles = _problem(dims, mass, 14, 3, 4)
    A = lambda v, s: staggered.A_apply(U, v, mass, dims, s)
    out = {}
    for switch in (1e-3, 0.0):
        ctx.set_option(lq.OPT_DF_SWITCH, switch)
        rc, st, xs, _ = gpu_mshift(ctx, b, poles, prec=prec)
        assert rc == 0
        tr = solvers.true_residuals(A, b, xs, poles)
        assert np.all(tr <= 1e-10), (switch, tr)
        assert (st["df_iterations"] > 0) == (switch > 0)
        out[switch] = (st, xs)
    assert out[1e-3][0]["refine_iterations"] < out[0.0][0]["refine_iterations"]
    assert abs(out[1e-3][0]["iterations"] - out[0.0][0]["iterations"]) <= 2
    oxs, _ = solvers.multishift_cg(lambda v: A(v, poles.min()), b, poles, tol=1e-12)
    lmin = 4 * mass ** 2
    for x, ox, s in zip(out[1e-3][1], oxs, poles):
        assert rel_norm(x, ox) <= 2 * (16 + lmin + s) / (lmin + s) * 1e-10
