"""Pins for oracle/solvers.py (Section 4, shifted CG): dense LU solves, independent CG solves, residual collinearity, b = 0."""
import numpy as np
import pytest

from oracle import rational, solvers, staggered
from paper_1710_09178_gb300 import inputs


def _setup(dims, mass, gseed=1, vseed=2):
    U = inputs.gauge_field(dims, seed=gseed)
    b = inputs.gaussian_vector(dims, vseed)
    return U, b


@pytest.mark.parametrize("dims,mass", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 4), 0.1), ((4, 2, 2, 4), 0.05)])
def test_multishift_matches_dense_lu(dims, mass):
    U, b = _setup(dims, mass)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    sig0 = poles.min()
    xs, info = solvers.multishift_cg(
        lambda v: staggered.A_apply(U, v, mass, dims, sig0), b, poles, tol=1e-12)
    A = staggered.dense_A(U, mass, dims)
    n = A.shape[0]
    for x, s in zip(xs, poles):
        As = A + s * np.eye(n)
        xd = np.linalg.solve(As, b.reshape(-1))
        kappa = np.linalg.cond(As)
        assert np.linalg.norm(x.reshape(-1) - xd) <= 10 * kappa * 1e-12 * np.linalg.norm(xd)
    assert info["iterations"] > 3


def test_multishift_equals_independent_cg():
    dims, mass = (4, 4, 4, 4), 0.1
    U, b = _setup(dims, mass)
    shifts = np.array([0.002, 0.05, 0.3, 1.7, 9.0])
    xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, shifts.min()), b, shifts, tol=1e-12)
    for x, s in zip(xs, shifts):
        xc, _ = solvers.cg(lambda v: staggered.A_apply(U, v, mass, dims, s), b, tol=1e-12)
        assert np.linalg.norm(x - xc) <= 1e-9 * np.linalg.norm(xc)
    tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, shifts)
    assert np.all(tr < 2e-12)


def test_multishift_shift_order_and_duplicates_do_not_matter():
    dims, mass = (2, 2, 2, 2), 0.1
    U, b = _setup(dims, mass)
    shifts = np.array([0.5, 0.01, 0.5, 3.0])
    xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, 0.01), b, shifts, tol=1e-13)
    A = staggered.dense_A(U, mass, dims)
    for x, s in zip(xs, shifts):
        xd = np.linalg.solve(A + s * np.eye(A.shape[0]), b.reshape(-1))
        assert np.linalg.norm(x.reshape(-1) - xd) < 1e-10 * np.linalg.norm(xd)


def test_zero_source_gives_zero_solution():
    dims, mass = (2, 2, 2, 2), 0.1
    U, _ = _setup(dims, mass)
    b = np.zeros((8, 3), dtype=np.complex128)
    xs, info = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims), b, [0.1, 0.2])
    assert info["iterations"] == 0 and all(np.all(x == 0) for x in xs)


def test_rational_apply_matches_dense_matrix_function():
    # r(A) b through the shifted solve equals A^{-1/2} b from the eigendecomposition, to the approximation error
    dims, mass = (4, 4, 4, 4), 0.1
    U, b = _setup(dims, mass)
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational.zolotarev_inv_sqrt(12, lo, hi)
    xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, poles.min()), b, poles, tol=1e-13)
    y = solvers.rational_apply(b, xs, c0, res)
    A = staggered.dense_A(U, mass, dims)
    w, Q = np.linalg.eigh(A)
    exact = Q @ ((w ** -0.5) * (Q.conj().T @ b.reshape(-1)))
    assert np.linalg.norm(y.reshape(-1) - exact) <= 1.5 * err * np.linalg.norm(exact) + 1e-11


def test_shift_iteration_count():
    # with no shift frozen every (iteration, shift) pair counts; with the stopping rule the count is
    # the sum of each shift's own stopping iteration, which independent single-shift CG runs give
    dims, mass = (4, 4, 4, 4), 0.1
    U = inputs.gauge_field(dims, seed=7)
    b = inputs.gaussian_vector(dims, 8)
    shifts = np.array([0.0, 0.05, 0.4, 3.0])
    base = lambda v: staggered.A_apply(U, v, mass, dims, shifts.min())
    _, info = solvers.multishift_cg(base, b, shifts, fixed_iters=9)
    assert info["shift_iterations"] == 9 * shifts.size
    _, info = solvers.multishift_cg(base, b, shifts, tol=1e-10)
    assert info["shift_iterations"] < shifts.size * info["iterations"]
    stops = []
    for sg in shifts:
        _, it = solvers.cg(lambda v: staggered.A_apply(U, v, mass, dims, sg), b, tol=1e-10)
        stops.append(it)
    assert abs(info["shift_iterations"] - sum(stops)) <= shifts.size  # rounding may move a stop by one


@pytest.mark.parametrize("iters", [1, 2, 5, 12])
def test_shifted_residuals_are_collinear_with_the_base_residual(iters):
    # Section 4, ref. [mcg]: the shifted CG keeps every shifted residual b - (A + sigma_k) x_k equal
    # to zeta_k times the base residual b - (A + sigma_0) x_0; a wrong sign or index anywhere in the
    # zeta recurrence or the x_k / p_k updates breaks this at the first iterations
    dims, mass = (4, 4, 2, 2), 0.1
    U, b = _setup(dims, mass, gseed=5, vseed=6)
    shifts = np.array([0.003, 0.04, 0.5, 2.0, 11.0])
    A = lambda v, s: staggered.A_apply(U, v, mass, dims, s)
    xs, info = solvers.multishift_cg(lambda v: A(v, shifts.min()), b, shifts, fixed_iters=iters)
    k0 = int(np.argmin(shifts))
    r0 = b - A(xs[k0], shifts[k0])
    assert np.isclose(np.vdot(r0, r0).real, info["rr"], rtol=1e-10)
    nb = np.linalg.norm(b)
    for k, s in enumerate(shifts):
        rk = b - A(xs[k], s)
        assert np.linalg.norm(rk - info["zeta"][k] * r0) <= 1e-12 * nb, (k, s)
    assert info["zeta"][k0] == 1.0
