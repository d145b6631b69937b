"""Pins for oracle/rational.py (Eq. ratapprx, Appendix).

The Chebyshev alternation theorem fixes the best approximation: a type (m, n)
rational whose relative error equioscillates at m+n+2 points is the unique
minimax solution.  The tests check that characterisation directly, the sign
structure of the partial fractions, and the Appendix remark that dropping c_0
roughly doubles the error.
"""
import numpy as np
import pytest

from oracle import rational


def _alternation(c0, res, poles, power, lo, hi):
    ext = rational.error_extrema(lambda x: rational.relative_error(c0, res, poles, power, x), lo, hi)
    vals = np.array([v for _, v in ext])
    return vals


@pytest.mark.parametrize("n,mass,ripple", [(5, 0.1, 1e-6), (8, 0.02, 1e-5), (12, 0.1, 1e-2), (14, 0.05, 1e-2),
                                           (16, 0.02, 1e-2)])
def test_zolotarev_equioscillates(n, mass, ripple):
    # ripple: how equal the extremal magnitudes must be; at ~1e-12 errors double-precision
    # evaluation noise (~1e-15) limits it.  By de la Vallee Poussin, max/min <= 1 + ripple puts
    # the error within that factor of the optimum.
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational.zolotarev_inv_sqrt(n, lo, hi)
    vals = _alternation(c0, res, poles, -0.5, lo, hi)
    assert vals.size == 2 * n + 2
    assert np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))
    assert np.max(np.abs(vals)) / np.min(np.abs(vals)) < 1 + ripple
    assert abs(np.max(np.abs(vals)) - err) < ripple * err
    assert c0 > 0 and np.all(res > 0) and np.all(poles > 0)


def test_zolotarev_without_c0_equioscillates_and_is_worse():
    n, lo, hi = 6, 0.04, 16.04
    c0, res, poles, err_nn = rational.zolotarev_inv_sqrt(n, lo, hi)
    c0b, resb, polesb, err_n1 = rational.zolotarev_inv_sqrt(n, lo, hi, with_c0=False)
    assert c0b == 0.0
    vals = _alternation(c0b, resb, polesb, -0.5, lo, hi)
    assert vals.size == 2 * n + 1
    assert np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))
    assert np.max(np.abs(vals)) / np.min(np.abs(vals)) < 1 + 1e-6
    # Appendix: keeping c_0 (same number of shifts) makes the error markedly smaller
    assert 1.5 < err_n1 / err_nn < 4.0


def test_error_decreases_geometrically_with_poles():
    lo, hi = 0.0016, 16.0016
    errs = [rational.zolotarev_inv_sqrt(n, lo, hi)[3] for n in (8, 10, 12, 14, 16)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    ratios = [b / a for a, b in zip(errs, errs[1:])]
    assert max(ratios) / min(ratios) < 1.2


@pytest.mark.parametrize("n,mass", [(12, 0.1), (16, 0.02)])
def test_remez_quarter_power_equioscillates(n, mass):
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational.remez_power(0.25, lo, hi, n)
    ext = rational.error_extrema(lambda x: rational.relative_error(c0, res, poles, 0.25, x), lo, hi, floor=0.1)
    vals = np.array([v for _, v in ext])
    assert vals.size == 2 * n + 2
    assert np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))
    assert np.max(np.abs(vals)) / np.min(np.abs(vals)) < 1.02
    # sign structure of x^{1/4}: c0 > 0, residues < 0, poles > 0
    assert c0 > 0 and np.all(res < 0) and np.all(poles > 0)
    assert err < 1e-10


def test_remez_reproduces_zolotarev_for_inverse_sqrt():
    lo, hi, n = 0.01, 16.01, 10
    c0, res, poles, err = rational.remez_power(-0.5, lo, hi, n)
    zc0, zres, zpoles, zerr = rational.zolotarev_inv_sqrt(n, lo, hi)
    assert np.allclose(np.sort(poles), np.sort(zpoles), rtol=1e-6)
    assert abs(err - zerr) < 0.02 * zerr


def test_appendix_claim_24_poles_quarter_power():
    # Appendix: degree 24/24 approximation of x^{1/4} on [5e-5, 34] has error below 1e-12
    c0, res, poles, err = rational.remez_power(0.25, 5e-5, 34.0, 24)
    assert err < 1e-12
    ext = rational.error_extrema(lambda x: rational.relative_error(c0, res, poles, 0.25, x), 5e-5, 34.0, floor=0.1)
    vals = np.array([v for _, v in ext])
    assert vals.size == 50 and np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))


def test_quarter_squared_times_inverse_sqrt_is_one():
    # r_{1/4}(x)^2 r_{-1/2}(x) = 1 up to the combined approximation errors on the whole interval
    lo, hi, n = 0.0016, 16.0016, 16
    a = rational.remez_power(0.25, lo, hi, n)
    b = rational.zolotarev_inv_sqrt(n, lo, hi)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 5001))
    prod = rational.rational_eval(*a[:3], x) ** 2 * rational.rational_eval(*b[:3], x)
    assert np.max(np.abs(prod - 1)) <= 2.2 * a[3] + 1.1 * b[3]


def test_quarter_power_of_a_dense_operator():
    from oracle import staggered
    from paper_1710_09178_gb300 import inputs

    dims, mass = (4, 4, 4, 4), 0.1
    U = inputs.gauge_field(dims, seed=1)
    A = staggered.dense_A(U, mass, dims)
    w, Q = np.linalg.eigh(A)
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational.remez_power(0.25, lo, hi, 12)
    rA = c0 * np.eye(A.shape[0]) + sum(c * np.linalg.inv(A + d * np.eye(A.shape[0])) for c, d in zip(res, poles))
    exact = (Q * w ** 0.25) @ Q.conj().T
    assert np.linalg.norm(rA - exact, 2) <= 1.5 * err * np.max(w ** 0.25)
