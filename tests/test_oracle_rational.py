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
