"""Rational approximations in partial fractions (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. ratapprx (Section 4) writes (M^dagger M)^{1/b} = c_0 + sum_k c_k / (M^dagger M + d_k);
the Appendix obtains c_0, c_k, d_k from a minimax approximation of type
(degnum, degden) = (n, n) followed by a partial-fraction split, and notes that
the type (n-1, n) approximation (c_0 = 0) has about twice the error.

Reading: "minimax" is taken in relative error, max_x |r(x)/f(x) - 1| on
[lo, hi] (the paper does not say absolute or relative).

For f(x) = x^{-1/2} the best relative approximation is known in closed form
(Zolotarev, 1877): on [1, kappa] with m' = 1 - 1/kappa, K' = K(m') and
c_l = sn^2(l K'/(2n+1) | m') / cn^2(l K'/(2n+1) | m'),

    R(x) = D prod_{l=1..n} (x + c_{2l}) / (x + c_{2l-1}),

with D chosen so that sqrt(x) R(x) - 1 swings equally above and below zero.
The type (n-1, n) solution uses 2n in place of 2n+1 and drops the last
numerator factor.  Section 4 asks for exactly these two functions (b = -2 and
b = 4); x^{1/4} has no closed form and comes from the exchange algorithm in
`remez_power`.
"""
from __future__ import annotations

import numpy as np
from scipy import special, optimize


def rational_eval(c0, residues, poles, x):
    """r(x) = c0 + sum_k c_k / (x + d_k)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.full_like(x, c0, dtype=np.float64)
    for c, d in zip(residues, poles):
        r = r + c / (x + d)
    return r


def product_to_partial_fractions(K, zeros, poles):
    """R(x) = K prod(x + e_l) / prod(x + d_k) -> (c0, residues) with simple poles d_k.

    c0 is K when numerator and denominator have the same degree, else 0; the
    residue at x = -d_k is K prod_l (e_l - d_k) / prod_{l != k} (d_l - d_k).
    """
    zeros = np.asarray(zeros, dtype=np.float64)
    poles = np.asarray(poles, dtype=np.float64)
    c0 = K if zeros.size == poles.size else 0.0
    res = np.empty(poles.size)
    for k, dk in enumerate(poles):
        num = np.prod(zeros - dk)
        den = np.prod(np.delete(poles, k) - dk)
        res[k] = K * num / den
    return c0, res


def zolotarev_inv_sqrt(n, lo, hi, with_c0=True):
    """Best relative rational approximation of x^{-1/2} on [lo, hi].

    Type (n, n) when with_c0, else (n-1, n).  Returns (c0, residues, poles, err)
    where err is the maximal relative error max |sqrt(x) r(x) - 1|.
    """
    kappa = hi / lo
    mprime = 1.0 - 1.0 / kappa
    Kp = special.ellipk(mprime)
    M = 2 * n + 1 if with_c0 else 2 * n
    l = np.arange(1, M)
    sn, cn, _, _ = special.ellipj(l * Kp / M, mprime)
    c = sn ** 2 / cn ** 2  # c[l-1] = c_l
    poles_u = c[0::2][:n]  # c_1, c_3, ... (n of them)
    zeros_u = c[1::2]  # c_2, c_4, ... (n or n-1 of them)
    # unnormalised g(x) = sqrt(x) prod(...) on [1, kappa]; D = 2 / (g_min + g_max)
    def g(xt):
        xt = np.asarray(xt, dtype=np.float64)
        v = np.sqrt(xt)
        for e in zeros_u:
            v = v * (xt + e)
        for d in poles_u:
            v = v / (xt + d)
        return v

    grid = np.exp(np.linspace(0.0, np.log(kappa), 20000))
    gg = g(grid)
    D_est = 2.0 / (gg.min() + gg.max())  # grid estimate, so that D_est g - 1 alternates in sign
    ext = error_extrema(lambda xt: D_est * g(xt) - 1.0, 1.0, kappa)
    gv = np.array([g(xe) for xe, _ in ext])
    D = 2.0 / (gv.min() + gv.max())
    err = (gv.max() - gv.min()) / (gv.max() + gv.min())
    # back to [lo, hi]: x = lo * xt
    zeros = lo * zeros_u
    poles = lo * poles_u
    K = D * lo ** -0.5 * lo ** (poles.size - zeros.size)
    c0, res = product_to_partial_fractions(K, zeros, poles)
    return c0, res, poles, err


def error_extrema(err, lo, hi, ngrid=20000, floor=1e-3):
    """Alternating extrema of err(x) on [lo, hi], refined by a bounded scalar search.

    The grid (logarithmic, since the intervals span several decades) is cut into
    maximal runs of one sign; each run contributes its extreme point.  Runs whose
    peak is below `floor` times the largest peak are rounding noise around a zero
    crossing and are merged away.  Returns a list of (x, err(x)) in increasing x.
    """
    xs = np.exp(np.linspace(np.log(lo), np.log(hi), ngrid))
    e = err(xs)
    sg = np.sign(e)
    runs = []  # (start, stop) index ranges of constant sign
    start = 0
    for i in range(1, ngrid + 1):
        if i == ngrid or sg[i] != sg[start]:
            runs.append((start, i))
            start = i
    peak = max(np.max(np.abs(e[a:b])) for a, b in runs)
    kept = [(a, b) for a, b in runs if np.max(np.abs(e[a:b])) >= floor * peak]
    merged = []
    for a, b in kept:
        if merged and sg[merged[-1][0]] == sg[a]:
            merged[-1] = (merged[-1][0], b)
        else:
            merged.append((a, b))
    out = []
    for a, b in merged:
        i = a + int(np.argmax(np.abs(e[a:b])))
        sgn = sg[i]
        if i == 0 or i == ngrid - 1:
            out.append((float(xs[i]), float(e[i])))
            continue
        f = lambda u: -sgn * float(err(np.array([np.exp(u)]))[0])
        sol = optimize.minimize_scalar(
            f, bounds=(np.log(xs[i - 1]), np.log(xs[i + 1])), method="bounded", options=dict(xatol=1e-14))
        xe = float(np.exp(sol.x))
        out.append((xe, float(err(np.array([xe]))[0])))
    return out


def relative_error(c0, residues, poles, power, x):
    """r(x) / x^power - 1."""
    x = np.asarray(x, dtype=np.float64)
    return rational_eval(c0, residues, poles, x) / x ** power - 1.0


def max_relative_error(c0, residues, poles, power, lo, hi):
    ext = error_extrema(lambda x: relative_error(c0, residues, poles, power, x), lo, hi)
    return max(abs(v) for _, v in ext)
