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
    cuts = np.nonzero(sg[1:] != sg[:-1])[0] + 1  # maximal runs of constant sign
    bounds = np.concatenate([[0], cuts, [ngrid]])
    runs = list(zip(bounds[:-1].tolist(), bounds[1:].tolist()))
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


# ---------------------------------------------------------------------------------------------
# Exchange (Remez) algorithm for x^power, power in (-1, 0), and its reciprocal for (0, 1).
#
# Reading: the Appendix uses Mathematica's MiniMaxApproximation (a Remez-type exchange) at
# 1000 digits.  Here the same characterisation is reached in double precision by working with
# the product form R(x) = C prod_l (x + z_l) / (x + p_l) and the logarithmic error
# E(x) = log R(x) - power log x, whose minimax solution agrees with the relative-error one to
# second order in the error (|log(1+e) - e| ~ e^2 / 2, i.e. ~1e-22 here).  Steps:
#   1. start from Zolotarev's solution for power = -1/2 and its alternation points;
#   2. move power in small steps towards the target; at each step
#      a. Newton-solve E(x_i) = (-1)^i eta at the 2n+2 reference points for (log C, log z_l,
#         log p_l, eta),
#      b. replace the reference points by the 2n+2 alternating extrema of E (exchange),
#      repeating a-b until the extrema are level;
#   3. for a positive target power, take the reciprocal of the solution for -power: zeros and
#      poles swap and C -> 1/C (the logarithmic error just changes sign).
# ---------------------------------------------------------------------------------------------
def _log_error(logC, z, p, power, x):
    x = np.asarray(x, dtype=np.float64)
    prod = np.full_like(x, np.exp(logC))
    for zl, pl in zip(z, p):
        prod = prod * ((x + zl) / (x + pl))
    return np.log(prod) - power * np.log(x)


def _newton_level(logC, z, p, power, xs, iters=30):
    """Solve E(x_i) = (-1)^i eta for the 2n+2 reference points by Newton's method."""
    n = z.size
    sgn = (-1.0) ** np.arange(xs.size)
    eta = 0.0
    u = np.concatenate([[logC], np.log(z), np.log(p), [eta]])
    for _ in range(iters):
        logC, lz, lp, eta = u[0], u[1:n + 1], u[n + 1:2 * n + 1], u[-1]
        z, p = np.exp(lz), np.exp(lp)
        F = _log_error(logC, z, p, power, xs) - sgn * eta
        J = np.empty((xs.size, 2 * n + 2))
        J[:, 0] = 1.0
        J[:, 1:n + 1] = z[None, :] / (xs[:, None] + z[None, :])
        J[:, n + 1:2 * n + 1] = -p[None, :] / (xs[:, None] + p[None, :])
        J[:, -1] = -sgn
        du = np.linalg.solve(J, -F)
        u = u + du
        if np.max(np.abs(du[:-1])) < 1e-14:
            break
    return u[0], np.exp(u[1:n + 1]), np.exp(u[n + 1:2 * n + 1]), u[-1]


def remez_power(power, lo, hi, n, steps=None, tol_level=1e-3, max_exchange=40):
    """Best relative (n, n) rational approximation of x^power on [lo, hi], -1 < power < 1.

    Returns (c0, residues, poles, err) with r(x) = c0 + sum_k residues[k] / (x + poles[k])
    and err = max_x |r(x) / x^power - 1|.
    """
    if not (-1.0 < power < 1.0) or power == 0.0:
        raise ValueError("power must lie in (-1, 0) or (0, 1)")
    target = -abs(power)
    # 1. Zolotarev start for -1/2
    c0, res, poles, _ = zolotarev_inv_sqrt(n, lo, hi)
    poles = np.sort(poles)
    # zeros of R from the partial fractions: recover them as the roots of the numerator by
    # using the closed form again (zeros interlace the poles)
    kappa = hi / lo
    mprime = 1.0 - 1.0 / kappa
    Kp = special.ellipk(mprime)
    l = np.arange(1, 2 * n + 1)
    sn, cn, _, _ = special.ellipj(l * Kp / (2 * n + 1), mprime)
    c = sn ** 2 / cn ** 2
    z = lo * c[1::2]
    p = lo * c[0::2]
    logC = np.log(c0)
    ext = error_extrema(lambda x: _log_error(logC, z, p, -0.5, x), lo, hi, floor=0.1)
    xs = np.array([x for x, _ in ext])
    # 2. continuation in the power
    nsteps = steps if steps is not None else max(1, int(round(abs(target + 0.5) / 0.025)))
    path = np.linspace(-0.5, target, nsteps + 1)[1:] if target != -0.5 else np.array([-0.5])
    for step, pw in enumerate(path):
        final = step == len(path) - 1
        for _ in range(max_exchange if final else 4):
            logC, z, p, eta = _newton_level(logC, z, p, pw, xs)
            # floor 0.1: the true extrema are within a small factor of each other, while rounding
            # noise of the ~1e-13 errors of the largest cases makes spurious sign runs near zeros
            ext = error_extrema(lambda x: _log_error(logC, z, p, pw, x), lo, hi, floor=0.1)
            vals = np.abs([v for _, v in ext])
            if len(ext) == 2 * n + 2:
                new = np.array([x for x, _ in ext])
                moved = np.max(np.abs(np.log(new / xs)))
                xs = new
                # level, or the reference no longer moves (rounding noise limits the levelling)
                if vals.max() / vals.min() - 1 < tol_level or moved < 1e-5:
                    break
    # 3. reciprocal for a positive power
    if power > 0:
        logC, z, p = -logC, p, z
    order = np.argsort(p)
    z, p = z, p[order]
    C = np.exp(logC)
    c0, res = product_to_partial_fractions(C, z, p)
    err = max_relative_error(c0, res, p, power, lo, hi)
    return c0, res, p, err
