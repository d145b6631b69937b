"""Conjugate gradient and shifted (multi-shift) conjugate gradient (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 4: the rational approximation turns (M^dagger M)^{1/b} phi into
c_0 phi + sum_k c_k (A + d_k)^{-1} phi, and all the shifted systems are solved
with one shifted conjugate gradient (ref. [mcg], Jegerlehner, hep-lat/9612014)
using as many shifts as there are coefficients.

The shifted CG below runs the ordinary CG on the base system A + sigma_0 with
sigma_0 = min_k sigma_k, and carries the other systems along through the
collinearity r_k = zeta_k r of their residuals.  With s_k = sigma_k - sigma_0,
iteration j computes

    q        = (A + sigma_0) p
    alpha_j  = (r, r) / (p, q)
    zeta_k'  = zeta_k zeta_k_prev alpha_{j-1}
               / ( alpha_j beta_{j-1} (zeta_k_prev - zeta_k) + zeta_k_prev alpha_{j-1} (1 + s_k alpha_j) )
    alpha_k  = alpha_j zeta_k' / zeta_k,     x_k += alpha_k p_k
    r       -= alpha_j q,                    beta_j = (r, r)_new / (r, r)_old
    beta_k   = beta_j (zeta_k' / zeta_k)^2,  p_k = zeta_k' r + beta_k p_k
    p        = r + beta_j p

starting from x_k = 0, r = p = p_k = b, zeta = zeta_prev = 1, alpha_{-1} = 1,
beta_{-1} = 0.  Readings: shift k stops (its x_k, p_k freeze) once
|zeta_k| |r| <= tol |b|; the solve ends when every shift has stopped; with b = 0
every x_k is 0.
"""
from __future__ import annotations

import numpy as np


def vdot(a, b):
    """<a, b> = sum conj(a) b over all components."""
    return np.vdot(a.reshape(-1), b.reshape(-1))


def norm2(a):
    return float(np.real(vdot(a, a)))


def cg(apply, b, tol=1e-10, maxiter=20000):
    """Plain CG for a Hermitian positive operator; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = b.copy()
    rr = norm2(r)
    bb = rr
    if bb == 0.0:
        return x, 0
    it = 0
    while rr > tol * tol * bb and it < maxiter:
        q = apply(p)
        alpha = rr / float(np.real(vdot(p, q)))
        x = x + alpha * p
        r = r - alpha * q
        rr_new = norm2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def multishift_cg(apply_base, b, shifts, tol=1e-10, maxiter=20000, fixed_iters=None):
    """Shifted CG for (A + sigma_k) x_k = b, all k at once.

    apply_base(v) must return (A + min(shifts)) v.  If fixed_iters is given the
    loop runs exactly that many iterations with no shift frozen (used to compare
    implementations iteration for iteration).  Returns (xs, info) with xs a list
    of solutions in the order of `shifts` and info a dict holding 'iterations',
    'zeta' (final per-shift zeta), 'rr' (final |r|^2) and 'shift_iterations' (the
    number of (iteration, shift) pairs in which the shift was still updated).
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    n = shifts.size
    sigma0 = shifts.min()
    s = shifts - sigma0
    xs = [np.zeros_like(b) for _ in range(n)]
    bb = norm2(b)
    if bb == 0.0:
        return xs, dict(iterations=0, zeta=np.ones(n), rr=0.0, shift_iterations=0)
    r = b.copy()
    p = b.copy()
    ps = [b.copy() for _ in range(n)]
    zeta = np.ones(n)
    zeta_prev = np.ones(n)
    active = np.ones(n, dtype=bool)
    alpha_prev, beta_prev = 1.0, 0.0
    rr = bb
    it = 0
    shift_iterations = 0
    while True:
        if fixed_iters is not None:
            if it >= fixed_iters:
                break
        elif not active.any() or it >= maxiter:
            break
        shift_iterations += int(active.sum())
        q = apply_base(p)
        alpha = rr / float(np.real(vdot(p, q)))
        zeta_new = zeta.copy()  # a stopped shift keeps its last zeta
        for k in range(n):
            if active[k]:
                den = alpha * beta_prev * (zeta_prev[k] - zeta[k]) + zeta_prev[k] * alpha_prev * (1.0 + s[k] * alpha)
                zeta_new[k] = zeta[k] * zeta_prev[k] * alpha_prev / den
        for k in range(n):
            if active[k]:
                xs[k] = xs[k] + (alpha * zeta_new[k] / zeta[k]) * ps[k]
        r = r - alpha * q
        rr_new = norm2(r)
        beta = rr_new / rr
        for k in range(n):
            if active[k]:
                beta_k = beta * (zeta_new[k] / zeta[k]) ** 2
                ps[k] = zeta_new[k] * r + beta_k * ps[k]
        p = r + beta * p
        zeta_prev = np.where(active, zeta, zeta_prev)
        zeta = zeta_new
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
        it += 1
        if fixed_iters is None:
            for k in range(n):
                if active[k] and abs(zeta[k]) * np.sqrt(rr) <= tol * np.sqrt(bb):
                    active[k] = False
    return xs, dict(iterations=it, zeta=zeta.copy(), rr=rr, shift_iterations=shift_iterations)


def true_residuals(apply_shifted, b, xs, shifts):
    """|b - (A + sigma_k) x_k| / |b| for every k; apply_shifted(v, sigma) = (A + sigma) v."""
    nb = np.sqrt(norm2(b))
    return np.array([np.sqrt(norm2(b - apply_shifted(x, sg))) / nb for x, sg in zip(xs, shifts)])


def rational_apply(b, xs, c0, residues):
    """y = c0 b + sum_k c_k x_k (Eq. ratapprx with x_k = (A + d_k)^{-1} b)."""
    y = c0 * b
    for c, x in zip(residues, xs):
        y = y + c * x
    return y
