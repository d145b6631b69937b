"""Fermion force of the pseudofermion action (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.1: the molecular-dynamics equations are dU/dt = i p U for the links and, from
dH/dt = 0, a momentum equation that needs the derivative of the action with respect to
the links.  For the pseudofermion action of Section 2/4,

    S_f = phi^dagger r(A) phi,   r(A) = c_0 + sum_k c_k (A + d_k)^{-1},   A = 4m^2 - D_eo D_oe,

a change of A gives d(phi^dagger (A + d_k)^{-1} phi) = -X_k^dagger dA X_k with
X_k = (A + d_k)^{-1} phi, and dA = -(dD_eo D_oe + D_eo dD_oe).  With Y_k = D_oe X_k and
D_eo = -D_oe^dagger:

    dS_f = sum_k c_k [ X_k^dagger dD_eo Y_k - Y_k^dagger dD_oe X_k ].

Link U_mu(x) enters D as 1/2 s [U psi(x+mu) at x] and -1/2 s [U^dagger psi(x) at x+mu]
(s = eta_mu(x) times the t-boundary sign).  Varying U -> exp(i w^a lambda^a/2) U gives
dS_f/dw^a = tr(lambda^a F_mu(x)) with the traceless Hermitian

    F = (H - tr(H)/3) / 2,   H = (i s / 2) (W - W^dagger),
    W = U sum_k c_k Y_k(x+mu) X_k(x)^dagger          (x even)
    W = -U sum_k c_k X_k(x+mu) Y_k(x)^dagger         (x odd)

(X_k lives on even sites, Y_k on odd sites).  The convention: the derivative with respect to
the real coordinates w^a of the left-multiplied algebra element, F_mu(x) its matrix form.
"""
from __future__ import annotations

import numpy as np

from . import lattice, staggered, solvers


def gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def action(U, phi, mass, dims, c0, residues, poles, tol=1e-13):
    """S_f = phi^dagger r(A) phi through the shifted CG (Eq. ratapprx)."""
    xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, min(poles)), phi, poles, tol=tol)
    y = solvers.rational_apply(phi, xs, c0, residues)
    return float(np.real(np.vdot(phi, y)))


def action_dense(U, phi, mass, dims, c0, residues, poles):
    """S_f with the matrix function formed densely (small lattices)."""
    A = staggered.dense_A(U, mass, dims)
    n = A.shape[0]
    v = phi.reshape(-1)
    y = c0 * v
    for c, d in zip(residues, poles):
        y = y + c * np.linalg.solve(A + d * np.eye(n), v)
    return float(np.real(np.vdot(v, y)))


def fermion_force(U, phi, mass, dims, c0, residues, poles, xs=None, tol=1e-13):
    """F_mu(x), shape (V, 4, 3, 3): dS_f/dw^a = tr(lambda^a F_mu(x)) for U_mu(x) -> exp(i w.lambda/2) U_mu(x)."""
    if xs is None:
        xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, min(poles)), phi, poles, tol=tol)
    V = int(np.prod(dims))
    # full-lattice Z_k: X_k on even sites, Y_k = D_oe X_k on odd sites
    Zs = []
    for x in xs:
        z = staggered.embed(x, dims, 0) + staggered.embed(staggered.D_oe(U, x, dims), dims, 1)
        Zs.append(z)
    par = lattice.parity(dims)
    F = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        xf = lattice.neighbour(dims, mu, +1)
        s = lattice.eta(mu, dims) * lattice.boundary_sign(dims, mu, +1)
        O = np.zeros((V, 3, 3), dtype=np.complex128)
        for c, z in zip(residues, Zs):
            # even x: c Y(x+mu) X(x)^dagger ; odd x: -c X(x+mu) Y(x)^dagger -- both are z(x+mu) z(x)^dagger
            O += c * np.einsum("xa,xb->xab", z[xf], np.conj(z))
        O[par == 1] *= -1
        W = U[:, mu] @ O
        H = 0.5j * s[:, None, None] * (W - np.conj(np.transpose(W, (0, 2, 1))))
        tr = np.trace(H, axis1=1, axis2=2)
        F[:, mu] = 0.5 * (H - tr[:, None, None] / 3 * np.eye(3))
    return F


def force_components(F):
    """Real components tr(lambda^a F), shape (..., 8)."""
    return np.real(np.einsum("aij,...ji->...a", gell_mann(), F))
