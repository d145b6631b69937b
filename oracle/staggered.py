"""Staggered Dirac operator and its even-odd blocks (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.2 writes the staggered matrix as M = 2m + sum_mu (U_mu(x) delta_{x+mu,k}
- U_mu(x-mu)^dagger delta_{x-mu,k}) with the phases absorbed into U, and splits it
into the blocks [[m_oo, D_oe], [D_eo, m_ee]] after grouping odd and even sites;
the half-lattice operator (M^dagger M)_ee = m_ee^2 + D_eo^dagger D_oe.

Normalisation used throughout (it differs from Section 3.2 only by rescaling the
hopping term): the hopping operator carries a factor 1/2 and explicit phases,

    (D psi)(x) = 1/2 sum_mu eta_mu(x) [ U_mu(x) psi(x+mu) - U_mu(x-mu)^dagger psi(x-mu) ],

with the t-boundary sign on hops that wrap in t, and M = 2m + D, so that on even
sites A = (M^dagger M)_ee = 4m^2 - D_eo D_oe (D^dagger = -D, hence D_eo^dagger = -D_oe).
D_oe maps even-site vectors to odd sites and D_eo odd to even (row index first,
as in the block matrix of Section 3.2).

Layouts: gauge U is (V, 4, 3, 3) complex128 [site][mu][row][col]; full-lattice
vectors are (V, 3); half-lattice vectors are (V/2, 3) in the order of
lattice.sites_of_parity.
"""
from __future__ import annotations

import numpy as np

from . import lattice


def dslash_full(U, psi, dims):
    """(D psi)(x) on the whole lattice, written out term by term from the formula above."""
    V = int(np.prod(dims))
    assert U.shape == (V, 4, 3, 3) and psi.shape == (V, 3)
    out = np.zeros((V, 3), dtype=np.complex128)
    for mu in range(4):
        eta = lattice.eta(mu, dims)
        xf = lattice.neighbour(dims, mu, +1)
        xb = lattice.neighbour(dims, mu, -1)
        bf = lattice.boundary_sign(dims, mu, +1)
        bb = lattice.boundary_sign(dims, mu, -1)
        # U_mu(x) psi(x + mu)
        fwd = np.einsum("xab,xb->xa", U[:, mu], psi[xf]) * bf[:, None]
        # U_mu(x - mu)^dagger psi(x - mu): (U^dagger)_{ab} = conj(U_{ba})
        bwd = np.einsum("xba,xb->xa", np.conj(U[xb, mu]), psi[xb]) * bb[:, None]
        out += 0.5 * eta[:, None] * (fwd - bwd)
    return out


def embed(half, dims, p):
    """Full-lattice vector that equals `half` on parity p and zero elsewhere."""
    V = int(np.prod(dims))
    full = np.zeros((V, 3), dtype=np.complex128)
    full[lattice.sites_of_parity(dims, p)] = half
    return full


def restrict(full, dims, p):
    """The parity-p part of a full-lattice vector, in half-lattice order."""
    return full[lattice.sites_of_parity(dims, p)]


def dslash_eo(U, psi_in, dims, out_parity):
    """Half-lattice hop: out_parity=1 gives D_oe psi_e, out_parity=0 gives D_eo psi_o."""
    return restrict(dslash_full(U, embed(psi_in, dims, 1 - out_parity), dims), dims, out_parity)


def D_oe(U, psi_e, dims):
    return dslash_eo(U, psi_e, dims, 1)


def D_eo(U, psi_o, dims):
    return dslash_eo(U, psi_o, dims, 0)


def A_apply(U, psi_e, mass, dims, sigma=0.0):
    """(A + sigma) psi_e with A = 4 m^2 - D_eo D_oe on even sites."""
    return (4.0 * mass * mass + sigma) * psi_e - D_eo(U, D_oe(U, psi_e, dims), dims)


def dense_A(U, mass, dims):
    """Dense matrix of A on even sites (for lattices with V/2*3 up to a few hundred)."""
    Vh = int(np.prod(dims)) // 2
    n = 3 * Vh
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = A_apply(U, e.reshape(Vh, 3), mass, dims).reshape(n)
    return A


def gauge_transform(U, g, dims):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger for a site field g of shape (V, 3, 3)."""
    Up = np.empty_like(U)
    for mu in range(4):
        xf = lattice.neighbour(dims, mu, +1)
        Up[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[xf], (0, 2, 1)))
    return Up
