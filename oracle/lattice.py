"""Lattice geometry: site address, even/odd split, neighbours, staggered phases (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2 labels a site by four integers and gives it the address
l = (((i_t-1)N_z + (i_z-1))N_y + (i_y-1))N_x + i_x with 1-based coordinates; with
0-based coordinates that is l = x + N_x*(y + N_y*(z + N_z*t)).

Section 3.2 splits the sites into even and odd and regroups the lattice "so that
the even sites and odd sites are grouped together" (figure "evenodd" shows a
checkerboard).  Reading taken here: a site is even when x+y+z+t is even (the
checkerboard of the figure; the parity of l alone would not make D connect only
opposite parities when N_x is even).  Within one parity the sites keep their
lexicographic order; the position of a site in that ordered list is its
half-lattice index.

Staggered phases (absorbed into the links in Section 3.2; explicit in the
operator used here): eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
eta_t = (-1)^(x+y+z); boundary conditions periodic in x, y, z and antiperiodic
in t (a hop across the t boundary carries an extra factor -1).
"""
from __future__ import annotations

import numpy as np


def coords(dims):
    """0-based coordinates (x, y, z, t) of every site, ordered by address l."""
    nx, ny, nz, nt = dims
    l = np.arange(nx * ny * nz * nt)
    x = l % nx
    y = (l // nx) % ny
    z = (l // (nx * ny)) % nz
    t = l // (nx * ny * nz)
    return x, y, z, t


def address(x, y, z, t, dims):
    """Section 2 site address with 0-based coordinates (periodic wrap applied)."""
    nx, ny, nz, nt = dims
    return (x % nx) + nx * ((y % ny) + ny * ((z % nz) + nz * (t % nt)))


def parity(dims):
    """0 for even sites, 1 for odd sites (checkerboard reading)."""
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def sites_of_parity(dims, p):
    """Addresses l of the sites of parity p, in increasing l (the half-lattice order)."""
    return np.nonzero(parity(dims) == p)[0]


def half_index(dims):
    """For every site l, its position within the ordered list of its own parity."""
    V = int(np.prod(dims))
    idx = np.empty(V, dtype=np.int64)
    for p in (0, 1):
        s = sites_of_parity(dims, p)
        idx[s] = np.arange(s.size)
    return idx


def eta(mu, dims):
    """Staggered phase eta_mu(x) for every site, as +-1 integers."""
    x, y, z, t = coords(dims)
    if mu == 0:
        return np.ones_like(x)
    if mu == 1:
        return (-1) ** x
    if mu == 2:
        return (-1) ** (x + y)
    if mu == 3:
        return (-1) ** (x + y + z)
    raise ValueError(mu)


def neighbour(dims, mu, step):
    """Address of x + step*mu_hat for every site (periodic wrap of the address)."""
    x, y, z, t = coords(dims)
    c = [x, y, z, t]
    c[mu] = c[mu] + step
    return address(*c, dims)


def boundary_sign(dims, mu, step):
    """-1 where a hop x -> x + step*mu_hat crosses the t boundary, else +1."""
    _, _, _, t = coords(dims)
    s = np.ones(int(np.prod(dims)), dtype=np.int64)
    if mu == 3:
        nt = dims[3]
        if step == +1:
            s[t == nt - 1] = -1
        else:
            s[t == 0] = -1
    return s


def neighbour_tables(dims):
    """Half-lattice neighbour tables of both parities.

    Returns (fwd, bwd, sfwd, sbwd), each an int array of shape (2, 4, V/2):
      fwd[p, mu, i]  half index (in parity 1-p) of x + mu_hat for the i-th site x of parity p
      bwd[p, mu, i]  half index of x - mu_hat
      sfwd[p, mu, i] eta_mu(x) times the boundary sign of the hop x -> x + mu_hat
      sbwd[p, mu, i] eta_mu(x - mu_hat) times the boundary sign of the hop x -> x - mu_hat
    """
    V = int(np.prod(dims))
    Vh = V // 2
    hidx = half_index(dims)
    fwd = np.empty((2, 4, Vh), dtype=np.int64)
    bwd = np.empty((2, 4, Vh), dtype=np.int64)
    sfwd = np.empty((2, 4, Vh), dtype=np.int64)
    sbwd = np.empty((2, 4, Vh), dtype=np.int64)
    for p in (0, 1):
        s = sites_of_parity(dims, p)
        for mu in range(4):
            nf = neighbour(dims, mu, +1)
            nb = neighbour(dims, mu, -1)
            fwd[p, mu] = hidx[nf[s]]
            bwd[p, mu] = hidx[nb[s]]
            sfwd[p, mu] = eta(mu, dims)[s] * boundary_sign(dims, mu, +1)[s]
            sbwd[p, mu] = eta(mu, dims)[nb[s]] * boundary_sign(dims, mu, -1)[s]
    return fwd, bwd, sfwd, sbwd
