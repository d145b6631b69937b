"""Pins for oracle/lattice.py: brute-force enumeration on small asymmetric lattices (Section 2, Section 3.2)."""
import itertools

import numpy as np
import pytest

from oracle import lattice

DIMS = [(2, 2, 2, 2), (4, 6, 2, 4), (6, 2, 4, 2)]


@pytest.mark.parametrize("dims", DIMS)
def test_half_index_is_address_shifted(dims):
    # Within each parity the lexicographic rank of a site equals l >> 1 (needs even N_x);
    # the CUDA path relies on this closed form.
    hidx = lattice.half_index(dims)
    l = np.arange(int(np.prod(dims)))
    assert np.array_equal(hidx, l >> 1)
    for p in (0, 1):
        assert lattice.sites_of_parity(dims, p).size == l.size // 2


@pytest.mark.parametrize("dims", DIMS)
def test_tables_against_brute_force(dims):
    nx, ny, nz, nt = dims
    fwd, bwd, sfwd, sbwd = lattice.neighbour_tables(dims)
    count = {0: 0, 1: 0}
    rank = {}
    for t, z, y, x in itertools.product(range(nt), range(nz), range(ny), range(nx)):
        p = (x + y + z + t) % 2
        rank[(x, y, z, t)] = count[p]
        count[p] += 1
    for (x, y, z, t), i in rank.items():
        p = (x + y + z + t) % 2
        c = [x, y, z, t]
        for mu in range(4):
            up = list(c)
            up[mu] = (up[mu] + 1) % dims[mu]
            dn = list(c)
            dn[mu] = (dn[mu] - 1) % dims[mu]
            assert fwd[p, mu, i] == rank[tuple(up)]
            assert bwd[p, mu, i] == rank[tuple(dn)]
            eta = [1, (-1) ** x, (-1) ** (x + y), (-1) ** (x + y + z)][mu]
            bc_up = -1 if (mu == 3 and t == nt - 1) else 1
            bc_dn = -1 if (mu == 3 and t == 0) else 1
            assert sfwd[p, mu, i] == eta * bc_up
            assert sbwd[p, mu, i] == eta * bc_dn


@pytest.mark.parametrize("dims", DIMS)
def test_tables_are_involutive_and_balanced(dims):
    fwd, bwd, _, _ = lattice.neighbour_tables(dims)
    Vh = int(np.prod(dims)) // 2
    for p in (0, 1):
        for mu in range(4):
            assert np.array_equal(bwd[1 - p, mu][fwd[p, mu]], np.arange(Vh))
            assert np.array_equal(fwd[1 - p, mu][bwd[p, mu]], np.arange(Vh))
        # every site of the other parity is hit exactly 4 times forward and 4 times backward
        assert np.all(np.bincount(fwd[p].reshape(-1), minlength=Vh) == 4)
        assert np.all(np.bincount(bwd[p].reshape(-1), minlength=Vh) == 4)


def test_eta_is_invariant_along_its_own_direction():
    # eta_mu(x +- mu) = eta_mu(x): the backward hop can reuse the site's own phase.
    dims = (4, 6, 2, 4)
    for mu in range(4):
        e = lattice.eta(mu, dims)
        assert np.array_equal(e[lattice.neighbour(dims, mu, +1)], e)
