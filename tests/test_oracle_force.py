"""Pins for oracle/force.py: central finite differences of S_f, gauge covariance, algebra structure.

S_f = phi^dagger r(A) phi with r from Eq. ratapprx; the force is the derivative with respect to
U_mu(x) -> exp(i w^a lambda^a / 2) U_mu(x), dS_f/dw^a = tr(lambda^a F_mu(x)) (Section 3.1 MD
equations need it).
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import force, lattice, rational, staggered
from paper_1710_09178_gb300 import inputs


@pytest.mark.parametrize("dims,mass,n", [((2, 2, 2, 2), 0.1, 6), ((4, 2, 2, 4), 0.05, 8)])
def test_force_matches_finite_differences(dims, mass, n):
    U = inputs.gauge_field(dims, seed=3)
    phi = inputs.gaussian_vector(dims, 4)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(n, 4 * mass ** 2, 16 + 4 * mass ** 2)
    Fa = force.force_components(force.fermion_force(U, phi, mass, dims, c0, res, poles))
    lam = force.gell_mann()
    rng = np.random.default_rng(1)
    V = int(np.prod(dims))
    eps = 1e-5
    for _ in range(10):
        l, mu, a = int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(8))

        def S(w):
            U2 = U.copy()
            U2[l, mu] = expm(1j * w * lam[a] / 2) @ U[l, mu]
            return force.action_dense(U2, phi, mass, dims, c0, res, poles)

        fd = (S(eps) - S(-eps)) / (2 * eps)
        assert abs(fd - Fa[l, mu, a]) <= 2e-8 * max(abs(fd), 1e-2)


def test_force_is_traceless_hermitian_and_gauge_covariant():
    dims, mass = (4, 4, 4, 4), 0.1
    U = inputs.gauge_field(dims, seed=5)
    phi = inputs.gaussian_vector(dims, 6)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(8, 4 * mass ** 2, 16 + 4 * mass ** 2)
    F = force.fermion_force(U, phi, mass, dims, c0, res, poles)
    assert np.max(np.abs(F - np.conj(np.swapaxes(F, -1, -2)))) < 1e-14
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-14
    # U' = g U g(x+mu)^dagger, phi' = g phi  =>  F'_mu(x) = g(x) F_mu(x) g(x)^dagger
    g = inputs.random_gauge_transform(dims, seed=7)
    Up = staggered.gauge_transform(U, g, dims)
    ge = g[lattice.sites_of_parity(dims, 0)]
    Fp = force.fermion_force(Up, np.einsum("xab,xb->xa", ge, phi), mass, dims, c0, res, poles)
    expect = np.einsum("xab,xmbc,xdc->xmad", g, F, np.conj(g))
    assert np.max(np.abs(Fp - expect)) < 1e-10 * np.max(np.abs(F))


def test_action_shifted_cg_equals_dense():
    dims, mass = (4, 2, 2, 4), 0.05
    U = inputs.gauge_field(dims, seed=8)
    phi = inputs.gaussian_vector(dims, 9)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(8, 4 * mass ** 2, 16 + 4 * mass ** 2)
    a = force.action(U, phi, mass, dims, c0, res, poles)
    b = force.action_dense(U, phi, mass, dims, c0, res, poles)
    assert abs(a - b) < 1e-10 * abs(b)
