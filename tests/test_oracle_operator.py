"""Pins for oracle/staggered.py and the input generator (Section 3.2).

Closed forms and invariants only: the free-field spectrum, anti-hermiticity of the
hopping blocks, hermiticity and the spectral bounds of A, gauge covariance.
"""
import itertools

import numpy as np
import pytest

from oracle import lattice, staggered
from paper_1710_09178_gb300 import inputs


def _plane_wave(dims, n, v):
    """e^{i p.x} v on the full lattice, p_mu = 2 pi n_mu / N_mu (x,y,z), 2 pi (n_t + 1/2)/N_t (t)."""
    x, y, z, t = lattice.coords(dims)
    p = [2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1], 2 * np.pi * n[2] / dims[2],
         2 * np.pi * (n[3] + 0.5) / dims[3]]
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[:, None] * v[None, :], p


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 4)])
def test_free_field_spectrum(dims):
    # U = 1: even-site restriction of e^{ipx} v is an eigenvector of -D_eo D_oe with eigenvalue sum sin^2 p_mu.
    U = inputs.unit_gauge_field(dims)
    rng = np.random.default_rng(0)
    v = rng.normal(size=3) + 1j * rng.normal(size=3)
    for n in itertools.product(*(range(d) for d in dims)):
        full, p = _plane_wave(dims, n, v)
        psi = staggered.restrict(full, dims, 0)
        out = -staggered.D_eo(U, staggered.D_oe(U, psi, dims), dims)
        lam = sum(np.sin(pm) ** 2 for pm in p)
        assert np.max(np.abs(out - lam * psi)) < 1e-13


def test_free_field_without_half_or_with_periodic_t_fails():
    # the pin above is sensitive to the 1/2 and to the antiperiodic t boundary
    dims = (4, 4, 4, 4)
    U = inputs.unit_gauge_field(dims)
    v = np.array([1.0, 0.5j, -0.25])
    full, p = _plane_wave(dims, (1, 2, 3, 0), v)
    psi = staggered.restrict(full, dims, 0)
    out = -staggered.D_eo(U, staggered.D_oe(U, psi, dims), dims)
    lam = sum(np.sin(pm) ** 2 for pm in p)
    assert np.max(np.abs(out - 4 * lam * psi)) > 1e-3
    p_per = p[:3] + [2 * np.pi * 0 / 4]
    assert abs(sum(np.sin(pm) ** 2 for pm in p_per) - lam) > 1e-3


@pytest.fixture(scope="module")
def field44():
    dims = (4, 4, 4, 4)
    return dims, inputs.gauge_field(dims, seed=1)


def test_generated_links_are_su3(field44):
    dims, U = field44
    M = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(np.conj(np.transpose(M, (0, 2, 1))) @ M - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(M) - 1)) < 1e-14
    # not close to the identity: the fields are genuinely rough
    assert np.mean(np.abs(M - eye)) > 0.1


def test_antihermiticity(field44):
    # <chi_o, D_oe psi_e> = -<D_eo chi_o, psi_e>, i.e. D_oe^dagger = -D_eo
    dims, U = field44
    psi = inputs.gaussian_vector(dims, 11)
    chi = inputs.gaussian_vector(dims, 12)
    lhs = np.vdot(chi, staggered.D_oe(U, psi, dims))
    rhs = -np.vdot(staggered.D_eo(U, chi, dims), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_A_hermitian_and_bounded(field44):
    dims, U = field44
    m = 0.1
    A = staggered.dense_A(U, m, dims)
    assert np.max(np.abs(A - A.conj().T)) < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 4 * m * m - 1e-12
    assert ev.max() <= 16 + 4 * m * m + 1e-12


def test_gauge_covariance(field44):
    # D[U'](g psi) = g D[U] psi with U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger
    dims, U = field44
    g = inputs.random_gauge_transform(dims, seed=99)
    Up = staggered.gauge_transform(U, g, dims)
    psi = inputs.gaussian_vector(dims, 13)
    ge = g[lattice.sites_of_parity(dims, 0)]
    go = g[lattice.sites_of_parity(dims, 1)]
    lhs = staggered.D_oe(Up, np.einsum("xab,xb->xa", ge, psi), dims)
    rhs = np.einsum("xab,xb->xa", go, staggered.D_oe(U, psi, dims))
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    A1 = staggered.A_apply(Up, np.einsum("xab,xb->xa", ge, psi), 0.1, dims)
    A0 = np.einsum("xab,xb->xa", ge, staggered.A_apply(U, psi, 0.1, dims))
    assert np.max(np.abs(A1 - A0)) < 1e-13


def test_gaussian_vector_moments():
    dims = (16, 16, 16, 8)
    xi = inputs.gaussian_vector(dims, 4)
    re = xi.real.reshape(-1)
    im = xi.imag.reshape(-1)
    n = re.size
    assert abs(re.mean()) < 5 / np.sqrt(n) and abs(im.mean()) < 5 / np.sqrt(n)
    assert abs(re.var() - 0.5) < 0.02 and abs(im.var() - 0.5) < 0.02
    assert abs(np.mean(re * im)) < 5 * 0.5 / np.sqrt(n)
