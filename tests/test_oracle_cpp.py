"""Pins for the C++ oracle (oracle/cpp/oracle.cpp), both builds (one core and OpenMP).

The C++ oracle is pinned the way the numpy oracle is -- brute-force geometry, the free-field
spectrum, anti-hermiticity, gauge covariance, hermiticity and spectral bounds of A, dense LU
solves, independent CG solves, collinearity of the shifted residuals, the 16-bit format's
rounding rules -- and it is compared element by element with the (separately pinned) numpy
oracle on small, ragged and mid-sized lattices.
"""
import itertools

import numpy as np
import pytest

from oracle import cpp_oracle, encode16, lattice, rational, solvers, staggered
from paper_1710_09178_gb300 import inputs


@pytest.fixture(scope="module", params=[False, True], ids=["serial", "omp"])
def orc(request):
    return cpp_oracle.load(threaded=request.param)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 2, 4), (6, 2, 4, 2)])
def test_tables_against_brute_force(orc, dims):
    nx, ny, nz, nt = dims
    lat = orc.lattice(dims, inputs.unit_gauge_field(dims), 0.1)
    fwd, bwd, sfwd, sbwd = lat.neighbour_tables()
    count = {0: 0, 1: 0}
    rank = {}
    for t, z, y, x in itertools.product(range(nt), range(nz), range(ny), range(nx)):
        p = (x + y + z + t) % 2
        rank[(x, y, z, t)] = count[p]
        count[p] += 1
    for (x, y, z, t), i in rank.items():
        p = (x + y + z + t) % 2
        for mu in range(4):
            up, dn = [x, y, z, t], [x, y, z, t]
            up[mu] = (up[mu] + 1) % dims[mu]
            dn[mu] = (dn[mu] - 1) % dims[mu]
            assert fwd[p, mu, i] == rank[tuple(up)]
            assert bwd[p, mu, i] == rank[tuple(dn)]
            eta = [1, (-1) ** x, (-1) ** (x + y), (-1) ** (x + y + z)][mu]
            assert sfwd[p, mu, i] == eta * (-1 if (mu == 3 and t == nt - 1) else 1)
            assert sbwd[p, mu, i] == eta * (-1 if (mu == 3 and t == 0) else 1)
    assert all(np.array_equal(a, b) for a, b in zip((fwd, bwd, sfwd, sbwd), lattice.neighbour_tables(dims)))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 4)])
def test_free_field_spectrum(orc, dims):
    # U = 1: the even-site part of e^{ipx} v is an eigenvector of -D_eo D_oe with eigenvalue sum_mu sin^2 p_mu
    lat = orc.lattice(dims, inputs.unit_gauge_field(dims), 0.0)
    x, y, z, t = lattice.coords(dims)
    v = np.array([0.3 - 1.1j, 0.7j, -0.45])
    even = lattice.sites_of_parity(dims, 0)
    for n in itertools.product(*(range(d) for d in dims)):
        p = [2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1], 2 * np.pi * n[2] / dims[2],
             2 * np.pi * (n[3] + 0.5) / dims[3]]
        psi = (np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[:, None] * v[None, :])[even]
        lam = sum(np.sin(pm) ** 2 for pm in p)
        out = -lat.D_eo(lat.D_oe(psi))
        assert np.max(np.abs(out - lam * psi)) < 1e-13
        # A = 4m^2 - D_eo D_oe with m = 0
        assert np.max(np.abs(lat.A_apply(psi, 0.25) - (lam + 0.25) * psi)) < 1e-13


@pytest.fixture(scope="module")
def field44():
    dims = (4, 4, 4, 4)
    return dims, inputs.gauge_field(dims, seed=1)


def test_antihermiticity(orc, field44):
    # <chi_o, D_oe psi_e> = -<D_eo chi_o, psi_e>
    dims, U = field44
    lat = orc.lattice(dims, U, 0.1)
    psi, chi = inputs.gaussian_vector(dims, 11), inputs.gaussian_vector(dims, 12)
    lhs = np.vdot(chi, lat.D_oe(psi))
    rhs = -np.vdot(lat.D_eo(chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_covariance(orc, field44):
    # U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger gives D[U'](g psi) = g D[U] psi and A[U'](g psi) = g A[U] psi
    dims, U = field44
    g = inputs.random_gauge_transform(dims, seed=99)
    Up = np.empty_like(U)
    for mu in range(4):
        xf = lattice.neighbour(dims, mu, +1)
        Up[:, mu] = np.einsum("xab,xbc,xdc->xad", g, U[:, mu], np.conj(g[xf]))
    lat, latp = orc.lattice(dims, U, 0.1), orc.lattice(dims, Up, 0.1)
    psi = inputs.gaussian_vector(dims, 13)
    ge, go = g[lattice.sites_of_parity(dims, 0)], g[lattice.sites_of_parity(dims, 1)]
    gpsi = np.einsum("xab,xb->xa", ge, psi)
    assert np.max(np.abs(latp.D_oe(gpsi) - np.einsum("xab,xb->xa", go, lat.D_oe(psi)))) < 1e-13
    assert np.max(np.abs(latp.A_apply(gpsi) - np.einsum("xab,xb->xa", ge, lat.A_apply(psi)))) < 1e-13


def test_A_hermitian_and_bounded(orc, field44):
    dims, U = field44
    m = 0.1
    lat = orc.lattice(dims, U, m)
    n = 3 * lat.Vh
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = lat.A_apply(e.reshape(lat.Vh, 3)).reshape(n)
    assert np.max(np.abs(A - A.conj().T)) < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 4 * m * m - 1e-12 and ev.max() <= 16 + 4 * m * m + 1e-12


@pytest.mark.parametrize("dims,mass", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 4), 0.1), ((4, 2, 2, 4), 0.05)])
def test_multishift_matches_dense_lu(orc, dims, mass):
    U, b = inputs.gauge_field(dims, seed=1), inputs.gaussian_vector(dims, 2)
    lat = orc.lattice(dims, U, mass)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    xs, info = lat.multishift_cg(b, poles, tol=1e-12)
    A = staggered.dense_A(U, mass, dims)
    for x, s in zip(xs, poles):
        As = A + s * np.eye(A.shape[0])
        xd = np.linalg.solve(As, b.reshape(-1))
        assert np.linalg.norm(x.reshape(-1) - xd) <= 10 * np.linalg.cond(As) * 1e-12 * np.linalg.norm(xd)
    assert info["iterations"] > 3


def test_multishift_equals_independent_cg(orc):
    dims, mass = (4, 4, 4, 4), 0.1
    U, b = inputs.gauge_field(dims, seed=1), inputs.gaussian_vector(dims, 2)
    lat = orc.lattice(dims, U, mass)
    shifts = np.array([0.002, 0.05, 0.3, 1.7, 9.0])
    xs, _ = lat.multishift_cg(b, shifts, tol=1e-12)
    for x, s in zip(xs, shifts):
        xc, _ = lat.cg(b, s, tol=1e-12)
        assert np.linalg.norm(x - xc) <= 1e-9 * np.linalg.norm(xc)
    assert np.all(lat.true_residuals(b, xs, shifts) < 2e-12)


@pytest.mark.parametrize("iters", [1, 2, 5, 12])
def test_shifted_residuals_are_collinear_with_the_base_residual(orc, iters):
    dims, mass = (4, 4, 2, 2), 0.1
    U, b = inputs.gauge_field(dims, seed=5), inputs.gaussian_vector(dims, 6)
    lat = orc.lattice(dims, U, mass)
    shifts = np.array([0.003, 0.04, 0.5, 2.0, 11.0])
    xs, info = lat.multishift_cg(b, shifts, fixed_iters=iters)
    k0 = int(np.argmin(shifts))
    r0 = b - lat.A_apply(xs[k0], shifts[k0])
    assert np.isclose(np.vdot(r0, r0).real, info["rr"], rtol=1e-10)
    nb = np.linalg.norm(b)
    for k, s in enumerate(shifts):
        assert np.linalg.norm(b - lat.A_apply(xs[k], s) - info["zeta"][k] * r0) <= 1e-12 * nb, (k, s)


def test_zero_source_gives_zero_solution(orc):
    dims = (2, 2, 2, 2)
    lat = orc.lattice(dims, inputs.gauge_field(dims, seed=1), 0.1)
    xs, info = lat.multishift_cg(np.zeros((8, 3), dtype=np.complex128), [0.1, 0.2])
    assert info["iterations"] == 0 and all(np.all(x == 0) for x in xs)


def test_rejects_odd_extents(orc):
    with pytest.raises(ValueError):
        orc.lattice((3, 2, 2, 2), np.zeros((24, 4, 3, 3), dtype=np.complex128), 0.1)


@pytest.mark.parametrize("dims,mass,npoles", [((4, 4, 4, 4), 0.1, 12), ((10, 6, 4, 6), 0.05, 14),
                                              ((8, 8, 8, 4), 0.02, 16)])
def test_equals_numpy_oracle(orc, dims, mass, npoles):
    # element by element against the numpy oracle: the hop and A in the same operation order (equal to
    # rounding), the shifted CG at a fixed iteration count and converged, true residuals, y
    U, b = inputs.gauge_field(dims, seed=3), inputs.gaussian_vector(dims, 4)
    lat = orc.lattice(dims, U, mass)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, b, dims, p)
        assert np.max(np.abs(lat.dslash_eo(b, p) - ref)) <= 1e-15 * np.max(np.abs(ref))
    ref = staggered.A_apply(U, b, mass, dims, 0.7)
    assert np.max(np.abs(lat.A_apply(b, 0.7) - ref)) <= 1e-14 * np.max(np.abs(ref))
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(npoles, 4 * mass ** 2, 16 + 4 * mass ** 2)
    base = lambda v: staggered.A_apply(U, v, mass, dims, poles.min())
    xs, info = lat.multishift_cg(b, poles, fixed_iters=15)
    xn, infn = solvers.multishift_cg(base, b, poles, fixed_iters=15)
    for a, c in zip(xs, xn):
        assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)
    assert np.allclose(info["zeta"], infn["zeta"], rtol=1e-12, atol=0)
    xs, info = lat.multishift_cg(b, poles, tol=1e-10)
    xn, infn = solvers.multishift_cg(base, b, poles, tol=1e-10)
    assert info["iterations"] == infn["iterations"]
    assert abs(info["shift_iterations"] - infn["shift_iterations"]) <= len(poles)
    tr = lat.true_residuals(b, xs, poles)
    trn = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, poles)
    assert np.allclose(tr, trn, rtol=1e-9, atol=0) and np.all(tr <= 1e-10)
    y = orc.rational_apply(b, xs, c0, res)
    yn = solvers.rational_apply(b, xs, c0, res)
    assert np.max(np.abs(y - yn)) <= 1e-15 * np.max(np.abs(yn))


def test_serial_and_threaded_builds_agree():
    # the OpenMP build only reorders the sums over sites
    dims, mass = (8, 8, 4, 4), 0.05
    U, b = inputs.gauge_field(dims, seed=2), inputs.gaussian_vector(dims, 3)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * mass ** 2, 16 + 4 * mass ** 2)
    out = []
    for thr in (False, True):
        lat = cpp_oracle.load(thr).lattice(dims, U, mass)
        out.append(lat.multishift_cg(b, poles, fixed_iters=30)[0])
    for a, c in zip(*out):
        assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)


def test_encode16_matches_numpy_and_rounds_half_to_even(orc):
    rng = np.random.default_rng(5)
    v = rng.normal(size=(4096, 6)).astype(np.float32) * np.float32(3.0)
    v[7] = 0.0
    v[8] = [1.0, -1.0, 0.5, -0.5, 0.25, 1e-30]
    q, s = orc.encode16(v)
    qn, sn = encode16.encode(v)
    assert np.array_equal(q, qn) and np.array_equal(s, sn)
    assert np.all(q[7] == 0) and s[7] == 0
    assert q[8, 0] == 32767 and q[8, 1] == -32767
    # 0.5 * 32767 = 16383.5 rounds to the even 16384
    assert q[8, 2] == 16384 and q[8, 3] == -16384
    dec = orc.decode16(q, s)
    assert np.array_equal(dec, encode16.decode(qn, sn))
    nrm = np.max(np.abs(v), axis=1)
    # |decode - v| <= s/2 plus float32 rounding of the scale products
    assert np.all(np.abs(dec - v) <= (0.5 * s + 4e-7 * nrm)[:, None])
    # components at (k + 1/2) / 32767 of the norm are exact float32 ties
    qt, _ = orc.encode16(np.array([[32767.0, 2.5, -3.5, 0.5, 1.5, -0.5]], dtype=np.float32))
    assert np.array_equal(qt[0], np.array([32767, 2, -4, 0, 2, 0], dtype=np.int16))


def test_full_size_solve_reproduces_the_numpy_oracle_record():
    # the 32^3 x 8 workload (16-pole x^{-1/2}, m = 0.02, tol 1e-10) solved by the numpy oracle once
    # (tests/golden/oracle_iterations_32c8.json, written by make_oracle_iterations.py): the C++ oracle
    # stops at the same iteration with the same true residuals up to rounding
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_iterations_32c8.json")) as f:
        rec = json.load(f)
    dims, mass = (32, 32, 32, 8), rec["mass"]
    U, b = inputs.gauge_field(dims, seed=rec["gauge_seed"]), inputs.gaussian_vector(dims, rec["source_seed"])
    c0, res, poles, err = rational.zolotarev_inv_sqrt(rec["poles"], 4 * mass ** 2, 16 + 4 * mass ** 2)
    lat = cpp_oracle.load(threaded=True).lattice(dims, U, mass)
    xs, info = lat.multishift_cg(b, poles, tol=rec["tol"])
    assert info["iterations"] == rec["iterations"]
    tr = lat.true_residuals(b, xs, poles)
    assert np.allclose(tr, rec["true_residuals"], rtol=1e-4, atol=0)
