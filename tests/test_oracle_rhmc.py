"""Pins for oracle/rhmc.py (Section 3.1 trajectory): gauge-force finite differences, SU(3) of the
updated links, exact reversibility of the integrator, second-order energy error, heatbath/action
consistency (phi = r_{1/4}(A) xi gives phi^+ r_{-1/2}(A) phi = xi^+ xi up to the approximations)."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import force, rational, rhmc
from paper_1710_09178_gb300 import inputs

DIMS, MASS, BETA = (4, 4, 4, 4), 0.1, 5.4


def _coeffs(n=8):
    lo, hi = 4 * MASS ** 2, 16 + 4 * MASS ** 2
    act = rational.zolotarev_inv_sqrt(n, lo, hi)[:3]
    heat = rational.remez_power(0.25, lo, hi, n)[:3]
    return act, heat


def _momenta(seed):
    V = int(np.prod(DIMS))
    return inputs.counter_normal_pairs(seed, np.arange(4 * V, dtype=np.uint64), 4).reshape(V, 4, 8)


def test_gauge_force_matches_finite_differences():
    U = inputs.gauge_field(DIMS, seed=21)
    Fa = force.force_components(rhmc.gauge_force(U, BETA, DIMS))
    lam = force.gell_mann()
    rng = np.random.default_rng(3)
    for _ in range(8):
        l, mu, a = int(rng.integers(256)), int(rng.integers(4)), int(rng.integers(8))

        def S(w):
            U2 = U.copy()
            U2[l, mu] = expm(1j * w * lam[a] / 2) @ U[l, mu]
            return rhmc.gauge_action(U2, BETA, DIMS)

        fd = (S(1e-5) - S(-1e-5)) / 2e-5
        # S_g ~ 4e3 here: rounding of S(+-eps) alone is ~1e-12, i.e. ~5e-8 after dividing by 2 eps
        assert abs(fd - Fa[l, mu, a]) <= 5e-7 * max(1.0, abs(fd))


def test_gauge_action_of_unit_field_is_zero_and_link_update_stays_su3():
    assert abs(rhmc.gauge_action(inputs.unit_gauge_field(DIMS), BETA, DIMS)) < 1e-12
    U = inputs.gauge_field(DIMS, seed=22)
    U2 = rhmc.update_links(U, _momenta(5), 0.3)
    M = U2.reshape(-1, 3, 3)
    assert np.max(np.abs(np.conj(np.swapaxes(M, 1, 2)) @ M - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(M) - 1)) < 1e-14


@pytest.fixture(scope="module")
def setup():
    act_c, heat_c = _coeffs()
    U = inputs.gauge_field(DIMS, seed=23)
    xi = inputs.gaussian_vector(DIMS, 24)
    p = _momenta(25)
    act = rhmc.Action(DIMS, MASS, BETA, act_c, tol=1e-13)
    phi = rhmc.heatbath(U, xi, MASS, DIMS, heat_c, tol=1e-13)
    return U, p, xi, phi, act, act_c, heat_c


def test_heatbath_and_action_are_consistent(setup):
    U, p, xi, phi, act, act_c, heat_c = setup
    Sf = act.fermion_action(U, phi)
    xx = float(np.real(np.vdot(xi, xi)))
    assert abs(Sf - xx) <= 1e-8 * xx


def test_integrator_is_reversible(setup):
    U, p, xi, phi, act, _, _ = setup
    U1, p1 = rhmc.integrate(U, p, phi, act, 0.5, 4)
    U2, p2 = rhmc.integrate(U1, -p1, phi, act, 0.5, 4)
    assert np.max(np.abs(U2 - U)) < 1e-10
    assert np.max(np.abs(p2 + p)) < 1e-9


def test_energy_error_is_second_order(setup):
    U, p, xi, phi, act, _, _ = setup
    H0, _ = rhmc.hamiltonian(U, p, phi, act)
    dH = []
    for n in (4, 8):
        U1, p1 = rhmc.integrate(U, p, phi, act, 0.5, n)
        dH.append(rhmc.hamiltonian(U1, p1, phi, act)[0] - H0)
    ratio = abs(dH[0]) / abs(dH[1])
    assert 2.5 < ratio < 6.5, dH
