"""RHMC trajectory for two staggered flavours (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.1: a trajectory draws momenta p (conjugate to U) and a Gaussian xi, sets the
pseudofermion phi = (M^dagger M)^{alpha/2} xi (alpha = 1/2: the x^{1/4} rational approximation of
Eq. ratapprx), integrates the molecular-dynamics equations dU/dt = i p U and dH/dt = 0 with
H = 1/2 p^2 + S, and accepts with probability min(1, exp(-(H(tau) - H(0)))).
Section 2 (Eq. pfact): S = phi^dagger (M^dagger M)^{-1/2} phi + gauge action.

Readings (the paper is silent or loose on them):
  - momenta P = sum_a p^a lambda^a / 2 with p^a ~ N(0, 1), kinetic energy 1/2 sum p^a^2 = sum tr P^2;
  - Wilson gauge action S_g = beta sum_{x, mu<nu} (1 - Re tr U_plaq / 3) (the standard beta = 6/g^2);
  - U -> exp(i h P) U with h the position sub-step, followed by projection onto SU(3);
  - the integrator is Omelyan's second-order minimum-norm scheme (2MN), lambda = 0.1931833275037836:
      p -= lam eps F;  U <- e^{i eps/2 P} U;  p -= (1 - 2 lam) eps F;  U <- e^{i eps/2 P} U;  p -= lam eps F,
    with F^a = dS/dw^a for U -> exp(i w.lambda/2) U (so dp^a/dt = -F^a);
  - the Metropolis uniform number and all Gaussian numbers are inputs.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

from . import force as force_mod
from . import lattice, rational, solvers, staggered

OMELYAN_LAMBDA = 0.1931833275037836


def momenta_matrix(p):
    """(V, 4, 8) components -> (V, 4, 3, 3) traceless Hermitian P = sum p^a lambda^a / 2."""
    return np.einsum("lma,aij->lmij", p, force_mod.gell_mann() / 2)


def staples(U, dims):
    """A_mu(x) with sum over plaquettes through U_mu(x) of Re tr = Re tr(U_mu(x) A_mu(x))."""
    V = int(np.prod(dims))
    A = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    dag = lambda M: np.conj(np.swapaxes(M, -1, -2))
    for mu in range(4):
        xpmu = lattice.neighbour(dims, mu, +1)
        for nu in range(4):
            if nu == mu:
                continue
            xpnu = lattice.neighbour(dims, nu, +1)
            xmnu = lattice.neighbour(dims, nu, -1)
            xpmu_mnu = xmnu[xpmu]  # x + mu - nu
            up = U[xpmu, nu] @ dag(U[xpnu, mu]) @ dag(U[:, nu])
            down = dag(U[xpmu_mnu, nu]) @ dag(U[xmnu, mu]) @ U[xmnu, nu]
            A[:, mu] += up + down
    return A


def gauge_action(U, beta, dims):
    """S_g = beta sum_{x, mu < nu} (1 - Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ / 3)."""
    dag = lambda M: np.conj(np.swapaxes(M, -1, -2))
    S = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            xpmu = lattice.neighbour(dims, mu, +1)
            xpnu = lattice.neighbour(dims, nu, +1)
            P = U[:, mu] @ U[xpmu, nu] @ dag(U[xpnu, mu]) @ dag(U[:, nu])
            S += np.sum(1.0 - np.real(np.trace(P, axis1=1, axis2=2)) / 3.0)
    return beta * S


def gauge_force(U, beta, dims):
    """F_mu(x) traceless Hermitian with dS_g/dw^a = tr(lambda^a F) for U_mu(x) -> exp(i w.lambda/2) U_mu(x).

    S_g depends on U_mu(x) through -(beta/3) Re tr(U A) (each plaquette counted once in the sum
    over mu < nu appears in exactly one staple of every link it contains), so
    dS_g/dw^a = (beta/3) Im tr(lambda^a/2 U A), i.e. F = -(i beta/12) (W - W^+) made traceless,
    W = U A.
    """
    W = U @ staples(U, dims)
    F = -1j * beta / 12.0 * (W - np.conj(np.swapaxes(W, -1, -2)))
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - tr[..., None, None] / 3 * np.eye(3)


def reunitarize(U):
    """Gram-Schmidt on rows 0, 1 and row 2 = conj(row0 x row1) (SU(3) projection)."""
    r0 = U[..., 0, :] / np.linalg.norm(U[..., 0, :], axis=-1, keepdims=True)
    r1 = U[..., 1, :] - np.sum(np.conj(r0) * U[..., 1, :], axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def update_links(U, p, h):
    """U_mu(x) <- exp(i h P_mu(x)) U_mu(x), projected onto SU(3)."""
    X = 1j * h * momenta_matrix(p)
    E = expm(X.reshape(-1, 3, 3)).reshape(X.shape)
    return reunitarize(E @ U)


class Action:
    """H pieces and force for fixed rational approximations and pseudofermion."""

    def __init__(self, dims, mass, beta, act_coeffs, tol=1e-12):
        self.dims, self.mass, self.beta, self.tol = dims, mass, beta, tol
        self.c0, self.res, self.poles = act_coeffs

    def fermion_action(self, U, phi):
        return force_mod.action(U, phi, self.mass, self.dims, self.c0, self.res, self.poles, tol=self.tol)

    def force(self, U, phi):
        Ff = force_mod.fermion_force(U, phi, self.mass, self.dims, self.c0, self.res, self.poles, tol=self.tol)
        return force_mod.force_components(Ff + gauge_force(U, self.beta, self.dims))


def heatbath(U, xi, mass, dims, heat_coeffs, tol=1e-12):
    """phi = r_{1/4}(A) xi (Section 3.1, alpha/2 = 1/4)."""
    c0, res, poles = heat_coeffs
    xs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, min(poles)), xi, poles, tol=tol)
    return solvers.rational_apply(xi, xs, c0, res)


def hamiltonian(U, p, phi, act):
    kin = 0.5 * float(np.sum(p * p))
    Sg = gauge_action(U, act.beta, act.dims)
    Sf = act.fermion_action(U, phi)
    return kin + Sg + Sf, dict(kinetic=kin, gauge=Sg, fermion=Sf)


def integrate(U, p, phi, act, tau, nsteps, lam=OMELYAN_LAMBDA):
    """Omelyan 2MN from (U, p) over time tau in nsteps steps; returns (U, p)."""
    eps = tau / nsteps
    p = p - lam * eps * act.force(U, phi)
    for step in range(nsteps):
        U = update_links(U, p, 0.5 * eps)
        p = p - (1.0 - 2.0 * lam) * eps * act.force(U, phi)
        U = update_links(U, p, 0.5 * eps)
        w = 2.0 * lam if step < nsteps - 1 else lam  # merged end/start kicks of consecutive steps
        p = p - w * eps * act.force(U, phi)
    return U, p


def trajectory(U0, p0, xi, uniform, dims, mass, beta, tau, nsteps, act_coeffs, heat_coeffs, tol=1e-12):
    """One RHMC trajectory; returns (U_new, accepted, info)."""
    act = Action(dims, mass, beta, act_coeffs, tol=tol)
    phi = heatbath(U0, xi, mass, dims, heat_coeffs, tol=tol)
    H0, parts0 = hamiltonian(U0, p0, phi, act)
    U1, p1 = integrate(U0, p0, phi, act, tau, nsteps)
    H1, parts1 = hamiltonian(U1, p1, phi, act)
    dH = H1 - H0
    accepted = bool(uniform < np.exp(-dH))
    return (U1 if accepted else U0), accepted, dict(dH=dH, H0=H0, H1=H1, parts0=parts0, parts1=parts1, U1=U1,
                                                      p1=p1, phi=phi)
