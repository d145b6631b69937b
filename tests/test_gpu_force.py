"""GPU parity of the fermion force (adjoint kernel, csrc/force.cu) against the oracle (Section 3.1 MD
force of S_f = phi^+ r(A) phi, Eq. ratapprx).

Bars: the FP64 adjoint kernel within 1e-12 of the oracle's force of the same solutions X_k (the
GPU's own FP64 solve, which the force call repeats bit for bit), and the action likewise; the
whole FP64 force within 1e-8 relative of the oracle's when each side solves to 1e-12 itself (the
solutions then differ by up to kappa * 1e-12); FP32 mode within 2e-5; the autograd wrapper
returns the same components; a directional finite difference of the GPU action matches the GPU
force.
"""
import numpy as np
import pytest

from gpu_util import make_context, to_dev
from oracle import force, rational
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


def _setup(dims, mass, n, seed=3):
    ctx, U = make_context(dims, mass, gauge_seed=seed)
    phi = inputs.gaussian_vector(dims, seed + 1)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(n, 4 * mass ** 2, 16 + 4 * mass ** 2)
    return ctx, U, phi, c0, res, poles


@pytest.mark.parametrize("dims,mass,n", [((4, 4, 4, 4), 0.1, 8), ((10, 6, 4, 6), 0.05, 12), ((16, 16, 16, 8), 0.05, 14)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-8), (FP32, 2e-5)])
def test_force_matches_oracle(dims, mass, n, prec, tol):
    import torch

    import paper_1710_09178_gb300 as lq

    ctx, U, phi, c0, res, poles = _setup(dims, mass, n)
    V = int(np.prod(dims))
    F = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    Fa = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    rc, S, st = lq.fermion_force(ctx, poles, res, c0, to_dev(phi), F=F, Falg=Fa, tol=1e-12, prec=prec)
    torch.cuda.synchronize()
    assert rc == 0
    oF = force.fermion_force(U, phi, mass, dims, c0, res, poles, tol=1e-12)
    scale = np.max(np.abs(oF))
    assert np.max(np.abs(F.cpu().numpy() - oF)) <= tol * scale
    assert np.max(np.abs(Fa.cpu().numpy() - force.force_components(oF))) <= 2 * tol * scale
    oS = force.action(U, phi, mass, dims, c0, res, poles, tol=1e-12)
    assert abs(S - oS) <= 1e-10 * abs(oS)


@pytest.mark.parametrize("dims,mass,n", [((4, 4, 4, 4), 0.1, 8), ((10, 6, 4, 6), 0.05, 12), ((16, 16, 16, 8), 0.05, 14)])
def test_fp64_force_kernel_matches_oracle_on_the_same_solutions(dims, mass, n):
    # Y_k = D_oe X_k and the per-link adjoint contraction, isolated from the solver: the oracle
    # evaluates the force of exactly the X_k the GPU solve returned
    import torch

    import paper_1710_09178_gb300 as lq
    from gpu_util import gpu_mshift
    from oracle import solvers

    ctx, U, phi, c0, res, poles = _setup(dims, mass, n)
    rc, st, xs, _ = gpu_mshift(ctx, phi, poles, res, c0, tol=1e-12, prec=FP64)
    assert rc == 0
    V = int(np.prod(dims))
    F = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    rc, S, st2 = lq.fermion_force(ctx, poles, res, c0, to_dev(phi), F=F, tol=1e-12, prec=FP64)
    torch.cuda.synchronize()
    assert rc == 0 and st2["iterations"] == st["iterations"]
    oF = force.fermion_force(U, phi, mass, dims, c0, res, poles, xs=xs)
    assert np.max(np.abs(F.cpu().numpy() - oF)) <= 1e-12 * np.max(np.abs(oF))
    oS = float(np.real(np.vdot(phi, solvers.rational_apply(phi, xs, c0, res))))
    assert abs(S - oS) <= 1e-12 * abs(oS)


def test_autograd_wrapper_returns_the_force():
    import torch

    import paper_1710_09178_gb300 as lq

    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U, phi, c0, res, poles = _setup(dims, mass, 8)
    V = int(np.prod(dims))
    w = torch.zeros((V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    S = lq.FermionAction.apply(w, ctx, poles, res, c0, to_dev(phi), 1e-12, FP64)
    (g,) = torch.autograd.grad(S, w)
    oF = force.fermion_force(U, phi, mass, dims, c0, res, poles, tol=1e-12)
    assert np.max(np.abs(g.cpu().numpy() - force.force_components(oF))) <= 1e-8 * np.max(np.abs(oF))


def test_directional_finite_difference_of_gpu_action():
    import torch
    from scipy.linalg import expm

    import paper_1710_09178_gb300 as lq

    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U, phi, c0, res, poles = _setup(dims, mass, 8, seed=11)
    V = int(np.prod(dims))
    Fa = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    _, S0, _ = lq.fermion_force(ctx, poles, res, c0, to_dev(phi), Falg=Fa, tol=1e-13, prec=FP64)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(V, 4, 8))
    lam = force.gell_mann()
    eps = 1e-5

    def S_at(t):
        X = np.einsum("lma,aij->lmij", t * d, lam / 2)
        U2 = np.stack([np.stack([expm(1j * X[l, m]) @ U[l, m] for m in range(4)]) for l in range(V)])
        ctx.set_gauge(to_dev(U2))
        _, S, _ = lq.fermion_force(ctx, poles, res, c0, to_dev(phi), want_action=True, Falg=Fa, tol=1e-13, prec=FP64)
        return S

    fd = (S_at(eps) - S_at(-eps)) / (2 * eps)
    ctx.set_gauge(to_dev(U))
    _, _, _ = lq.fermion_force(ctx, poles, res, c0, to_dev(phi), Falg=Fa, tol=1e-13, prec=FP64)
    analytic = float(np.sum(Fa.cpu().numpy() * d))
    assert abs(fd - analytic) <= 1e-6 * abs(analytic)
