"""GPU parity of rhmc_trajectory (Section 3.1) against the oracle trajectory, and reversibility.

Bars (FP64 solves to 1e-12): Hamiltonian pieces within 1e-9 relative; dH within 1e-7 absolute, and
|dH| about 4 times smaller at half the step size (the integrator is second order);
proposed links and final momenta within 1e-8; integrating back with -p returns the links to 1e-10.
"""
import numpy as np
import pytest

from gpu_util import make_context, to_dev
from oracle import rational, rhmc
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64 = 0
DIMS, MASS, BETA, TAU, NSTEPS = (4, 4, 4, 4), 0.1, 5.4, 0.3, 3


def _coeffs():
    lo, hi = 4 * MASS ** 2, 16 + 4 * MASS ** 2
    return rational.zolotarev_inv_sqrt(8, lo, hi)[:3], rational.remez_power(0.25, lo, hi, 8)[:3]


def _momenta(seed):
    V = int(np.prod(DIMS))
    return inputs.counter_normal_pairs(seed, np.arange(4 * V, dtype=np.uint64), 4).reshape(V, 4, 8)


@pytest.mark.parametrize("prec_action", [0, 6])  # heatbath and Hamiltonian solves in FP64 or double-FP32
def test_trajectory_matches_oracle(prec_action):
    import torch

    import paper_1710_09178_gb300 as lq

    act, heat = _coeffs()
    ctx, U0 = make_context(DIMS, MASS, gauge_seed=31)
    p0 = _momenta(32)
    xi = inputs.gaussian_vector(DIMS, 33)
    V = int(np.prod(DIMS))
    Ud = to_dev(U0)
    links = torch.empty_like(Ud)
    mom = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    rc, res = lq.rhmc_trajectory(ctx, Ud, to_dev(p0), to_dev(xi), 0.999999, BETA, TAU, NSTEPS,
                                 (act[0], act[1], act[2]), (heat[0], heat[1], heat[2]), tol=1e-12, prec=FP64,
                                 prec_action=prec_action, mom_out=mom, links_out=links)
    assert rc == 0
    Uo, acc, info = rhmc.trajectory(U0, p0, xi, 0.999999, DIMS, MASS, BETA, TAU, NSTEPS, act, heat, tol=1e-12)
    for k in ("kinetic", "gauge", "fermion"):
        assert abs(res[k + "0"] - info["parts0"][k]) <= 1e-9 * abs(info["parts0"][k])
        assert abs(res[k + "1"] - info["parts1"][k]) <= 1e-9 * abs(info["parts1"][k])
    assert abs(res["dH"] - info["dH"]) <= 1e-7
    assert np.max(np.abs(links.cpu().numpy() - info["U1"])) <= 1e-8
    assert np.max(np.abs(mom.cpu().numpy() - info["p1"])) <= 1e-8
    assert res["accepted"] == int(acc)
    assert res["solves"] == 2 * NSTEPS + 1 + 3  # MD forces + heatbath + two Hamiltonians
    torch.cuda.synchronize()
    if res["accepted"]:
        assert np.array_equal(Ud.cpu().numpy(), links.cpu().numpy())


def test_trajectory_is_reversible_and_reject_keeps_links():
    import torch

    import paper_1710_09178_gb300 as lq

    act, heat = _coeffs()
    ctx, U0 = make_context(DIMS, MASS, gauge_seed=41)
    p0 = _momenta(42)
    phi = rhmc.heatbath(U0, inputs.gaussian_vector(DIMS, 43), MASS, DIMS, heat, tol=1e-13)
    V = int(np.prod(DIMS))
    Ud = to_dev(U0)
    links = torch.empty_like(Ud)
    mom = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    # uniform = 1: reject whatever dH is (exp(-dH) < 1 unless dH <= 0); links must stay
    rc, r1 = lq.rhmc_trajectory(ctx, Ud, to_dev(p0), to_dev(phi), 1.0 + 1e9, BETA, TAU, NSTEPS, act, tol=1e-13,
                                prec=FP64, prec_action=FP64, phi_given=True, mom_out=mom, links_out=links)
    assert rc == 0 and r1["accepted"] == 0
    assert np.array_equal(Ud.cpu().numpy(), U0)
    # backwards from the proposal with reversed momenta
    U1 = links.clone()
    back_links = torch.empty_like(Ud)
    back_mom = torch.empty_like(mom)
    rc, r2 = lq.rhmc_trajectory(ctx, U1, -mom, to_dev(phi), 1.0 + 1e9, BETA, TAU, NSTEPS, act, tol=1e-13,
                                prec=FP64, prec_action=FP64, phi_given=True, mom_out=back_mom, links_out=back_links)
    assert rc == 0
    assert np.max(np.abs(back_links.cpu().numpy() - U0)) < 1e-10
    assert np.max(np.abs(back_mom.cpu().numpy() + p0)) < 1e-9
    assert abs(r1["dH"] + r2["dH"]) < 1e-8


def test_chain_satisfies_exp_minus_dH_identity():
    # Section 3.1: the MD map is reversible and area-preserving, so over an equilibrium ensemble
    # <exp(-dH)> = 1 exactly (and hence <dH> >= 0).  A 4^4 chain at beta 5.4, m 0.1, tau 1 in 12
    # Omelyan steps: 30 thermalising trajectories from the random start, then 100 measured ones;
    # bar 4 standard errors.
    import torch

    import paper_1710_09178_gb300 as lq

    lo, hi = 4 * MASS ** 2, 16 + 4 * MASS ** 2
    act = rational.zolotarev_inv_sqrt(12, lo, hi)[:3]
    heat = rational.remez_power(0.25, lo, hi, 12)[:3]
    ctx, U0 = make_context(DIMS, MASS, gauge_seed=41)
    Ud = to_dev(U0)
    n_therm, n_meas = 30, 100
    dH, acc = [], []
    for t in range(n_therm + n_meas):
        p = _momenta(5000 + t)
        xi = inputs.gaussian_vector(DIMS, 7000 + t)
        u = float(inputs.counter_uniform(9000, np.array([t], dtype=np.uint64), 0)[0])
        rc, res = lq.rhmc_trajectory(ctx, Ud, to_dev(p), to_dev(xi), u, BETA, 1.0, 12, act, heat, tol=1e-10,
                                     md_tol=1e-9, prec=lq.FP32, prec_action=FP64)
        assert rc == 0
        if t >= n_therm:
            dH.append(res["dH"])
            acc.append(res["accepted"])
    torch.cuda.synchronize()
    dH = np.array(dH)
    w = np.exp(-dH)
    err = np.std(w, ddof=1) / np.sqrt(n_meas)
    assert abs(np.mean(w) - 1.0) <= 4 * err, (np.mean(w), err, np.mean(dH))
    assert np.mean(dH) >= -4 * np.std(dH, ddof=1) / np.sqrt(n_meas)
    assert 0.3 < np.mean(acc) <= 1.0


def test_chain_resumes_from_checkpoint(tmp_path):
    # three trajectories in one run, and the same chain stopped after the first, written to a
    # checkpoint, read back into a fresh context and continued: the same links, bit for bit, and
    # the same energies (the random numbers are drawn from streams keyed by the step)
    import torch

    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import checkpoint

    act, heat = _coeffs()
    seed = 61

    def run(ctx, Ud, steps):
        out = []
        for t in steps:
            p = _momenta(seed * 1000 + t)
            xi = inputs.gaussian_vector(DIMS, seed * 1000 + 500 + t)
            u = float(inputs.counter_uniform(seed, np.array([t], dtype=np.uint64), 0)[0])
            rc, res = lq.rhmc_trajectory(ctx, Ud, to_dev(p), to_dev(xi), u, BETA, TAU, NSTEPS, act, heat,
                                         tol=1e-10, md_tol=1e-9, prec=lq.FP32, prec_action=FP64)
            assert rc == 0
            out.append((res["dH"], res["accepted"]))
        torch.cuda.synchronize()
        return out

    ctx, U0 = make_context(DIMS, MASS, gauge_seed=62)
    Ua = to_dev(U0)
    full = run(ctx, Ua, range(3))
    ctx.close()

    ctx1, _ = make_context(DIMS, MASS, U=U0)
    Ub = to_dev(U0)
    first = run(ctx1, Ub, range(1))
    ctx1.close()
    path = str(tmp_path / "chain")
    checkpoint.save(path, Ub, DIMS, step=1, seed=seed)
    U1, h = checkpoint.load(path, DIMS)
    ctx2, _ = make_context(DIMS, MASS, U=U1)
    Uc = to_dev(U1)
    rest = run(ctx2, Uc, range(h["step"], 3))
    ctx2.close()
    assert first + rest == full
    assert np.array_equal(Uc.cpu().numpy().view(np.uint64), Ua.cpu().numpy().view(np.uint64))


def test_trajectory_is_reversible_at_24c6():
    # The RHMC workload's lattice and integrator (24^3 x 6, beta 5.4, m 0.025, tau 1 in 25 Omelyan
    # steps, 16-pole x^{-1/2}): with every solve and the MD in FP64, one trajectory forward and one
    # back from the proposal with reversed momenta return the links to 1e-10 (Section 3.1: the MD map
    # is reversible) and dH changes sign
    import torch

    import paper_1710_09178_gb300 as lq

    dims, mass, beta, tau, nsteps = (24, 24, 24, 6), 0.025, 5.4, 1.0, 25
    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, _ = lq.rational_coeffs(-0.5, lo, hi, 16)
    ctx, U0 = make_context(dims, mass, gauge_seed=9)
    V = int(np.prod(dims))
    p0 = inputs.counter_normal_pairs(9000, np.arange(4 * V, dtype=np.uint64), 4).reshape(V, 4, 8)
    phi = to_dev(inputs.gaussian_vector(dims, 9500))  # any pseudofermion field serves for reversibility
    Ud = to_dev(U0)
    links = torch.empty_like(Ud)
    mom = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    act = (c0, res, poles)
    rc, r1 = lq.rhmc_trajectory(ctx, Ud, to_dev(p0), phi, 1.0 + 1e9, beta, tau, nsteps, act, tol=1e-12,
                                prec=FP64, prec_action=FP64, phi_given=True, mom_out=mom, links_out=links)
    assert rc == 0 and r1["accepted"] == 0
    U1 = links.clone()
    back_links = torch.empty_like(Ud)
    back_mom = torch.empty_like(mom)
    rc, r2 = lq.rhmc_trajectory(ctx, U1, -mom, phi, 1.0 + 1e9, beta, tau, nsteps, act, tol=1e-12, prec=FP64,
                                prec_action=FP64, phi_given=True, mom_out=back_mom, links_out=back_links)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(back_links.cpu().numpy() - U0)) < 1e-10
    assert np.max(np.abs(back_mom.cpu().numpy() + p0)) < 1e-8
    assert abs(r1["dH"] + r2["dH"]) < 1e-6 * max(1.0, abs(r1["dH"]))


def test_energy_error_is_second_order():
    # Omelyan's 2MN integrator (Section 3.1 molecular dynamics) is second order: from the same links,
    # momenta and heatbath source, halving the step size cuts |dH| by about 4
    import paper_1710_09178_gb300 as lq

    act, heat = _coeffs()
    ctx, U0 = make_context(DIMS, MASS, gauge_seed=31)
    p0 = _momenta(32)
    xi = inputs.gaussian_vector(DIMS, 33)
    dH = []
    for n in (4, 8):
        rc, res = lq.rhmc_trajectory(ctx, to_dev(U0), to_dev(p0), to_dev(xi), 0.5, BETA, 0.5, n, act, heat,
                                     tol=1e-12, prec=FP64)
        assert rc == 0
        dH.append(res["dH"])
    ratio = abs(dH[0]) / abs(dH[1])
    assert 2.5 < ratio < 6.5, dH
