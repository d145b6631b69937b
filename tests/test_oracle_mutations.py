"""The oracle's pins catch plausible mistakes (Section 3.2 operator, Section 4 shifted CG).

Each case plants one mistake in an in-memory copy of an oracle module: a wrong staggered phase,
a periodic instead of antiperiodic t boundary, a dropped 1/2, a missing dagger or conjugation,
a wrong sign between the hops or in A, a wrong sign, power or ratio in the shifted-CG
recurrences.  The compact pins below must all hold for the real oracle and at least one must
fail for every mutant.  The files under oracle/ are never modified.
"""
import inspect
import itertools
import types

import numpy as np
import pytest

from oracle import lattice, solvers, staggered
from paper_1710_09178_gb300 import inputs


def _module(name, src, **inject):
    m = types.ModuleType(name)
    m.__dict__.update(inject)
    exec(compile(src, name, "exec"), m.__dict__)
    return m


def _oracle(lat_edit=None, stag_edit=None):
    """(lattice, staggered) modules, optionally with one source replacement each."""
    lsrc = inspect.getsource(lattice)
    ssrc = inspect.getsource(staggered)
    if lat_edit:
        assert lat_edit[0] in lsrc
        lsrc = lsrc.replace(lat_edit[0], lat_edit[1], 1)
    if stag_edit:
        assert stag_edit[0] in ssrc
        ssrc = ssrc.replace(stag_edit[0], stag_edit[1], 1)
    lat = _module("lattice_copy", lsrc)
    ssrc = ssrc.replace("from . import lattice\n", "")
    return lat, _module("staggered_copy", ssrc, lattice=lat)


def _operator_pins(lat, stag):
    """Free-field spectrum, anti-hermiticity of the hops, hermiticity of A, gauge covariance."""
    ok = {}
    dims = (4, 4, 4, 4)  # every extent > 2: on 2 sites the forward and backward hops coincide
    U1 = inputs.unit_gauge_field(dims)
    x, y, z, t = lat.coords(dims)
    v = np.array([1.0, 0.5j, -0.25])
    worst = 0.0
    for n in itertools.product(range(dims[0]), range(dims[1]), range(dims[2]), range(dims[3])):
        p = [2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1], 2 * np.pi * n[2] / dims[2],
             2 * np.pi * (n[3] + 0.5) / dims[3]]
        full = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[:, None] * v[None, :]
        psi = stag.restrict(full, dims, 0)
        out = -stag.D_eo(U1, stag.D_oe(U1, psi, dims), dims)
        worst = max(worst, np.max(np.abs(out - sum(np.sin(q) ** 2 for q in p) * psi)))
    ok["free field"] = worst < 1e-12
    U = inputs.gauge_field(dims, seed=3)
    pe = inputs.gaussian_vector(dims, 4)
    po = inputs.gaussian_vector(dims, 5)
    lhs = np.vdot(po, stag.D_oe(U, pe, dims))
    rhs = -np.vdot(stag.D_eo(U, po, dims), pe)
    ok["anti-hermiticity"] = abs(lhs - rhs) < 1e-12 * abs(lhs)
    m, sigma = 0.1, 0.02
    a1 = np.vdot(po, stag.A_apply(U, pe, m, dims, sigma))
    a2 = np.vdot(stag.A_apply(U, po, m, dims, sigma), pe)
    lo = np.vdot(pe, stag.A_apply(U, pe, m, dims, sigma)).real / np.vdot(pe, pe).real
    ok["A hermitian, >= 4m^2"] = abs(a1 - a2) < 1e-12 * abs(a1) and lo >= 4 * m * m
    g = inputs.random_gauge_transform(dims, 6)
    Ug = stag.gauge_transform(U, g, dims)
    full = stag.embed(pe, dims, 0)
    gpsi = stag.restrict(np.einsum("xab,xb->xa", g, full), dims, 0)
    lhs = stag.D_oe(Ug, gpsi, dims)
    rhs = stag.restrict(np.einsum("xab,xb->xa", g, stag.embed(stag.D_oe(U, pe, dims), dims, 1)), dims, 1)
    ok["gauge covariance"] = np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))
    return ok


OPERATOR_MUTANTS = {
    "eta_y from y instead of x": (("        return (-1) ** x\n", "        return (-1) ** y\n"), None),
    "eta_t without z": (("        return (-1) ** (x + y + z)\n", "        return (-1) ** (x + y)\n"), None),
    "periodic in t": (("            s[t == nt - 1] = -1\n", "            pass\n"), None),
    "no dagger on the backward link": (None, ('np.einsum("xba,xb->xa", np.conj(U[xb, mu])',
                                              'np.einsum("xab,xb->xa", np.conj(U[xb, mu])')),
    "no conjugation on the backward link": (None, ('np.conj(U[xb, mu])', '(U[xb, mu])')),
    "factor 1 instead of 1/2": (None, ("out += 0.5 * eta[:, None]", "out += 1.0 * eta[:, None]")),
    "hops added": (None, ("* (fwd - bwd)", "* (fwd + bwd)")),
    "A = 4m^2 + D_eo D_oe": (None, ("* psi_e - D_eo(", "* psi_e + D_eo(")),
}


def test_operator_pins_hold_for_the_oracle():
    ok = _operator_pins(lattice, staggered)
    assert all(ok.values()), ok


@pytest.mark.parametrize("name", sorted(OPERATOR_MUTANTS))
def test_operator_pins_catch_planted_mistake(name):
    lat_edit, stag_edit = OPERATOR_MUTANTS[name]
    ok = _operator_pins(*_oracle(lat_edit, stag_edit))
    assert not all(ok.values()), (name, ok)


def _collinearity_error(solv):
    dims, mass = (4, 4, 2, 2), 0.1
    U = inputs.gauge_field(dims, seed=5)
    b = inputs.gaussian_vector(dims, 6)
    shifts = np.array([0.003, 0.04, 0.5, 2.0, 11.0])
    A = lambda v, s: staggered.A_apply(U, v, mass, dims, s)
    xs, info = solv.multishift_cg(lambda v: A(v, shifts.min()), b, shifts, fixed_iters=5)
    r0 = b - A(xs[0], shifts[0])
    return max(np.linalg.norm(b - A(xk, s) - info["zeta"][k] * r0) for k, (xk, s) in enumerate(zip(xs, shifts))) \
        / np.linalg.norm(b)


SOLVER_MUTANTS = {
    "sign of the shift in the zeta recurrence": ("(1.0 + s[k] * alpha)", "(1.0 - s[k] * alpha)"),
    "beta_k with the first power of the zeta ratio": ("(zeta_new[k] / zeta[k]) ** 2", "(zeta_new[k] / zeta[k])"),
    "x_k step with the inverted zeta ratio": ("(alpha * zeta_new[k] / zeta[k])", "(alpha * zeta[k] / zeta_new[k])"),
    "p_k from the old zeta": ("ps[k] = zeta_new[k] * r", "ps[k] = zeta[k] * r"),
}


def test_collinearity_holds_for_the_oracle():
    assert _collinearity_error(solvers) < 1e-12


@pytest.mark.parametrize("name", sorted(SOLVER_MUTANTS))
def test_collinearity_catches_planted_mistake(name):
    a, b = SOLVER_MUTANTS[name]
    src = inspect.getsource(solvers)
    assert a in src
    mutant = _module("solvers_copy", src.replace(a, b, 1))
    assert _collinearity_error(mutant) > 1e-6
