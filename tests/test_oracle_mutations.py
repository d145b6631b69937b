"""The oracle's pins catch plausible mistakes (Section 3.2 operator, Section 4 shifted CG,
Section 3.1 fermion force, gauge force and molecular dynamics, Eq. ratapprx / Appendix
rational approximation, Section 5 16-bit and compressed-link storage).

Each case plants one mistake in an in-memory copy of an oracle module: a wrong staggered phase,
a periodic instead of antiperiodic t boundary, a dropped 1/2, a missing dagger or conjugation,
a wrong sign between the hops or in A; a wrong sign, power or ratio in the shifted-CG
recurrences; a dropped sign, phase or factor, the wrong Hermitian part or a transposed outer
product in the fermion force; a wrong normalisation or staple in the gauge force; a wrong kick
or drift in the Omelyan integrator; a wrong residue, node order or scale in the Zolotarev
approximation; a wrong rounding or scale in the 16-bit codes, a wrong reconstruction in the
compressed links.  The compact pins below (free field, anti-hermiticity,
hermiticity, gauge covariance; residual collinearity; central finite differences of S_f and
S_g; reversibility and the second-order energy error; the relative error of the partial
fractions against x^{-1/2}) must all hold for the real oracle, and
at least one must fail for every mutant.  The files under oracle/ are never modified.
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


# ---- fermion force (Section 3.1 MD equations): central finite differences of S_f ----------
def _force_copy(edit=None):
    from oracle import force

    src = inspect.getsource(force)
    if edit:
        assert edit[0] in src
        src = src.replace(edit[0], edit[1], 1)
    src = src.replace("from . import lattice, staggered, solvers\n", "")
    return _module("force_copy", src, lattice=lattice, staggered=staggered, solvers=solvers)


def _force_fd_error(fmod):
    from scipy.linalg import expm

    from oracle import rational

    dims, mass = (4, 2, 2, 4), 0.1
    U = inputs.gauge_field(dims, seed=3)
    phi = inputs.gaussian_vector(dims, 4)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(6, 4 * mass ** 2, 16 + 4 * mass ** 2)
    Fa = fmod.force_components(fmod.fermion_force(U, phi, mass, dims, c0, res, poles))
    lam = fmod.gell_mann()
    rng = np.random.default_rng(11)
    V = int(np.prod(dims))
    worst, eps = 0.0, 1e-5
    for _ in range(8):
        l, mu, a = int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(8))

        def S(w):
            U2 = U.copy()
            U2[l, mu] = expm(1j * w * lam[a] / 2) @ U[l, mu]
            return fmod.action_dense(U2, phi, mass, dims, c0, res, poles)

        fd = (S(eps) - S(-eps)) / (2 * eps)
        worst = max(worst, abs(fd - Fa[l, mu, a]) / max(abs(fd), 1e-2))
    return worst


FORCE_MUTANTS = {
    "odd-site sign dropped": ("        O[par == 1] *= -1\n", ""),
    "staggered phase and boundary sign dropped": (
        "H = 0.5j * s[:, None, None] * (W - np.conj(np.transpose(W, (0, 2, 1))))",
        "H = 0.5j * (W - np.conj(np.transpose(W, (0, 2, 1))))"),
    "Hermitian instead of anti-Hermitian part": (
        "(W - np.conj(np.transpose(W, (0, 2, 1))))", "(W + np.conj(np.transpose(W, (0, 2, 1))))"),
    "factor 1 instead of 1/2": ("F[:, mu] = 0.5 * (H", "F[:, mu] = 1.0 * (H"),
    "outer product transposed": ('np.einsum("xa,xb->xab", z[xf], np.conj(z))',
                                 'np.einsum("xa,xb->xba", z[xf], np.conj(z))'),
}


def test_force_finite_differences_hold_for_the_oracle():
    from oracle import force

    assert _force_fd_error(force) < 1e-7


@pytest.mark.parametrize("name", sorted(FORCE_MUTANTS))
def test_force_finite_differences_catch_planted_mistake(name):
    assert _force_fd_error(_force_copy(FORCE_MUTANTS[name])) > 1e-3


# ---- gauge force and the Omelyan integrator (Section 3.1) --------------------------------
def _rhmc_copy(edit=None):
    from oracle import force, rational, rhmc

    src = inspect.getsource(rhmc)
    if edit:
        assert edit[0] in src
        src = src.replace(edit[0], edit[1], 1)
    src = src.replace("from . import force as force_mod\n", "").replace(
        "from . import lattice, rational, solvers, staggered\n", "")
    return _module("rhmc_copy", src, force_mod=force, lattice=lattice, rational=rational, solvers=solvers,
                   staggered=staggered)


GDIMS, GBETA = (4, 4, 4, 4), 5.4


def _gauge_fd_error(rmod):
    from scipy.linalg import expm

    from oracle import force

    U = inputs.gauge_field(GDIMS, seed=21)
    Fa = force.force_components(rmod.gauge_force(U, GBETA, GDIMS))
    lam = force.gell_mann()
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(6):
        l, mu, a = int(rng.integers(256)), int(rng.integers(4)), int(rng.integers(8))

        def S(w):
            U2 = U.copy()
            U2[l, mu] = expm(1j * w * lam[a] / 2) @ U[l, mu]
            return rmod.gauge_action(U2, GBETA, GDIMS)

        fd = (S(1e-5) - S(-1e-5)) / 2e-5
        worst = max(worst, abs(fd - Fa[l, mu, a]) / max(1.0, abs(fd)))
    return worst


class _GaugeOnly:
    """H = 1/2 p^2 + S_g: the integrator's pins without solves."""

    def __init__(self, rmod):
        from oracle import force

        self.r, self.f = rmod, force

    def force(self, U, phi):
        return self.f.force_components(self.r.gauge_force(U, GBETA, GDIMS))

    def H(self, U, p):
        return 0.5 * float(np.sum(p * p)) + self.r.gauge_action(U, GBETA, GDIMS)


def _integrator_pins(rmod):
    """(reversibility error, |dH(eps)| / |dH(eps/2)|) on 4^4 with the gauge action alone."""
    act = _GaugeOnly(rmod)
    U = inputs.gauge_field(GDIMS, seed=23)
    V = int(np.prod(GDIMS))
    p = inputs.counter_normal_pairs(24, np.arange(4 * V, dtype=np.uint64), 4).reshape(V, 4, 8)
    U1, p1 = rmod.integrate(U, p, None, act, 0.2, 4)
    U2, p2 = rmod.integrate(U1, -p1, None, act, 0.2, 4)
    rev = max(np.max(np.abs(U2 - U)), np.max(np.abs(p2 + p)))
    H0 = act.H(U, p)
    dH = [act.H(*rmod.integrate(U, p, None, act, 0.2, n)) - H0 for n in (4, 8)]
    return rev, abs(dH[0]) / abs(dH[1])


GAUGE_MUTANTS = {
    "force normalised with beta/6": ("F = -1j * beta / 12.0 *", "F = -1j * beta / 6.0 *"),
    "upper staple without the last dagger": ("@ dag(U[xpnu, mu]) @ dag(U[:, nu])", "@ dag(U[xpnu, mu]) @ U[:, nu]"),
    "lower staple with the wrong first link": ("down = dag(U[xpmu_mnu, nu])", "down = dag(U[xmnu, nu])"),
}

INTEGRATOR_MUTANTS = {
    "middle kick 1 - lambda": ("p = p - (1.0 - 2.0 * lam) * eps", "p = p - (1.0 - lam) * eps"),
    "last kick 2 lambda": ("w = 2.0 * lam if step < nsteps - 1 else lam", "w = 2.0 * lam"),
    "drift of a full step": ("U = update_links(U, p, 0.5 * eps)\n        p = p -", "U = update_links(U, p, eps)\n        p = p -"),
}


def test_gauge_force_and_integrator_pins_hold_for_the_oracle():
    from oracle import rhmc

    assert _gauge_fd_error(rhmc) < 5e-7
    rev, ratio = _integrator_pins(rhmc)
    assert rev < 1e-10 and 3.0 < ratio < 5.5, (rev, ratio)


@pytest.mark.parametrize("name", sorted(GAUGE_MUTANTS))
def test_gauge_force_finite_differences_catch_planted_mistake(name):
    assert _gauge_fd_error(_rhmc_copy(GAUGE_MUTANTS[name])) > 1e-3


@pytest.mark.parametrize("name", sorted(INTEGRATOR_MUTANTS))
def test_integrator_pins_catch_planted_mistake(name):
    rev, ratio = _integrator_pins(_rhmc_copy(INTEGRATOR_MUTANTS[name]))
    assert rev > 1e-8 or not (3.0 < ratio < 5.5), (name, rev, ratio)


# ---- rational approximation (Eq. ratapprx, Appendix) --------------------------------------
def _rational_copy(edit=None):
    from oracle import rational

    src = inspect.getsource(rational)
    if edit:
        assert edit[0] in src
        src = src.replace(edit[0], edit[1], 1)
    return _module("rational_copy", src)


def _rational_error(rmod):
    """Max relative error of the partial-fraction form of the 12-pole x^{-1/2} on [0.04, 16.04],
    evaluated term by term on a dense logarithmic grid (not through the routine's own estimate)."""
    lo, hi = 0.04, 16.04
    c0, res, poles, _ = rmod.zolotarev_inv_sqrt(12, lo, hi)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 40001))
    r = np.full_like(x, c0)
    for c, d in zip(res, poles):
        r += c / (x + d)
    return float(np.max(np.abs(r * np.sqrt(x) - 1.0)))


RATIONAL_MUTANTS = {
    "residue with the reversed pole differences": ("np.prod(np.delete(poles, k) - dk)", "np.prod(dk - np.delete(poles, k))"),
    "zeros and poles interleaved the other way": ("poles_u = c[0::2][:n]", "poles_u = c[1::2][:n]"),
    "wrong power of the interval scale": ("K = D * lo ** -0.5 *", "K = D * lo ** 0.5 *"),
    "Jacobi nodes of the wrong order": ("M = 2 * n + 1 if with_c0 else 2 * n", "M = 2 * n + 2 if with_c0 else 2 * n"),
}


def test_rational_error_holds_for_the_oracle():
    assert _rational_error(_rational_copy()) < 1e-10


@pytest.mark.parametrize("name", sorted(RATIONAL_MUTANTS))
def test_rational_error_catches_planted_mistake(name):
    assert _rational_error(_rational_copy(RATIONAL_MUTANTS[name])) > 1e-6


# ---- 16-bit vector storage and compressed links (Section 5) --------------------------------
def _copy_of(modname, edit=None):
    import importlib

    src = inspect.getsource(importlib.import_module("oracle." + modname))
    if edit:
        assert edit[0] in src
        src = src.replace(edit[0], edit[1], 1)
    return _module(modname + "_copy", src)


def _encode16_pins(m):
    """Error bound and extreme code on random sites, exact codes, ties to even."""
    rng = np.random.default_rng(5)
    v = (rng.normal(size=(2048, 6)) * np.exp(rng.normal(size=(2048, 1)) * 3)).astype(np.float32)
    q, s = m.encode(v)
    d = m.decode(q, s)
    n = np.max(np.abs(v), axis=1)
    imax = np.argmax(np.abs(v), axis=1)
    bound = bool(np.all(np.abs(d - v) <= (0.5 * s + 4e-7 * n)[:, None]))
    extreme = bool(np.all(np.abs(q[np.arange(v.shape[0]), imax]) == 32767))
    qt, _ = m.encode(np.array([[32767.0, 2.5, -3.5, 0.5, 1.5, -0.5]], dtype=np.float32))
    ties = bool(np.array_equal(qt[0], np.array([32767, 2, -4, 0, 2, 0], dtype=np.int16)))
    return bound and extreme and ties


def _linkcomp_pins(m):
    """8-real and 16-bit round trips of random SU(3) links within their storage error."""
    U = inputs.gauge_field((2, 2, 2, 4), seed=17).reshape(-1, 3, 3)
    r8 = np.max(np.abs(m.decode_r8(m.encode_r8(U)) - U))
    l16 = np.max(np.abs(m.decode_l16(m.encode_l16(U)) - U))
    return r8 < 1e-10 and l16 < 5e-5


STORAGE_MUTANTS = {
    "encode16: floor instead of round to nearest": ("encode16", ("np.clip(np.rint(prod)", "np.clip(np.floor(prod)")),
    "encode16: scale 32768": ("encode16", ("QMAX = np.float32(32767.0)", "QMAX = np.float32(32768.0)")),
    "linkcomp: third row without conjugation": ("linkcomp", ("return np.conj(np.cross(a, b))", "return np.cross(a, b)")),
    "linkcomp: c1 from |b1| alone": ("linkcomp", ("np.sqrt(np.maximum(N - np.abs(b1) ** 2, 0.0))",
                                                  "np.sqrt(np.maximum(1.0 - np.abs(b1) ** 2, 0.0))")),
    "linkcomp: b3 with the wrong conjugate": ("linkcomp", ("b3 = (a3 * rhs_b[0] + np.conj(a2) * rhs_b[1]) / N",
                                                           "b3 = (a3 * rhs_b[0] + a2 * rhs_b[1]) / N")),
}


def test_storage_pins_hold_for_the_oracle():
    assert _encode16_pins(_copy_of("encode16")) and _linkcomp_pins(_copy_of("linkcomp"))


@pytest.mark.parametrize("name", sorted(STORAGE_MUTANTS))
def test_storage_pins_catch_planted_mistake(name):
    modname, edit = STORAGE_MUTANTS[name]
    pins = _encode16_pins if modname == "encode16" else _linkcomp_pins
    assert not pins(_copy_of(modname, edit))
