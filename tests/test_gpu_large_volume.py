"""A lattice at the top of the device's range: 128^3 x 16 = 2^25 sites.

Its FP32 link array holds 2.4 G floats and its FP64 one 19 GB, so every link and vector address
that a kernel forms in 32-bit arithmetic would overflow here.  No FP64 oracle run is affordable at
this volume, so the checks go through translation symmetry: the seeded 8^3 x 16 field and sources
tiled 16 times in x, y and z (even periods keep the staggered phases, and t, with its antiperiodic
boundary, is not tiled) define an operator that acts on a tiled vector as the small lattice's
operator acts on the tile (Section 3.2's hops only read the neighbours).

- Half-Dslash, every link format and both parities: the large lattice's output is the tiled
  output of the small lattice, bit for bit (each output site runs the same arithmetic on the same
  links and neighbours); the small lattice's output is checked against the oracle.
- Mixed-precision shifted CG (Section 4) on the tiled source: every shift certified by the
  library's true residual, and every x_k within 2 kappa_k tol of the oracle's FP64 solve of the
  small lattice, tiled (the tiled solution solves the large system exactly).
- The fermion force and action (Section 3.1) in the mixed mode against the oracle's force of the
  small lattice, tiled.
"""
import numpy as np
import pytest

from gpu_util import make_context, rel_max, tiled_gauge, tiled_half_index, to_dev
from oracle import rational, solvers, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

SMALL = (8, 8, 8, 16)
TILE = (16, 16, 16, 1)
LARGE = tuple(s * k for s, k in zip(SMALL, TILE))  # (128, 128, 128, 16)
MASS = 0.05


def tiled_index(parity):
    return tiled_half_index(SMALL, TILE, parity)


def dslash_dev(ctx, src, out_parity, prec):
    """canonical complex128 half vector (device) -> D_{out_parity} src (device), via the library"""
    import torch

    import paper_1710_09178_gb300 as lq

    vin, vout = ctx.new_vector(prec), ctx.new_vector(prec)
    ctx.pack(vin, prec, src)
    lq.dslash_eo(ctx, vout, vin, out_parity, prec)
    out = torch.empty_like(src)
    ctx.unpack(out, vout, prec)
    return out


@pytest.fixture(scope="module")
def contexts():
    import torch

    import paper_1710_09178_gb300 as lq

    small, U = make_context(SMALL, MASS, gauge_seed=81)
    large = lq.Context(LARGE, MASS)
    Ub = tiled_gauge(to_dev(U), SMALL, TILE)
    large.set_gauge(Ub)
    torch.cuda.synchronize()
    del Ub  # the context keeps its own link copies
    torch.cuda.empty_cache()
    yield small, large, U
    large.close()
    small.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6), (2, 2e-6), (4, 1e-4), (5, 2e-4), (6, 1e-13)])
def test_dslash_every_format_is_the_tiled_small_lattice(contexts, prec, tol):
    # FP64, FP32, 12-real, 8-real, 16-bit links, double-FP32; the small lattice's output against the
    # oracle at the format's bar (8-real and 16-bit links: max-norm bars of their link precision)
    import torch

    small, large, U = contexts
    psi = inputs.gaussian_vector(SMALL, 82)
    for p in (0, 1):
        src_s = to_dev(psi)
        out_s = dslash_dev(small, src_s, p, prec)
        ref = staggered.dslash_eo(U, psi, SMALL, p)
        assert rel_max(out_s.cpu().numpy(), ref) < tol
        src_b = src_s[tiled_index(1 - p)]
        out_b = dslash_dev(large, src_b, p, prec)
        assert torch.equal(out_b, out_s[tiled_index(p)])
        del src_b, out_b
        torch.cuda.empty_cache()


def test_mixed_solve_certified_against_the_tiled_oracle_solution(contexts):
    import torch

    import paper_1710_09178_gb300 as lq

    small, large, U = contexts
    b = inputs.gaussian_vector(SMALL, 83)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * MASS ** 2, 16 + 4 * MASS ** 2)
    oxs, _ = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, MASS, SMALL, poles.min()), b, poles, tol=1e-12)
    idx = tiled_index(0)
    bb = to_dev(b)[idx]
    xs = [torch.empty_like(bb) for _ in poles]
    y = torch.empty_like(bb)
    rc, st = lq.mshift_cg(large, poles, res, c0, bb, xs, y, tol=1e-10, prec=lq.FP32, raise_on_error=False)
    torch.cuda.synchronize()
    assert rc == 0, st
    assert max(st["true_residual"][: len(poles)]) <= 1e-10
    lmin = 4 * MASS ** 2
    for x, ox, s in zip(xs, oxs, poles):
        ref = to_dev(ox)[idx]
        err = float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))
        assert err <= 2 * (16 + lmin + s) / (lmin + s) * 1e-10, (s, err)
    yo = c0 * bb
    for x, c in zip(xs, res):
        yo += c * x
    assert float(torch.linalg.vector_norm(y - yo) / torch.linalg.vector_norm(yo)) < 1e-13


def test_force_and_action_against_the_tiled_oracle(contexts):
    # the MD force of S_f = phi^+ r(A) phi (Section 3.1) in the mixed mode: every link's force within the
    # FP32-mode bar of the oracle's force on the small lattice, tiled; the action is the oracle's times
    # the number of tiles (to the solves' kappa tol)
    import torch

    import paper_1710_09178_gb300 as lq
    from oracle import force

    small, large, U = contexts
    phi = inputs.gaussian_vector(SMALL, 84)
    c0, res, poles, _ = rational.zolotarev_inv_sqrt(12, 4 * MASS ** 2, 16 + 4 * MASS ** 2)
    V = int(np.prod(LARGE))
    F = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    rc, S, _ = lq.fermion_force(large, poles, res, c0, to_dev(phi)[tiled_index(0)], F=F, tol=1e-10, prec=lq.FP32,
                                raise_on_error=False)
    torch.cuda.synchronize()
    assert rc == 0
    oF = force.fermion_force(U, phi, MASS, SMALL, c0, res, poles, tol=1e-12)
    ref = tiled_gauge(to_dev(oF), SMALL, TILE)
    scale = float(ref.abs().max())
    err = 0.0
    for a in range(0, V, 1 << 22):
        err = max(err, float((F[a:a + (1 << 22)] - ref[a:a + (1 << 22)]).abs().max()))
    assert err <= 2e-5 * scale, err / scale
    del F, ref
    torch.cuda.empty_cache()
    tiles = int(np.prod(TILE))
    oS = force.action(U, phi, MASS, SMALL, c0, res, poles, tol=1e-12)
    assert abs(S - tiles * oS) <= 1e-6 * abs(tiles * oS)
