"""GPU parity of the half-lattice hopping operator (Section 3.2) against the FP64 oracle.

Bars: neighbour tables and 16-bit codes bit-exact; FP64 results within 1e-12
relative (max-norm); FP32 paths within 2e-6 relative (FP32 rounding of links and
vectors, 8 accumulated mat-vecs).
"""
import numpy as np
import pytest

from gpu_util import gpu_apply_A, gpu_dslash, make_context, rel_max, to_dev
from oracle import encode16, lattice, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32, FP32_R12, FP16FIX, DF64 = 0, 1, 2, 3, 6
# (10, 6, 4, 6): V/2 = 720 sites is not a multiple of any block, so every launch has a ragged tail
DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 2), (10, 6, 4, 6), (16, 16, 16, 8)]


@pytest.mark.parametrize("dims", DIMS)
def test_neighbour_tables_bit_exact(dims):
    import torch

    ctx, _ = make_context(dims, 0.1)
    Vh = int(np.prod(dims)) // 2
    fwd = torch.empty(2 * 4 * Vh, dtype=torch.int32, device="cuda")
    bwd = torch.empty_like(fwd)
    sgn = torch.empty_like(fwd)
    ctx.neighbour_table(fwd, bwd, sgn)
    torch.cuda.synchronize()
    ofwd, obwd, osf, _ = lattice.neighbour_tables(dims)
    assert np.array_equal(fwd.cpu().numpy().reshape(2, 4, Vh), ofwd)
    assert np.array_equal(bwd.cpu().numpy().reshape(2, 4, Vh), obwd)
    assert np.array_equal(sgn.cpu().numpy().reshape(2, 4, Vh), osf)


@pytest.mark.parametrize("dims", DIMS)
def test_dslash_fp64_matches_oracle(dims):
    ctx, U = make_context(dims, 0.1, gauge_seed=3)
    psi = inputs.gaussian_vector(dims, 21)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        assert rel_max(gpu_dslash(ctx, psi, p, FP64), ref) < 1e-12


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", [FP32, FP32_R12])
@pytest.mark.parametrize("tps", [1, 2, 4, 8])
def test_dslash_fp32_matches_oracle(dims, prec, tps):
    import paper_1710_09178_gb300 as lq

    ctx, U = make_context(dims, 0.1, gauge_seed=3)
    ctx.set_option(lq.OPT_DSLASH_TPS, tps)
    psi = inputs.gaussian_vector(dims, 22)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        assert rel_max(gpu_dslash(ctx, psi, p, prec), ref) < 2e-6


def test_dslash_full_size_32c8_fp32_and_r12():
    # the configuration the benchmark times, compared element by element
    dims = (32, 32, 32, 8)
    ctx, U = make_context(dims, 0.02, gauge_seed=5)
    psi = inputs.gaussian_vector(dims, 6)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        assert rel_max(gpu_dslash(ctx, psi, p, FP32), ref) < 2e-6
        assert rel_max(gpu_dslash(ctx, psi, p, FP32_R12), ref) < 2e-6
    ref = staggered.dslash_eo(U, psi, dims, 1)
    assert rel_max(gpu_dslash(ctx, psi, 1, FP64), ref) < 1e-12


def test_dslash_beyond_l2_40c8():
    # 40^3 x 8: FP32 links of 147 MB, more than L2 holds; every format against the oracle
    dims = (40, 40, 40, 8)
    ctx, U = make_context(dims, 0.05, gauge_seed=71)
    psi = inputs.gaussian_vector(dims, 73)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        assert rel_max(gpu_dslash(ctx, psi, p, FP64), ref) < 1e-12
        assert rel_max(gpu_dslash(ctx, psi, p, FP32), ref) < 2e-6
        assert rel_max(gpu_dslash(ctx, psi, p, FP32_R12), ref) < 2e-6
        assert rel_max(gpu_dslash(ctx, psi, p, DF64), ref) < 1e-13


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 2e-6), (FP32_R12, 2e-6)])
def test_apply_A_and_dot(prec, tol):
    dims, m, sigma = (10, 6, 4, 6), 0.05, 0.013
    ctx, U = make_context(dims, m, gauge_seed=4)
    psi = inputs.gaussian_vector(dims, 23)
    q, pq = gpu_apply_A(ctx, psi, sigma, prec)
    ref = staggered.A_apply(U, psi, m, dims, sigma)
    assert rel_max(q, ref) < tol
    oref = float(np.real(np.vdot(psi, ref)))
    assert abs(pq - oref) < max(tol, 1e-12) * abs(oref)


@pytest.mark.parametrize("dims", DIMS)
def test_dslash_double_fp32_matches_oracle(dims):
    # (hi, lo) links and vectors with exact products and compensated sums: ~2^-48 relative
    ctx, U = make_context(dims, 0.1, gauge_seed=3)
    psi = inputs.gaussian_vector(dims, 24)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        assert rel_max(gpu_dslash(ctx, psi, p, DF64), ref) < 1e-13


def test_apply_A_double_fp32_and_free_field():
    dims, m, sigma = (10, 6, 4, 6), 0.05, 0.013
    ctx, U = make_context(dims, m, gauge_seed=4)
    psi = inputs.gaussian_vector(dims, 25)
    q, pq = gpu_apply_A(ctx, psi, sigma, DF64)
    ref = staggered.A_apply(U, psi, m, dims, sigma)
    assert rel_max(q, ref) < 1e-13
    assert abs(pq - float(np.real(np.vdot(psi, ref)))) < 1e-12 * abs(pq)
    dims, m = (4, 4, 4, 4), 0.1
    ctx, U = make_context(dims, m, U=inputs.unit_gauge_field(dims))
    x, y, z, t = lattice.coords(dims)
    p = [2 * np.pi / 4, 2 * np.pi * 2 / 4, 0.0, 2 * np.pi * 1.5 / 4]
    full = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[:, None] * np.array([1.0, -0.5j, 0.25])
    psi = staggered.restrict(full, dims, 0)
    q, _ = gpu_apply_A(ctx, psi, 0.0, DF64)
    lam = 4 * m * m + sum(np.sin(pm) ** 2 for pm in p)
    assert np.max(np.abs(q - lam * psi)) < 1e-13


def test_free_field_on_gpu():
    dims, m = (4, 4, 4, 4), 0.1
    ctx, U = make_context(dims, m, U=inputs.unit_gauge_field(dims))
    x, y, z, t = lattice.coords(dims)
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 1, 0, 2)]:
        p = [2 * np.pi * n[0] / 4, 2 * np.pi * n[1] / 4, 2 * np.pi * n[2] / 4, 2 * np.pi * (n[3] + 0.5) / 4]
        full = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[:, None] * np.array([1.0, -0.5j, 0.25])
        psi = staggered.restrict(full, dims, 0)
        q, _ = gpu_apply_A(ctx, psi, 0.0, FP64)
        lam = 4 * m * m + sum(np.sin(pm) ** 2 for pm in p)
        assert np.max(np.abs(q - lam * psi)) < 1e-13


def test_antihermiticity_and_gauge_covariance_on_gpu():
    dims = (4, 6, 2, 4)
    ctx, U = make_context(dims, 0.1, gauge_seed=8)
    psi = inputs.gaussian_vector(dims, 31)
    chi = inputs.gaussian_vector(dims, 32)
    lhs = np.vdot(chi, gpu_dslash(ctx, psi, 1, FP64))
    rhs = -np.vdot(gpu_dslash(ctx, chi, 0, FP64), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g = inputs.random_gauge_transform(dims, seed=5)
    ctx2, _ = make_context(dims, 0.1, U=staggered.gauge_transform(U, g, dims))
    ge = g[lattice.sites_of_parity(dims, 0)]
    go = g[lattice.sites_of_parity(dims, 1)]
    a = gpu_dslash(ctx2, np.einsum("xab,xb->xa", ge, psi), 1, FP64)
    b = np.einsum("xab,xb->xa", go, gpu_dslash(ctx, psi, 1, FP64))
    assert np.max(np.abs(a - b)) < 1e-13


def test_pack_unpack_formats():
    import torch

    dims = (10, 6, 4, 6)
    ctx, _ = make_context(dims, 0.1)
    psi = inputs.gaussian_vector(dims, 41) * np.exp(inputs.gaussian_vector(dims, 42).real * 2)
    psi[3] = 0.0  # a zero site
    src = to_dev(psi)
    for prec in (FP64, FP32, FP16FIX):
        v = ctx.new_vector(prec)
        ctx.pack(v, prec, src)
        back = torch.empty_like(src)
        ctx.unpack(back, v, prec)
        torch.cuda.synchronize()
        got = back.cpu().numpy()
        if prec == FP64:
            assert np.array_equal(got, psi)
        elif prec == FP32:
            assert np.array_equal(got, psi.astype(np.complex64).astype(np.complex128))
        else:
            raw = v.cpu().numpy()
            q = raw.view(np.int16).reshape(-1, 8)[:, :6]
            s = raw.view(np.float32).reshape(-1, 4)[:, 3]
            oq, os_ = encode16.encode(encode16.complex_to_reals(psi))
            assert np.array_equal(q, oq) and np.array_equal(s, os_)
            dec = encode16.reals_to_complex(encode16.decode(oq, os_))
            assert np.array_equal(got, dec)
