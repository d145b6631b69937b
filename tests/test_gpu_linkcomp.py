"""GPU parity of the half-Dslash with compressed links (Section 5 outlook: link compression).

16-bit links: the GPU decodes the same int16 codes the oracle writes (q = rint(32767 u)), so its
output must match the oracle's FP64 Dslash on the oracle-decoded links to FP32 rounding (2e-6
relative, max-norm); a single code off by one would move a site by ~3e-5.

8-real links: FP32 storage of (a2, a3, b1, arg a1, arg c1) rebuilds most links to FP32
rounding, but |c1| = sqrt(N - |b1|^2) and |a1| = sqrt(1 - N) lose up to half their digits where
they are near 0 (at most ~sqrt(eps_32) absolute, rare links).  Bars against the oracle's Dslash
on the original links: the 99.9th percentile of the site errors within 2e-6, the norm-wise error
within 2e-6 and the max within 1e-4 (relative to max |out|).  A wrong reconstruction formula
moves almost every site by O(1).
"""
import numpy as np
import pytest

from gpu_util import gpu_apply_A, gpu_dslash, make_context, rel_max, rel_norm
from oracle import linkcomp, staggered
from paper_1710_09178_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_R8, FP32_L16 = 4, 5
DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (10, 6, 4, 6), (16, 16, 16, 8)]


def _l16_links(U):
    return linkcomp.decode_l16(linkcomp.encode_l16(U.reshape(-1, 3, 3))).reshape(U.shape)


def _r8_bars(out, ref):
    site_err = np.max(np.abs(out - ref), axis=-1) / np.max(np.abs(ref))
    return float(np.quantile(site_err, 0.999)), rel_norm(out, ref), rel_max(out, ref)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("tps", [1, 2, 4, 8])
def test_dslash_l16_matches_oracle_on_decoded_links(dims, tps):
    import paper_1710_09178_gb300 as lq

    ctx, U = make_context(dims, 0.1, gauge_seed=3)
    ctx.set_option(lq.OPT_DSLASH_TPS, tps)
    Uc = _l16_links(U)
    psi = inputs.gaussian_vector(dims, 41)
    for p in (0, 1):
        out = gpu_dslash(ctx, psi, p, FP32_L16)
        assert rel_max(out, staggered.dslash_eo(Uc, psi, dims, p)) < 2e-6
        # and the compression error itself is at the 16-bit level
        assert rel_max(out, staggered.dslash_eo(U, psi, dims, p)) < 2e-4


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("tps", [1, 2, 4, 8])
def test_dslash_r8_matches_oracle(dims, tps):
    import paper_1710_09178_gb300 as lq

    ctx, U = make_context(dims, 0.1, gauge_seed=3)
    ctx.set_option(lq.OPT_DSLASH_TPS, tps)
    psi = inputs.gaussian_vector(dims, 42)
    for p in (0, 1):
        q999, rn, rm = _r8_bars(gpu_dslash(ctx, psi, p, FP32_R8), staggered.dslash_eo(U, psi, dims, p))
        assert q999 < 2e-6 and rn < 2e-6 and rm < 1e-4, (q999, rn, rm)


def _block_diagonal_links(rng, n):
    # a1 (+) sqrt(conj a1) B with B in SU(2): SU(3) links with N = 0, the 8-real form's marked case
    phi = rng.uniform(-np.pi, np.pi, n)
    th, al, be = rng.uniform(0, np.pi / 2, n), rng.uniform(-np.pi, np.pi, n), rng.uniform(-np.pi, np.pi, n)
    u, v = np.cos(th) * np.exp(1j * al), np.sin(th) * np.exp(1j * be)
    M = np.zeros((n, 3, 3), dtype=np.complex128)
    a1 = np.exp(1j * phi)
    s = np.exp(-0.5j * phi)
    M[:, 0, 0] = a1
    M[:, 1, 1], M[:, 1, 2] = s * u, s * v
    M[:, 2, 1], M[:, 2, 2] = -s * np.conj(v), s * np.conj(u)
    return M


def test_dslash_r8_unit_and_mixed_block_diagonal_links():
    # the unit field (every link block-diagonal) and a random field with 20 % block-diagonal
    # links (divergent decode paths inside a warp)
    dims = (10, 6, 4, 6)
    psi = inputs.gaussian_vector(dims, 43)
    Ue = inputs.unit_gauge_field(dims)
    ctx, _ = make_context(dims, 0.1, U=Ue)
    for p in (0, 1):
        assert rel_max(gpu_dslash(ctx, psi, p, FP32_R8), staggered.dslash_eo(Ue, psi, dims, p)) < 2e-6
    U = inputs.gauge_field(dims, seed=44).copy()
    flat = U.reshape(-1, 3, 3)
    rng = np.random.default_rng(45)
    pick = rng.random(flat.shape[0]) < 0.2
    flat[pick] = _block_diagonal_links(rng, int(pick.sum()))
    assert np.max(np.abs(np.linalg.det(flat) - 1)) < 1e-13
    ctx, _ = make_context(dims, 0.1, U=U)
    for p in (0, 1):
        q999, rn, rm = _r8_bars(gpu_dslash(ctx, psi, p, FP32_R8), staggered.dslash_eo(U, psi, dims, p))
        assert q999 < 2e-6 and rn < 2e-6 and rm < 1e-4, (q999, rn, rm)


def test_dslash_full_size_32c8_compressed():
    dims = (32, 32, 32, 8)
    ctx, U = make_context(dims, 0.02, gauge_seed=5)
    psi = inputs.gaussian_vector(dims, 6)
    Uc = _l16_links(U)
    for p in (0, 1):
        ref = staggered.dslash_eo(U, psi, dims, p)
        q999, rn, rm = _r8_bars(gpu_dslash(ctx, psi, p, FP32_R8), ref)
        assert q999 < 2e-6 and rn < 2e-6 and rm < 1e-4, (q999, rn, rm)
        assert rel_max(gpu_dslash(ctx, psi, p, FP32_L16), staggered.dslash_eo(Uc, psi, dims, p)) < 2e-6


def test_apply_A_and_dot_compressed():
    dims, m, sigma = (10, 6, 4, 6), 0.05, 0.013
    ctx, U = make_context(dims, m, gauge_seed=4)
    psi = inputs.gaussian_vector(dims, 46)
    q, pq = gpu_apply_A(ctx, psi, sigma, FP32_L16)
    ref = staggered.A_apply(_l16_links(U), psi, m, dims, sigma)
    assert rel_max(q, ref) < 2e-6
    assert abs(pq - np.real(np.vdot(psi, ref))) < 2e-6 * abs(pq)
    q, pq = gpu_apply_A(ctx, psi, sigma, FP32_R8)
    ref = staggered.A_apply(U, psi, m, dims, sigma)
    assert rel_norm(q, ref) < 2e-6
    assert abs(pq - np.real(np.vdot(psi, ref))) < 2e-6 * abs(pq)


def test_autotune_compressed_modes():
    import paper_1710_09178_gb300 as lq

    dims = (16, 16, 16, 8)
    ctx, U = make_context(dims, 0.05, gauge_seed=3)
    psi = inputs.gaussian_vector(dims, 47)
    for prec in (FP32_R8, FP32_L16):
        tps = ctx.autotune(prec)
        assert tps in (1, 2, 4, 8)
    Uc = _l16_links(U)
    assert rel_max(gpu_dslash(ctx, psi, 1, FP32_L16), staggered.dslash_eo(Uc, psi, dims, 1)) < 2e-6
    _ = lq  # the tuned option stays set on the context
