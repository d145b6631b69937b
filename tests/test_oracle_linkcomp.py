"""Pins for oracle/linkcomp.py (compressed link storage, Section 5 "compression" outlook): the
8-real form reconstructs SU(3) links exactly (random links and hand-made ones), fails only where
N = 0, and the 16-bit form obeys its quantisation bound with exact codes for known entries."""
import numpy as np
import pytest

from oracle import linkcomp
from paper_1710_09178_gb300 import inputs


def _links():
    return inputs.gauge_field((4, 4, 4, 4), seed=31).reshape(-1, 3, 3)


def test_r8_round_trip_reconstructs_random_su3_links():
    U = _links()
    assert np.min(linkcomp.r8_norm(U)) > 1e-6
    V = linkcomp.decode_r8(linkcomp.encode_r8(U))
    assert np.max(np.abs(V - U)) < 1e-12


def _rot(i, j, th):
    R = np.eye(3, dtype=np.complex128)
    c, s = np.cos(th), np.sin(th)
    R[i, i], R[i, j], R[j, i], R[j, j] = c, s, -s, c
    return R


def test_r8_round_trip_of_hand_made_su3_matrices():
    # products of real plane rotations and a diagonal phase matrix: exactly SU(3); generic angles
    # keep |a1| and |c1| away from 0 and 1
    D = np.diag(np.exp(1j * np.array([0.4, -1.1, 0.7])))
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=np.complex128)  # cyclic permutation, det +1
    for M in (_rot(1, 2, 0.8) @ _rot(0, 1, 0.3) @ D, D @ _rot(0, 2, 1.1) @ _rot(0, 1, -0.5),
              _rot(1, 2, 0.6) @ P @ _rot(0, 1, 0.9) @ D):
        assert abs(np.linalg.det(M) - 1) < 1e-14
        assert np.max(np.abs(linkcomp.decode_r8(linkcomp.encode_r8(M)) - M)) < 1e-14


def test_r8_loses_half_the_digits_where_c1_vanishes():
    # |c1| = sqrt(N - |b1|^2): with c1 = 0 the rounding of N - |b1|^2 (~eps) becomes sqrt(eps) in c1
    M = _rot(0, 1, 0.3) @ np.diag(np.exp(1j * np.array([0.4, -1.1, 0.7])))
    assert M[2, 0] == 0
    err = np.max(np.abs(linkcomp.decode_r8(linkcomp.encode_r8(M)) - M))
    assert 1e-12 < err < 4 * np.sqrt(np.finfo(float).eps)


def test_r8_block_diagonal_links():
    # N = 0: the unit link and a1 (+) U(2) blocks with det = conj(a1) round-trip exactly
    E = np.eye(3, dtype=np.complex128)
    assert linkcomp.r8_norm(E) == 0
    assert linkcomp.encode_r8(E)[7] == linkcomp.R8_MARK
    assert np.array_equal(linkcomp.decode_r8(linkcomp.encode_r8(E)), E)
    a1 = np.exp(0.7j)
    B = _rot(0, 1, 0.4)[:2, :2] @ np.diag(np.exp(1j * np.array([0.3, -0.3])))  # SU(2)
    M = np.zeros((3, 3), dtype=np.complex128)
    M[0, 0] = a1
    M[1:, 1:] = np.conj(a1) ** 0.5 * B  # det of the block = conj(a1)
    assert abs(np.linalg.det(M) - 1) < 1e-14
    assert np.max(np.abs(linkcomp.decode_r8(linkcomp.encode_r8(M)) - M)) < 1e-15
    # just below the threshold the dropped entries (|.| <= sqrt N) are the only error
    eps = 1e-8
    Mn = _rot(0, 1, eps) @ M
    assert linkcomp.r8_norm(Mn) < linkcomp.R8_DEGENERATE_N
    assert np.max(np.abs(linkcomp.decode_r8(linkcomp.encode_r8(Mn)) - Mn)) <= 2 * eps


def test_r8_detects_a_wrong_reconstruction():
    # a plausible slip (dropping the conjugate on c1 in the b-system) breaks the round trip, so the
    # round-trip pin above would catch it
    U = _links()[:64]
    r = linkcomp.encode_r8(U)
    r[..., 7] = -r[..., 7]  # arg c1 -> -arg c1 is what a missing conjugate would produce
    assert np.max(np.abs(linkcomp.decode_r8(r) - U)) > 1e-2


def test_third_row_completes_su3():
    U = _links()
    c = linkcomp.third_row(U[:, 0, :], U[:, 1, :])
    assert np.max(np.abs(c - U[:, 2, :])) < 1e-14


def test_l16_quantisation_bound():
    U = _links()
    q = linkcomp.encode_l16(U)
    assert q.dtype == np.int16
    V = linkcomp.decode_l16(q)
    # rows a, b: each real part within half a code step
    assert np.max(np.abs((V[:, :2] - U[:, :2]).real)) <= 0.5 / 32767 + 1e-16
    assert np.max(np.abs((V[:, :2] - U[:, :2]).imag)) <= 0.5 / 32767 + 1e-16
    # row c = conj(a x b): each entry is a difference of two products of entries of modulus <= 1,
    # each complex entry off by at most sqrt(2)/2 code steps, so <= 4 * sqrt(2)/2 / 32767
    assert np.max(np.abs(V[:, 2] - U[:, 2])) <= 2 * np.sqrt(2) / 32767


def test_l16_exact_codes():
    E = np.eye(3, dtype=np.complex128)
    assert np.array_equal(linkcomp.encode_l16(E), np.array([32767, 0, 0, 0, 0, 0, 0, 0, 32767, 0, 0, 0],
                                                           dtype=np.int16))
    assert np.array_equal(linkcomp.decode_l16(linkcomp.encode_l16(E)), E)
    # ties go to the even code; -1 maps to -32767
    M = np.zeros((3, 3), dtype=np.complex128)
    M[0, 0] = 0.5 / 32767 + 1j * 1.5 / 32767
    M[0, 1] = -2.5 / 32767 - 1j
    assert np.array_equal(linkcomp.encode_l16(M)[:4], np.array([0, 2, -2, -32767], dtype=np.int16))


@pytest.mark.parametrize("fmt", ["r8", "l16"])
def test_compressed_dslash_stays_anti_hermitian(fmt):
    # D_oe^dagger = -D_eo holds for any link matrices, so also for decoded ones
    from oracle import staggered
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, seed=32)
    shape = U.shape
    if fmt == "r8":
        Uc = linkcomp.decode_r8(linkcomp.encode_r8(U.reshape(-1, 3, 3))).reshape(shape)
    else:
        Uc = linkcomp.decode_l16(linkcomp.encode_l16(U.reshape(-1, 3, 3))).reshape(shape)
    e = inputs.gaussian_vector(dims, 33)
    o = inputs.gaussian_vector(dims, 34)
    lhs = np.vdot(o, staggered.D_oe(Uc, e, dims))
    rhs = -np.vdot(staggered.D_eo(Uc, o, dims), e)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
