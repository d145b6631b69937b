"""Compressed storage of SU(3) gauge links (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 5 lists link compression as a way to cut the Dslash's memory traffic (a link is an SU(3)
matrix, 8 real degrees of freedom, stored as 18 reals) without giving a format.  Two compact forms
are defined here (readings), written for a link U with rows a, b, c:

8-real form ("r8").  Store a2, a3, b1 (six reals) and the phases th_a = arg a1, th_c = arg c1.
Decoding uses only U^dagger U = 1 and det U = 1:
    N = |a2|^2 + |a3|^2 = 1 - |a1|^2,        a1 = sqrt(1 - N) e^{i th_a}
    |c1|^2 = N - |b1|^2   (column 1 has unit norm),   c1 = |c1| e^{i th_c}
    rows a and b are orthogonal and c = conj(a x b), so (b2, b3) solves the 2x2 system
        conj(a2) b2 + conj(a3) b3 = -conj(a1) b1,     -a3 b2 + a2 b3 = conj(c1)
    whose determinant is N; rows a and c are orthogonal and b = conj(c x a), so (c2, c3) solves
        conj(a2) c2 + conj(a3) c3 = -conj(a1) c1,     -a3 c2 + a2 c3 = -conj(b1).
  When N < 1e-14 (|a1| = 1 up to 1e-7; the unit link is one) the system is singular.  Such a link
  is block-diagonal up to O(sqrt N): a2 = a3 = b1 = c1 = 0 and the lower 2x2 block is unitary
  with determinant conj(a1).  It is stored as [Re b2, Im b2, Re b3, Im b3, 0, 0, th_a, 8] (the
  phase slot th_c = 8 lies outside [-pi, pi] and marks the case) and decoded as
      a1 = e^{i th_a},  c2 = -conj(b3) conj(a1),  c3 = conj(b2) conj(a1).

16-bit form ("l16").  Rows a and b as int16 codes q = rint(u * 32767) of their real and imaginary
parts (round half to even; every entry of a unitary matrix lies in [-1, 1]), decoded as q / 32767;
row c = conj(a x b) is rebuilt from the decoded rows, as in the 12-real form.
"""
from __future__ import annotations

import numpy as np

QMAX = 32767.0
R8_DEGENERATE_N = 1e-14
R8_MARK = 8.0


def encode_r8(U):
    """(..., 3, 3) SU(3) -> (..., 8) float64 [Re a2, Im a2, Re a3, Im a3, Re b1, Im b1, th_a, th_c]
    (block-diagonal links: [Re b2, Im b2, Re b3, Im b3, 0, 0, th_a, R8_MARK])."""
    U = np.asarray(U, dtype=np.complex128)
    deg = r8_norm(U) < R8_DEGENERATE_N
    x2 = np.where(deg, U[..., 1, 1], U[..., 0, 1])
    x3 = np.where(deg, U[..., 1, 2], U[..., 0, 2])
    b1 = np.where(deg, 0.0, U[..., 1, 0])
    out = np.empty(U.shape[:-2] + (8,), dtype=np.float64)
    out[..., 0], out[..., 1] = x2.real, x2.imag
    out[..., 2], out[..., 3] = x3.real, x3.imag
    out[..., 4], out[..., 5] = b1.real, b1.imag
    out[..., 6] = np.angle(U[..., 0, 0])
    out[..., 7] = np.where(deg, R8_MARK, np.angle(U[..., 2, 0]))
    return out


def r8_norm(U):
    """N = |a2|^2 + |a3|^2 of each link; below R8_DEGENERATE_N the block-diagonal case is used."""
    U = np.asarray(U)
    return np.abs(U[..., 0, 1]) ** 2 + np.abs(U[..., 0, 2]) ** 2


def decode_r8(r):
    """(..., 8) real -> (..., 3, 3) complex128 by the unitarity relations above."""
    r = np.asarray(r, dtype=np.float64)
    deg = r[..., 7] > 4.0
    a2 = r[..., 0] + 1j * r[..., 1]
    a3 = r[..., 2] + 1j * r[..., 3]
    b1 = r[..., 4] + 1j * r[..., 5]
    N = np.abs(a2) ** 2 + np.abs(a3) ** 2
    a1 = np.sqrt(np.maximum(1.0 - N, 0.0)) * np.exp(1j * r[..., 6])
    c1 = np.sqrt(np.maximum(N - np.abs(b1) ** 2, 0.0)) * np.exp(1j * r[..., 7])
    with np.errstate(divide="ignore", invalid="ignore"):
        # 2x2 solves by Cramer's rule; the inverse of [[conj a2, conj a3], [-a3, a2]] is
        # [[a2, -conj a3], [a3, conj a2]] / N
        rhs_b = (-np.conj(a1) * b1, np.conj(c1))
        b2 = (a2 * rhs_b[0] - np.conj(a3) * rhs_b[1]) / N
        b3 = (a3 * rhs_b[0] + np.conj(a2) * rhs_b[1]) / N
        rhs_c = (-np.conj(a1) * c1, -np.conj(b1))
        c2 = (a2 * rhs_c[0] - np.conj(a3) * rhs_c[1]) / N
        c3 = (a3 * rhs_c[0] + np.conj(a2) * rhs_c[1]) / N
    # block-diagonal links: the first four slots hold b2, b3
    e1 = np.exp(1j * r[..., 6])
    zero = np.zeros_like(a2)
    a1 = np.where(deg, e1, a1)
    b2, b3 = np.where(deg, a2, b2), np.where(deg, a3, b3)
    c2 = np.where(deg, -np.conj(a3) * np.conj(e1), c2)
    c3 = np.where(deg, np.conj(a2) * np.conj(e1), c3)
    a2, a3 = np.where(deg, zero, a2), np.where(deg, zero, a3)
    b1, c1 = np.where(deg, zero, b1), np.where(deg, zero, c1)
    U = np.empty(r.shape[:-1] + (3, 3), dtype=np.complex128)
    U[..., 0, 0], U[..., 0, 1], U[..., 0, 2] = a1, a2, a3
    U[..., 1, 0], U[..., 1, 1], U[..., 1, 2] = b1, b2, b3
    U[..., 2, 0], U[..., 2, 1], U[..., 2, 2] = c1, c2, c3
    return U


def encode_l16(U):
    """(..., 3, 3) -> (..., 12) int16: rows a and b as (re, im) pairs, q = rint(u * 32767)."""
    U = np.asarray(U, dtype=np.complex128)
    rows = U[..., :2, :].reshape(U.shape[:-2] + (6,))
    re = np.empty(rows.shape[:-1] + (12,), dtype=np.float64)
    re[..., 0::2], re[..., 1::2] = rows.real, rows.imag
    return np.clip(np.rint(re * QMAX), -32767, 32767).astype(np.int16)


def third_row(a, b):
    """c = conj(a x b): the row that completes rows a, b of an SU(3) matrix."""
    return np.conj(np.cross(a, b))


def decode_l16(q):
    """(..., 12) int16 -> (..., 3, 3) complex128 with row c rebuilt from the decoded rows a, b."""
    x = np.asarray(q, dtype=np.float64) / QMAX
    rows = (x[..., 0::2] + 1j * x[..., 1::2]).reshape(x.shape[:-1] + (2, 3))
    U = np.empty(x.shape[:-1] + (3, 3), dtype=np.complex128)
    U[..., :2, :] = rows
    U[..., 2, :] = third_row(rows[..., 0, :], rows[..., 1, :])
    return U
