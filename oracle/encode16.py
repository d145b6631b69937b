"""16-bit fixed-point colour-vector storage with a per-site scale (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 5 mentions single and half precision storage (and notes that the paper
itself stays in double precision).  The compact form used here for Krylov vectors
stores one site's 3 complex numbers as six int16 codes and one float32 scale
(16 bytes per site).  Definition (reading; the paper gives none), with
every floating-point step in IEEE float32, round to nearest even:

    n   = max_i |v_i|                 over the six real components v_i (float32)
    if n == 0:  q_i = 0, s = 0
    else:       q_i = rint(v_i * (32767 / n)),  s = n / 32767
    decode:     v_i ~ q_i * s

so |decode - v_i| <= s/2 up to float32 rounding of the products.
"""
from __future__ import annotations

import numpy as np

QMAX = np.float32(32767.0)


def encode(v):
    """v: (..., 6) float32 real components of a site -> (q int16 (..., 6), s float32 (...))."""
    v = np.asarray(v, dtype=np.float32)
    n = np.max(np.abs(v), axis=-1)
    nz = n > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(nz, QMAX / np.where(nz, n, np.float32(1)), np.float32(0)).astype(np.float32)
        s = np.where(nz, n / QMAX, np.float32(0)).astype(np.float32)
    prod = (v * inv[..., None]).astype(np.float32)
    q = np.clip(np.rint(prod), -32767, 32767).astype(np.int16)
    return q, s


def decode(q, s):
    """(q, s) -> float32 components q_i * s."""
    return (np.asarray(q, dtype=np.float32) * np.asarray(s, dtype=np.float32)[..., None]).astype(np.float32)


def complex_to_reals(vec):
    """(Vh, 3) complex -> (Vh, 6) float32 as (re0, im0, re1, im1, re2, im2)."""
    vec = np.asarray(vec)
    out = np.empty(vec.shape[:-1] + (6,), dtype=np.float32)
    out[..., 0::2] = vec.real
    out[..., 1::2] = vec.imag
    return out


def reals_to_complex(r):
    r = np.asarray(r, dtype=np.float64)
    return r[..., 0::2] + 1j * r[..., 1::2]
