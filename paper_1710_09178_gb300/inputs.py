"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This module holds no arithmetic of the method itself (no Dirac operator, no
solver, no rational approximation): it only draws random numbers and builds the
gauge links and Gaussian vectors that both sides receive as inputs, so that the
oracle and the GPU path see byte-identical data.

Random numbers come from a counter-based generator built on the SplitMix64
output function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): a value is a pure function of (seed, stream,
counter), so any site's numbers can be regenerated independently.  Uniforms
are turned into normal deviates with the Box-Muller transform.

Gauge links are synthetic: for every link
(site l, direction mu) draw eight N(0,1) numbers h_a, form the traceless
Hermitian H = sum_a h_a lambda_a / 2 (Gell-Mann matrices), take
U = exp(i * 0.5 * H) by scaling-and-squaring of the Taylor series, and project
the result onto SU(3) by Gram-Schmidt on rows 1 and 2 with row 3 = conj(r1 x r2).
The paper itself uses thermalised ensembles (Section 7) that are not available;
these fields stand in for them.

Pseudofermion-type Gaussian vectors use P(xi) ~ exp(-xi^dagger xi): real and
imaginary parts of every colour component are N(0, 1/2) (Section 3.1 heatbath
noise; the paper leaves the normalisation implicit).

Layouts (the C-ABI "canonical" layouts):
  gauge  : complex128 array of shape (V, 4, 3, 3), [site l][mu][row][col],
           l = x + Nx*(y + Ny*(z + Nz*t)), mu = 0..3 for x, y, z, t.
  vector : complex128 array of shape (V/2, 3) on one parity, site order = l >> 1.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (one step of the published finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, stream: np.ndarray, counter: int) -> np.ndarray:
    """64-bit random word for (seed, stream, counter); pure function of its arguments."""
    stream = np.asarray(stream, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(0x632BE59BD9B4E019))
        s = _mix64(key + (stream + np.uint64(1)) * _GOLDEN)
        return _mix64(s + np.uint64(counter + 1) * _GOLDEN)


def counter_uniform(seed: int, stream: np.ndarray, counter: int) -> np.ndarray:
    """Uniform double in (0, 1]: top 53 bits of the word, offset by one ulp."""
    w = counter_u64(seed, stream, counter)
    return ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def counter_normal_pairs(seed: int, stream: np.ndarray, npairs: int) -> np.ndarray:
    """2*npairs N(0,1) deviates per stream via Box-Muller; shape (len(stream), 2*npairs)."""
    stream = np.asarray(stream, dtype=np.uint64)
    out = np.empty((stream.shape[0], 2 * npairs), dtype=np.float64)
    for j in range(npairs):
        u1 = counter_uniform(seed, stream, 2 * j)
        u2 = counter_uniform(seed, stream, 2 * j + 1)
        rad = np.sqrt(-2.0 * np.log(u1))
        out[:, 2 * j] = rad * np.cos(2.0 * np.pi * u2)
        out[:, 2 * j + 1] = rad * np.sin(2.0 * np.pi * u2)
    return out


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def expm_taylor(X: np.ndarray) -> np.ndarray:
    """exp of a stack of 3x3 complex matrices by scaling and squaring of the Taylor series."""
    norm = np.sqrt(np.sum(np.abs(X) ** 2, axis=(-2, -1)))
    s = int(max(0, np.ceil(np.log2(max(float(norm.max(initial=0.0)), 1e-300) / 0.25))))
    Y = X / (2.0 ** s)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), X.shape)
    term = eye.copy()
    E = eye.copy()
    for k in range(1, 20):  # |Y| <= 1/4: 1/4^20/20! is far below 1e-16
        term = term @ Y / k
        E = E + term
    for _ in range(s):
        E = E @ E
    return E


def project_su3(W: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): lands exactly in SU(3)."""
    r0 = W[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = W[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def lattice_volume(dims) -> int:
    nx, ny, nz, nt = (int(d) for d in dims)
    return nx * ny * nz * nt


def check_dims(dims) -> None:
    if len(dims) != 4 or any(int(d) <= 0 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be four positive even integers, got {dims}")


def random_su3_from_streams(seed: int, streams: np.ndarray, scale: float = 0.5) -> np.ndarray:
    """U = exp(i*scale*H), H = sum_a h_a lambda_a/2, projected to SU(3); one matrix per stream."""
    h = counter_normal_pairs(seed, streams, 4)  # (n, 8)
    H = np.einsum("na,aij->nij", h.astype(np.complex128), gell_mann() / 2)
    return project_su3(expm_taylor(1j * scale * H))


def gauge_field(dims, seed: int, scale: float = 0.5, chunk: int = 1 << 18) -> np.ndarray:
    """Synthetic SU(3) gauge field, canonical layout (V, 4, 3, 3) complex128; link (l, mu) uses stream 4l+mu."""
    check_dims(dims)
    V = lattice_volume(dims)
    U = np.empty((V * 4, 3, 3), dtype=np.complex128)
    for a in range(0, 4 * V, chunk):
        b = min(4 * V, a + chunk)
        U[a:b] = random_su3_from_streams(seed, np.arange(a, b, dtype=np.uint64), scale)
    return U.reshape(V, 4, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    """U = 1 on every link (free field)."""
    check_dims(dims)
    V = lattice_volume(dims)
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()


def gaussian_vector(dims, seed: int) -> np.ndarray:
    """Complex Gaussian colour vector on one parity, (V/2, 3) complex128, Re/Im ~ N(0, 1/2).

    Half-lattice site i draws from stream i, so the vector does not depend on which
    parity it is later used on.
    """
    check_dims(dims)
    Vh = lattice_volume(dims) // 2
    g = counter_normal_pairs(seed, np.arange(Vh, dtype=np.uint64), 3) * np.sqrt(0.5)
    return (g[:, 0::2] + 1j * g[:, 1::2]).astype(np.complex128)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site, shape (V, 3, 3) (used for covariance checks)."""
    check_dims(dims)
    V = lattice_volume(dims)
    return random_su3_from_streams(seed, np.arange(V, dtype=np.uint64), scale=2.0)


# Lattice, mass and pole-count of each synthetic workload (Section 7 stand-ins).
WORKLOADS = {
    "4^4": dict(dims=(4, 4, 4, 4), mass=0.1, npoles=12, gauge_seed=1, vec_seed=2),
    "16^3x8": dict(dims=(16, 16, 16, 8), mass=0.05, npoles=14, gauge_seed=3, vec_seed=4),
    "32^3x8": dict(dims=(32, 32, 32, 8), mass=0.02, npoles=16, gauge_seed=5, vec_seed=6),
}
