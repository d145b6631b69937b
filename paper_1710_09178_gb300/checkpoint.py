"""Gauge-field checkpoints for RHMC chains (Section 3.1: the configurations of U are what a run keeps).

A checkpoint is two files:

- ``<path>``: the links as raw little-endian complex128 in the canonical layout of
  ``lqcd_set_gauge`` and ``rhmc_trajectory``, ``[V][4][3][3]`` with
  ``l = x + Nx (y + Ny (z + Nz t))`` and ``mu = x, y, z, t``;
- ``<path>.json``: the lattice, the layout, the SHA-256 of the raw bytes, and the chain
  position (``step``, the index of the next trajectory, and ``seed``), plus any caller metadata.

The random numbers of a trajectory (momenta, Gaussian source, Metropolis number) are inputs
of ``rhmc_trajectory``.  A chain that draws them from counter-based streams keyed by
(seed, step) therefore continues from a checkpoint exactly as it would have run on.
Host I/O only; no GPU code.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

LAYOUT = "canonical [V][4][3][3] complex128 little-endian, l = x + Nx(y + Ny(z + Nz t)), mu = x,y,z,t"
FORMAT = "lqcd-gauge-1"


def _as_numpy(U) -> np.ndarray:
    if hasattr(U, "detach"):  # a torch tensor, on any device
        U = U.detach().cpu().numpy()
    return np.ascontiguousarray(U, dtype="<c16")


def save(path: str, U, dims, step: int, seed: int, meta: dict | None = None) -> dict:
    """Write U (numpy array or torch tensor, shape (V, 4, 3, 3)) and its header; return the header.
    The raw file is written first and renamed into place, then the header, so that a header on
    disk always describes a complete raw file."""
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    a = _as_numpy(U)
    if a.shape != (V, 4, 3, 3):
        raise ValueError(f"U has shape {a.shape}, expected {(V, 4, 3, 3)} for dims {dims}")
    raw = a.tobytes()
    header = {"format": FORMAT, "dims": list(dims), "layout": LAYOUT, "bytes": len(raw),
              "sha256": hashlib.sha256(raw).hexdigest(), "step": int(step), "seed": int(seed),
              "meta": meta or {}}
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(raw)
    os.replace(tmp, path)
    with open(path + ".json.tmp", "w") as f:
        json.dump(header, f, indent=1)
    os.replace(path + ".json.tmp", path + ".json")
    return header


def load(path: str, dims=None):
    """Read a checkpoint; return (U as a (V, 4, 3, 3) complex128 numpy array, header).  Raises
    ValueError if the header's format, size or checksum does not match the raw file, or if dims
    is given and differs from the stored lattice."""
    with open(path + ".json") as f:
        header = json.load(f)
    if header.get("format") != FORMAT:
        raise ValueError(f"{path}: not a {FORMAT} checkpoint")
    sd = tuple(header["dims"])
    if dims is not None and tuple(int(d) for d in dims) != sd:
        raise ValueError(f"{path}: lattice {sd}, expected {tuple(dims)}")
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) != header["bytes"]:
        raise ValueError(f"{path}: {len(raw)} bytes, header says {header['bytes']}")
    if hashlib.sha256(raw).hexdigest() != header["sha256"]:
        raise ValueError(f"{path}: checksum mismatch")
    V = int(np.prod(sd))
    U = np.frombuffer(raw, dtype="<c16").reshape(V, 4, 3, 3).astype(np.complex128)
    return U, header
