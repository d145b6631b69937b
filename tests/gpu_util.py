"""Helpers for the GPU parity tests: move seeded inputs to the device and run the library."""
import functools

import numpy as np

from paper_1710_09178_gb300 import inputs


def torch_mod():
    import torch

    return torch


def to_dev(a):
    torch = torch_mod()
    a = np.ascontiguousarray(a)
    if not a.flags.writeable:  # the shared seeded fields
        a = a.copy()
    return torch.from_numpy(a).cuda()


@functools.lru_cache(maxsize=4)
def seeded_gauge(dims, seed):
    """inputs.gauge_field, generated once per (dims, seed) in a test session and read-only (the
    large lattices take seconds to generate); callers that modify links take a copy."""
    U = inputs.gauge_field(tuple(dims), seed=seed)
    U.flags.writeable = False
    return U


def make_context(dims, mass, U=None, gauge_seed=1):
    import paper_1710_09178_gb300 as lq

    ctx = lq.Context(dims, mass)
    if U is None:
        U = seeded_gauge(tuple(dims), gauge_seed)
    ctx.set_gauge(to_dev(U))
    return ctx, U


def gpu_dslash(ctx, psi, out_parity, prec):
    """Canonical complex128 numpy vector in -> canonical numpy vector out, via pack / dslash_eo / unpack."""
    import paper_1710_09178_gb300 as lq

    torch = torch_mod()
    src = to_dev(psi)
    vin = ctx.new_vector(prec)
    vout = ctx.new_vector(prec)
    ctx.pack(vin, prec, src)
    lq.dslash_eo(ctx, vout, vin, out_parity, prec)
    res = torch.empty_like(src)
    ctx.unpack(res, vout, prec)
    torch.cuda.synchronize()
    return res.cpu().numpy()


def gpu_apply_A(ctx, psi, sigma, prec):
    torch = torch_mod()
    src = to_dev(psi)
    vin = ctx.new_vector(prec)
    vout = ctx.new_vector(prec)
    ctx.pack(vin, prec, src)
    pq = ctx.apply_A(vout, vin, sigma, prec, want_dot=True)
    res = torch.empty_like(src)
    ctx.unpack(res, vout, prec)
    torch.cuda.synchronize()
    return res.cpu().numpy(), pq


def gpu_mshift(ctx, b, shifts, residues=None, c0=0.0, tol=1e-10, maxiter=20000, prec=0, want_y=False):
    import paper_1710_09178_gb300 as lq

    torch = torch_mod()
    bd = to_dev(b)
    xs = [torch.empty_like(bd) for _ in shifts]
    y = torch.empty_like(bd) if want_y else None
    rc, st = lq.mshift_cg(ctx, shifts, residues if residues is not None else [0.0] * len(shifts), c0, bd, xs, y,
                          tol=tol, maxiter=maxiter, prec=prec, raise_on_error=False)
    torch.cuda.synchronize()
    return rc, st, [x.cpu().numpy() for x in xs], (y.cpu().numpy() if want_y else None)


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_norm(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tiled_half_index(small, tile, parity, device="cuda"):
    """Tiling a lattice `small` (all extents even) k_mu times along each axis: for every site of the
    large lattice's half vector of `parity`, the index of the small lattice's site it copies (torch
    int64 on `device`).  Checkerboard index cb = l >> 1 with l = x + Nx (y + Ny (z + Nz t)); the sites
    l and l + 1 (l even) differ only in x, so exactly one of them has the parity."""
    torch = torch_mod()
    large = [s * k for s, k in zip(small, tile)]
    X, Y, Z, _ = large
    xs, ys, zs, _ = small
    l0 = 2 * torch.arange(int(np.prod(large)) // 2, device=device, dtype=torch.int64)
    x0 = l0 % X
    rest = l0 // X
    y = rest % Y
    rest = rest // Y
    z = rest % Z
    t = rest // Z
    x = x0 + ((parity + y + z + t) & 1)
    ls = (x % xs) + xs * ((y % ys) + ys * ((z % zs) + zs * (t % small[3])))
    return ls >> 1


def tiled_gauge(U_small, small, tile):
    """The canonical (V, 4, 3, 3) gauge tensor U_small (any device) repeated k_mu times per axis."""
    X, Y, Z, T = small
    u = U_small.reshape(T, Z, Y, X, 4, 3, 3)
    return u.repeat(tile[3], tile[2], tile[1], tile[0], 1, 1, 1).reshape(-1, 4, 3, 3).contiguous()
