"""The translation-symmetry premise of the large-volume GPU tests, checked on the CPU with the oracle.

A gauge field and a half vector tiled k times along x, y and z (the small extents even, t not tiled:
its boundary is antiperiodic) give the tiled output of the small lattice's hopping operator
(Section 3.2) and of A.  The gather index that tiles a half vector stays inside the small vector and
takes every small site equally often, for the exact sizes the GPU test uses.
"""
import numpy as np
import pytest

from gpu_util import tiled_gauge, tiled_half_index
from oracle import staggered
from paper_1710_09178_gb300 import inputs

torch = pytest.importorskip("torch")


def test_gather_index_in_range_and_uniform_at_the_gpu_test_size():
    small, tile = (8, 8, 8, 16), (16, 16, 16, 1)
    vh_small = int(np.prod(small)) // 2
    for parity in (0, 1):
        idx = tiled_half_index(small, tile, parity, device="cpu")
        assert idx.numel() == vh_small * int(np.prod(tile))
        assert int(idx.min()) == 0 and int(idx.max()) == vh_small - 1
        counts = torch.bincount(idx, minlength=vh_small)
        assert bool(torch.all(counts == int(np.prod(tile))))


@pytest.mark.parametrize("small,tile", [((4, 2, 4, 4), (3, 2, 2, 1)), ((2, 4, 2, 6), (2, 1, 3, 1))])
def test_tiled_operator_acts_as_the_small_one(small, tile):
    large = tuple(s * k for s, k in zip(small, tile))
    U = inputs.gauge_field(small, seed=91)
    Ub = tiled_gauge(torch.from_numpy(U), small, tile).numpy()
    psi = inputs.gaussian_vector(small, 92)
    for p in (0, 1):
        src = psi[tiled_half_index(small, tile, 1 - p, device="cpu").numpy()]
        out = staggered.dslash_eo(Ub, src, large, p)
        ref = staggered.dslash_eo(U, psi, small, p)[tiled_half_index(small, tile, p, device="cpu").numpy()]
        assert np.max(np.abs(out - ref)) <= 1e-14 * np.max(np.abs(ref))
    idx = tiled_half_index(small, tile, 0, device="cpu").numpy()
    out = staggered.A_apply(Ub, psi[idx], 0.05, large, 0.01)
    ref = staggered.A_apply(U, psi, 0.05, small, 0.01)[idx]
    assert np.max(np.abs(out - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_tiling_along_t_breaks_the_premise():
    # the antiperiodic t boundary sits at the large lattice's edge only: a tiled t is a different
    # operator, which is why the GPU tests never tile t
    small, tile = (4, 2, 4, 4), (1, 1, 1, 2)
    large = tuple(s * k for s, k in zip(small, tile))
    U = inputs.gauge_field(small, seed=93)
    Ub = tiled_gauge(torch.from_numpy(U), small, tile).numpy()
    psi = inputs.gaussian_vector(small, 94)
    src = psi[tiled_half_index(small, tile, 0, device="cpu").numpy()]
    out = staggered.dslash_eo(Ub, src, large, 1)
    ref = staggered.dslash_eo(U, psi, small, 1)[tiled_half_index(small, tile, 1, device="cpu").numpy()]
    assert np.max(np.abs(out - ref)) > 0.1 * np.max(np.abs(ref))
