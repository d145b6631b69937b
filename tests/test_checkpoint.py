"""Gauge-field checkpoints (host I/O): exact round trip, header contents, and refusal of a
corrupted or mismatched file."""
import json

import numpy as np
import pytest

from paper_1710_09178_gb300 import checkpoint, inputs

DIMS = (4, 4, 2, 6)


def test_round_trip_is_bit_exact(tmp_path):
    U = inputs.gauge_field(DIMS, seed=11)
    p = str(tmp_path / "cfg")
    h = checkpoint.save(p, U, DIMS, step=7, seed=123, meta={"beta": 5.4})
    U2, h2 = checkpoint.load(p, DIMS)
    assert U2.dtype == np.complex128 and U2.shape == U.shape
    assert np.array_equal(U2.view(np.uint64), U.view(np.uint64))
    assert h2 == h and h2["step"] == 7 and h2["seed"] == 123 and h2["meta"] == {"beta": 5.4}
    assert h2["dims"] == list(DIMS) and h2["bytes"] == U.nbytes


def test_torch_tensor_input(tmp_path):
    torch = pytest.importorskip("torch")
    U = inputs.gauge_field(DIMS, seed=12)
    p = str(tmp_path / "cfg")
    checkpoint.save(p, torch.from_numpy(U), DIMS, step=0, seed=0)
    assert np.array_equal(checkpoint.load(p)[0], U)


def test_corruption_and_mismatch_are_refused(tmp_path):
    U = inputs.gauge_field(DIMS, seed=13)
    p = str(tmp_path / "cfg")
    checkpoint.save(p, U, DIMS, step=1, seed=1)
    with pytest.raises(ValueError):
        checkpoint.load(p, (4, 4, 4, 6))
    raw = bytearray(open(p, "rb").read())
    raw[1000] ^= 0x01
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="checksum"):
        checkpoint.load(p)
    open(p, "wb").write(bytes(raw[:-16]))
    with pytest.raises(ValueError):
        checkpoint.load(p)
    h = json.load(open(p + ".json"))
    h["format"] = "other"
    json.dump(h, open(p + ".json", "w"))
    with pytest.raises(ValueError):
        checkpoint.load(p)


def test_wrong_shape_is_refused(tmp_path):
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "cfg"), np.zeros((10, 4, 3, 3), np.complex128), DIMS, step=0, seed=0)
