"""Pins for oracle/encode16.py: error bound, extreme codes, zero sites, exact round trips."""
import numpy as np

from oracle import encode16


def test_error_bound_and_extreme_code():
    rng = np.random.default_rng(5)
    v = (rng.normal(size=(4096, 6)) * np.exp(rng.normal(size=(4096, 1)) * 3)).astype(np.float32)
    q, s = encode16.encode(v)
    d = encode16.decode(q, s)
    n = np.max(np.abs(v), axis=1)
    # |decode - v| <= s/2 plus float32 rounding of the scale products
    assert np.all(np.abs(d - v) <= (0.5 * s + 4e-7 * n)[:, None])
    # the largest component of every site maps to +-32767
    imax = np.argmax(np.abs(v), axis=1)
    assert np.all(np.abs(q[np.arange(v.shape[0]), imax]) == 32767)
    assert q.dtype == np.int16 and s.dtype == np.float32


def test_zero_site_and_exact_values():
    v = np.zeros((3, 6), dtype=np.float32)
    v[1] = [1.0, -1.0, 0.5, 0.0, -0.25, 0.125]
    q, s = encode16.encode(v)
    assert np.all(q[0] == 0) and s[0] == 0 and np.all(q[2] == 0)
    assert np.array_equal(q[1], np.array([32767, -32767, 16384, 0, -8192, 4096], dtype=np.int16))
    d = encode16.decode(q, s)
    assert np.all(d[0] == 0)
    assert np.max(np.abs(d[1] - v[1])) <= 0.5 / 32767


def test_ties_round_to_even():
    # components equal to (k + 1/2) / 32767 of the norm land exactly on a tie in float32
    v = np.array([[32767.0, 2.5, -3.5, 0.5, 1.5, -0.5]], dtype=np.float32)
    q, s = encode16.encode(v)
    assert np.array_equal(q[0], np.array([32767, 2, -4, 0, 2, 0], dtype=np.int16))
