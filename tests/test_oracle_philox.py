"""Pins for the oracle's Philox4x32-10 streams (published known answers, distribution checks)."""

import os

import numpy as np
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[:4], w[4:6], w[6:]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(*ctr, *key)
        assert [int(x) for x in got] == out


def test_vectorised_matches_scalar_calls():
    c0 = np.arange(5, dtype=np.uint64)
    got = philox.philox4x32_10(c0, 7, 9, 3, 11, 13)
    for i in range(5):
        one = philox.philox4x32_10(i, 7, 9, 3, 11, 13)
        assert all(int(a[i]) == int(b) for a, b in zip(got, one))


def test_gaussian_stream_is_standard_normal():
    z = philox.philox_gaussian(4000, 51, seed=123).ravel()
    assert z.shape[0] == 4000 * 51
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 1e-2
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_gaussian_stream_seed_and_shape():
    a = philox.philox_gaussian(50, 7, seed=1)
    b = philox.philox_gaussian(50, 8, seed=1)
    # odd width is the leading columns of the next even width
    np.testing.assert_array_equal(a, b[:, :7])
    c = philox.philox_gaussian(50, 7, seed=2)
    assert not np.allclose(a, c)


def test_uniform_factor_range_and_moments():
    u = philox.philox_uniform_factor(3000, 16, seed=5)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    assert stats.kstest(u.ravel(), "uniform").pvalue > 1e-3


def test_sample_words_are_64_bit_uniform():
    w = np.array(philox.philox_sample_words(100000, it=3, side=1, seed=9), dtype=np.float64)
    u = w / 2.0 ** 64
    assert u.min() >= 0 and u.max() < 1
    assert stats.kstest(u, "uniform").pvalue > 1e-3
