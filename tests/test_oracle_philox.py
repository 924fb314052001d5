"""Pins of oracle/philox.py: the published Philox4x32-10 known-answer vectors
and the distribution of the Box-Muller stream."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle.philox import gaussian, philox4x32_10, philox_words

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        a = [int(x, 16) for x in lhs.split()]
        b = [int(x, 16) for x in rhs.split()]
        rows.append((a[:4], a[4:6], b))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_known_answer_vectors(ctr, key, out):
    got = philox4x32_10(np.array(ctr, np.uint64), np.array(key, np.uint64))
    assert [int(v) for v in got] == out


def test_stream_layout_matches_counter_convention():
    seed, stream = (0x0123456789ABCDEF, 3)
    w = philox_words(seed, stream, 4 * 5 + 2)
    for b in range(6):
        ctr = np.array([b, 0, stream, 0], np.uint64)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint64)
        ref = philox4x32_10(ctr, key)
        n = min(4, w.size - 4 * b)
        assert np.array_equal(w[4 * b:4 * b + n], ref[:n])


def test_gaussian_stream_is_standard_normal():
    z = gaussian(7, 0, 400, 250).ravel()
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the four words of a block give four different values
    assert np.unique(z[:4]).size == 4


def test_streams_and_seeds_differ():
    a = gaussian(1, 0, 8, 8)
    assert not np.allclose(a, gaussian(1, 1, 8, 8))
    assert not np.allclose(a, gaussian(2, 0, 8, 8))
    assert np.array_equal(a, gaussian(1, 0, 8, 8))
