"""Pins of the oracle's counter-based generator and normal transform."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(np.array(r[0:4], dtype=np.uint32), np.array(r[4:6], dtype=np.uint32))
        assert [int(x) for x in out] == r[6:10]


def test_philox_vectorised_equals_scalar():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (64, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
    batch = philox.philox4x32_10(ctr, key)
    for i in range(0, 64, 7):
        assert np.array_equal(batch[i], philox.philox4x32_10(ctr[i], key))


def test_uniform52_range_and_exactness():
    zero = np.array([0], dtype=np.uint32)
    ones = np.array([0xFFFFFFFF], dtype=np.uint32)
    assert philox.uniform52(zero, zero)[0] == 2.0 ** -53
    assert philox.uniform52(ones, ones)[0] == 1.0 - 2.0 ** -53
    # the 20 top bits of the low word enter, the 12 bottom bits do not
    lo = np.array([0xFFF], dtype=np.uint32)
    assert philox.uniform52(zero, lo)[0] == 2.0 ** -53


def test_stream_map_distinct():
    """Every (cell, step, purpose, block, box) gives distinct words."""
    base = philox.words(5, 0, np.arange(4), 3, 0, 6)
    assert len({tuple(r) for r in base.reshape(-1, 4)}) == 24
    for args in [(5, 1, np.arange(4), 3, 0, 6), (5, 0, np.arange(4), 4, 0, 6),
                 (5, 0, np.arange(4), 3, 1, 6), (6, 0, np.arange(4), 3, 0, 6)]:
        assert not np.any(philox.words(*args) == base)


def test_normals_are_standard_and_independent():
    z = philox.stress_normals(seed=123, box=0, step=7, ncells=20000)
    assert z.shape == (12, 20000)
    flat = z.reshape(-1)
    n = flat.size
    assert abs(flat.mean()) < 5.0 / np.sqrt(n)
    assert abs(flat.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    c = np.corrcoef(z)
    assert np.max(np.abs(c - np.eye(12))) < 5.0 / np.sqrt(z.shape[1])
    # fourth moment of a normal is 3
    assert abs(np.mean(flat ** 4) - 3.0) < 0.1


def test_thermal_normals_standard():
    z = philox.thermal_normals(seed=9, box=2, ncells=30000)
    assert z.shape == (4, 30000)
    assert stats.kstest(z.reshape(-1), "norm").pvalue > 1e-4
