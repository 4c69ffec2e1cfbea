"""The device generator itself (ic_philox4x32_10 runs the code the noise and
thermal kernels call) against the published known-answer vectors of
Philox4x32-10 and against the oracle's generator on random counters and
keys, bit for bit."""
import os

import numpy as np
import pytest

from oracle import philox as ophilox

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_device_philox_known_answers():
    from paper_1307_0702_gb300.ic import philox4x32_10

    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    rows = np.array(rows, dtype=np.uint64).astype(np.uint32)
    out = philox4x32_10(rows[:, :6])
    assert np.array_equal(out, rows[:, 6:10])


def test_device_philox_equals_oracle():
    from paper_1307_0702_gb300.ic import philox4x32_10

    rng = np.random.default_rng(7)
    inp = rng.integers(0, 2 ** 32, (5000, 6), dtype=np.uint64).astype(np.uint32)
    # also the counters the method uses: (cell, step, purpose << 16 | block, box)
    inp[:64, 0] = np.arange(64)
    inp[:64, 2] = (1 << 16) | 2
    out = philox4x32_10(inp)
    ref = ophilox.philox4x32_10(inp[:, :4], inp[:, 4:6])
    assert np.array_equal(out, ref)
