"""Properties of the oracle's Philox4x32-10 stream and Rademacher sketch.

The exact bit stream is pinned separately, block for block, against
PyTorch's independently written Philox4x32-10 engine
(tests/test_oracle_philox_pin.py); these tests check the statistical
properties the sketch relies on.
"""
import numpy as np

from oracle.philox import philox4x32_10, rademacher


def test_deterministic_and_pm1():
    a = rademacher(300, 200, seed=7, step=3)
    b = rademacher(300, 200, seed=7, step=3)
    assert a.shape == (300, 200)
    assert np.array_equal(a, b)
    assert set(np.unique(a)) == {-1.0, 1.0}


def test_streams_differ():
    base = rademacher(64, 256, seed=1, step=2)
    for other in (rademacher(64, 256, seed=2, step=2), rademacher(64, 256, seed=1, step=3),
                  rademacher(64, 256, seed=1 << 32 | 1, step=2)):
        agree = np.mean(base == other)
        assert 0.45 < agree < 0.55


def test_column_prefix_is_stable():
    # growing l keeps the earlier columns (fresh columns continue the stream)
    a = rademacher(50, 40, seed=3, step=1)
    b = rademacher(50, 300, seed=3, step=1)
    assert np.array_equal(a, b[:, :40])


def test_bit_frequencies_chi2():
    n = 4096
    w = philox4x32_10(np.arange(n), np.zeros(n), np.zeros(n), np.zeros(n), 123, 456)
    bits = np.stack([(wi[:, None] >> np.arange(32, dtype=np.uint32)) & 1 for wi in w], 1).reshape(n, 128)
    ones = bits.sum(0)
    chi2 = np.sum((ones - n / 2) ** 2 / (n / 2) + (ones - n / 2) ** 2 / (n / 2))
    # 128 degrees of freedom: mean 128, sd 16
    assert chi2 < 128 + 6 * 16


def test_avalanche():
    n = 512
    c = np.arange(n, dtype=np.uint32)
    a = philox4x32_10(c, 0, 0, 0, 9, 9)
    b = philox4x32_10(c ^ np.uint32(1), 0, 0, 0, 9, 9)
    flips = sum(np.unpackbits((x ^ y).view(np.uint8)).sum() for x, y in zip(a, b))
    assert abs(flips / (n * 128) - 0.5) < 0.02


def test_sketch_columns_nearly_orthogonal():
    O = rademacher(4096, 64, seed=0, step=4)
    G = O.T @ O / 4096
    assert np.abs(G - np.eye(64)).max() < 6 / np.sqrt(4096)
