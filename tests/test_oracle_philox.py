"""Pins of the oracle's Philox4x64-10 and integer helpers (CPU only)."""
import numpy as np
import pytest

from oracle import philox


def _numpy_block(ctr, key):
    # numpy's Philox pre-increments its 256-bit counter before each block, so the block
    # for counter c is produced from state counter c - 1.
    c = list(ctr)
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


@pytest.mark.parametrize("trial", range(6))
def test_philox_matches_numpy_library(trial):
    rng = np.random.default_rng(trial)
    ctr = [int(x) for x in rng.integers(0, 2 ** 63, size=4)] if trial else [1, 0, 0, 0]
    if trial == 5:
        ctr = [0, 7, 0, 0]   # exercises the borrow in the counter shift
    key = [int(x) for x in rng.integers(0, 2 ** 63, size=2)]
    ours = philox.philox4x64(np.uint64(ctr[0]), np.uint64(ctr[1]), np.uint64(ctr[2]), np.uint64(ctr[3]), key[0], key[1])
    assert [int(x) for x in ours] == _numpy_block(ctr, key)


def test_philox_vectorised_equals_scalar():
    c0 = np.arange(50, dtype=np.uint64)
    out = philox.draw(1234, philox.INPUT, c0, 3, 5, 0, word=(c0 % np.uint64(4)).astype(np.int64))
    for i in range(50):
        ref = philox.philox4x64(np.uint64(i), np.uint64(3), np.uint64(5), np.uint64(0), 1234, philox.INPUT)[i % 4]
        assert int(out[i]) == int(ref)


def test_mulhi_matches_big_integers():
    rng = np.random.default_rng(7)
    u = rng.integers(0, 2 ** 64 - 1, size=2000, dtype=np.uint64, endpoint=True)
    n = rng.integers(1, 2 ** 32 - 1, size=2000, dtype=np.uint64)
    got = philox.mulhi(u, n)
    for a, b, g in zip(u, n, got):
        assert int(g) == (int(a) * int(b)) >> 64
    assert int(philox.mulhi(np.uint64(2 ** 64 - 1), 5)) == 4


def test_threshold_edges():
    assert philox.threshold(0.0) == 0
    assert philox.threshold(-1.0) == 0
    assert philox.threshold(0.5) == 2 ** 63
    assert philox.threshold(1.0) == 2 ** 64 - 1
    assert philox.threshold(1.225) == 2 ** 64 - 1
    assert philox.threshold(0.25) == 2 ** 62
