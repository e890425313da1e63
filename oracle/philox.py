"""Philox4x64-10 counter-based generator (oracle side; test infrastructure only).

Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
a 4 x 64-bit counter and a 2 x 64-bit key; each of 10 rounds multiplies counter words
0 and 2 by two fixed odd constants into 128-bit products and mixes hi/lo halves with the
other counter words and the key, and the key is bumped by two Weyl constants between
rounds.  The paper's method needs random numbers per row for regrowth ("Access to RNG",
Sec. 2.1; DEEP R formation, Sec. 2.1.2; rewiring attempts and probabilistic
elimination/formation, Sec. 2.1.3); a counter-based generator makes every draw a pure
function of (seed, purpose, counter) so that GPU threads and this oracle draw the same
numbers without sharing state.

Pinned against numpy.random.Philox (a library implementation of the same generator)
in tests/test_oracle_philox.py.

Conventions used by the whole method (both sides implement them independently):
  key     = (seed, purpose)
  counter = (c0, c1, c2, c3) purpose-specific fields
  uniform integer in [0, n):  (u * n) >> 64              (multiply-high, Lemire)
  Bernoulli(p):               u < thr,  thr = floor(p * 2^64) (saturated)
  32-bit Bernoulli(p) (classifier input only): one 32-bit half h of a word, h < thr32,
                              thr32 = floor(p * 2^32) (saturated)
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK64 = (1 << 64) - 1

# purposes (key word 1)
INPUT = 1          # classifier Poisson input: counter (trial, t, ch // 8, 0), word (ch % 8) // 2,
                   # 32-bit half ch % 2 (0: low, 1: high)
SIGN = 2           # DEEP R sign bitfield init: counter (row, word, 0, 0), word 0 low 32 bits
DEEPR_DIST = 3     # DEEP R activation rows: counter (rewire, round, k // 4, 0), word k % 4
DEEPR_FORM = 4     # DEEP R new target: counter (rewire, row, k, 0), word 0
TOPO_ATT = 5       # topo attempt rows: counter (rewire, k // 4, 0, 0), word k % 4
TOPO_CAND = 6      # topo candidate targets: counter (rewire, row, k, 0), word 0
TOPO_DRAW = 7      # topo elimination/formation R: counter (rewire, row, target, 0), word 0
TOPO_FOCUS = 8     # topo stimulus centre: counter (period, 0, 0, 0), words 0 (x), 1 (y)
TOPO_INPUT = 9     # topo Poisson input: counter (t, ch // 4, 0, 0), word ch % 4
DEEPR_NOISE = 10   # DEEP R noise term: counter (noise_idx, row, slot, 0), words 0 and 1

_U64 = np.uint64
_LO32 = _U64(0xFFFFFFFF)
_S32 = _U64(32)


def _mulhilo(a: int, b: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """128-bit product of a constant a and uint64 array b, as (hi, lo), using only
    32 x 32 -> 64 partial products (numpy has no 128-bit integers)."""
    a0, a1 = _U64(a & 0xFFFFFFFF), _U64(a >> 32)
    b0, b1 = b & _LO32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
    lo = (p00 & _LO32) | ((mid & _LO32) << _S32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0: int, k1: int) -> tuple[np.ndarray, ...]:
    """Philox4x64-10 of counter (c0..c3) (uint64 arrays, broadcast) under key (k0, k1)."""
    c = [np.asarray(x, dtype=np.uint64) for x in np.broadcast_arrays(c0, c1, c2, c3)]
    c = [x.copy() for x in c]
    k0 &= MASK64
    k1 &= MASK64
    with np.errstate(over="ignore"):
        for r in range(10):
            hi0, lo0 = _mulhilo(M0, c[0])
            hi1, lo1 = _mulhilo(M1, c[2])
            c = [hi1 ^ c[1] ^ _U64(k0), lo1, hi0 ^ c[3] ^ _U64(k1), lo0]
            k0 = (k0 + W0) & MASK64
            k1 = (k1 + W1) & MASK64
    return tuple(c)


def draw(seed: int, purpose: int, c0, c1=0, c2=0, c3=0, word=0) -> np.ndarray:
    """Word `word` (0..3, broadcastable array allowed) of Philox(key=(seed, purpose),
    counter=(c0, c1, c2, c3)) as uint64."""
    out = philox4x64(c0, c1, c2, c3, int(seed), int(purpose))
    word = np.asarray(word)
    if word.ndim == 0:
        return out[int(word)]
    stacked = np.stack(np.broadcast_arrays(*out, word)[:4], axis=0)
    w = np.broadcast_to(word, stacked.shape[1:])
    return np.take_along_axis(stacked, w[None].astype(np.int64), axis=0)[0]


def mulhi(u, n) -> np.ndarray:
    """floor(u * n / 2^64) for uint64 u and 0 <= n < 2^32 (uniform index in [0, n))."""
    u = np.asarray(u, dtype=np.uint64)
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        hi, lo = u >> _S32, u & _LO32
        # u * n = hi*n*2^32 + lo*n ; both partial products < 2^64 because n < 2^32
        t = hi * n + ((lo * n) >> _S32)
        return t >> _S32


def threshold(p: float) -> int:
    """64-bit Bernoulli threshold: floor(p * 2^64), 0 for p <= 0, 2^64-1 for p >= 1."""
    if p <= 0.0:
        return 0
    if p >= 1.0:
        return MASK64
    return int(p * float(2 ** 64))
