"""DEEP R on a ragged matrix with sign and connectivity bitfields — FP64 oracle
(test infrastructure).

Sec. 2.1.2 and Fig. 2 of the paper:

* init (Fig. 2A): clear all connectivity bits, randomise all sign bits, then for every
  initial synapse set its connectivity bit and force its sign bit to the sign of its
  weight (bit set = positive; a zero weight leaves the random bit).
* elimination (Fig. 2B): a synapse whose weight sign is strictly opposite to its sign
  bit is removed (a zero weight survives), the row's `dormant` counter counts the
  removals and the connectivity bit is cleared.  Rows are compacted stably: survivors
  keep their relative order (the paper's move-last removal yields the same row *set*).
* formation (Fig. 2C): the dormant counts are summed, D = sum dormant, and the D
  activations are redistributed uniformly over rows, then every activation creates a
  synapse to a random target that is not yet connected (connectivity bitfield as the
  duplicate check), with weight 0 and zero optimiser state (unreferenced variables of a
  new synapse start at zero, Sec. 2.1) and the potential connection's fixed sign.

Readings where the paper is silent (the same readings bind the CUDA path):
* "uniformly" redistributed: in rounds r = 0, 1, ...; round r draws its remaining
  activations' rows with Philox (DEEP_DIST; counter (rewire, r, k // 4), word k % 4,
  row = mulhi(u, P)); a row accepts min(count, room left) where its room is
  min(C - row_len, free targets); rejected activations go to round r + 1; after 64
  rounds the leftover count is reported as overflow.
* which target: the k-th activation of row i takes the m-th (0-based, ascending) free
  target with m = mulhi(u, n_free), u = Philox(DEEPR_FORM; (rewire, i, k)), where the
  self target of a recurrent projection without autapses counts as occupied.

Noise term (optional; Sec. 2.1.2 notes that the paper, like Bellec et al. 2020, leaves
out the noise of the original DEEP R, Bellec et al. 2018, whose parameter update adds
sqrt(2 eta T) nu with nu ~ N(0, 1) to every active parameter): `langevin_normals` gives
the nu of each active slot from Philox (DEEPR_NOISE; counter (noise_idx, row, slot, 0))
by the Box-Muller transform of words 0 and 1; the classifier oracle's Adam step adds
sqrt(2 lr T) nu after the Adam update.

Pins (tests/test_oracle_deepr.py): synapse count preserved; no duplicate targets;
survivors agree with their sign bits; bitfield == rows; dormant == removed; a scripted
5x4 example of Fig. 2's shape; chi-square uniformity of the chosen targets and of the
activation rows; zero-initialised state of new synapses; Box-Muller closed forms at the
ends of the word range and a Kolmogorov-Smirnov test against the normal law; guided
formation with equal (or all-zero) weights equals uniform formation bit for bit, the
weighted pick by hand, and the chosen targets' distances follow n(d^2) q[d^2].
"""
from __future__ import annotations

import math

import numpy as np

from . import philox


def _bit(words: np.ndarray, i: int, j: int) -> int:
    return (int(words[i, j >> 5]) >> (j & 31)) & 1


def init_bitfields(row_len, ind, w, Q: int, seed: int):
    """Fig. 2A: returns (sign_bits, conn_bits), uint32 [P, ceil(Q/32)]."""
    P = len(row_len)
    Qw = (Q + 31) // 32
    rows = np.repeat(np.arange(P, dtype=np.uint64), Qw)
    cols = np.tile(np.arange(Qw, dtype=np.uint64), P)
    u = philox.draw(seed, philox.SIGN, rows, cols, 0, 0, word=0)
    sign = (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).reshape(P, Qw)
    conn = np.zeros((P, Qw), dtype=np.uint32)
    for i in range(P):
        for s in range(int(row_len[i])):
            j = int(ind[i, s])
            conn[i, j >> 5] |= np.uint32(1 << (j & 31))
            if w[i, s] > 0:
                sign[i, j >> 5] |= np.uint32(1 << (j & 31))
            elif w[i, s] < 0:
                sign[i, j >> 5] &= np.uint32(~(1 << (j & 31)) & 0xFFFFFFFF)
    return sign, conn


def eliminate(row_len, ind, w, m, v, sign_bits, conn_bits):
    """Fig. 2B.  Returns new (row_len, ind, w, m, v, conn_bits, dormant); slots at or
    beyond the new row length are left as they were (only s < row_len is meaningful)."""
    row_len = row_len.copy()
    ind, w, m, v, conn = ind.copy(), w.copy(), m.copy(), v.copy(), conn_bits.copy()
    dormant = np.zeros(len(row_len), dtype=np.int32)
    for i in range(len(row_len)):
        n = int(row_len[i])
        keep = []
        for s in range(n):
            j = int(ind[i, s])
            sb = _bit(sign_bits, i, j)
            opposite = (sb == 1 and w[i, s] < 0) or (sb == 0 and w[i, s] > 0)
            if opposite:
                conn[i, j >> 5] &= np.uint32(~(1 << (j & 31)) & 0xFFFFFFFF)
            else:
                keep.append(s)
        k = len(keep)
        for arr in (ind, w, m, v):
            arr[i, :k] = arr[i, keep]
        dormant[i] = n - k
        row_len[i] = k
    return row_len, ind, w, m, v, conn, dormant


def n_forbidden(i: int, Q: int, no_autapse: bool) -> int:
    return 1 if (no_autapse and i < Q) else 0


def distribute(row_len, dormant, C: int, Q: int, no_autapse: bool, seed: int, rewire_idx: int,
               max_rounds: int = 64):
    """Redistribute D = sum(dormant) activations over rows.  Returns (taken[P], overflow)."""
    P = len(row_len)
    room = np.array([min(C - int(row_len[i]), Q - n_forbidden(i, Q, no_autapse) - int(row_len[i]))
                     for i in range(P)], dtype=np.int64)
    taken = np.zeros(P, dtype=np.int64)
    remaining = int(np.sum(dormant))
    r = 0
    while remaining > 0 and r < max_rounds:
        k = np.arange(remaining, dtype=np.uint64)
        u = philox.draw(seed, philox.DEEPR_DIST, np.uint64(rewire_idx), np.uint64(r), k // np.uint64(4), 0,
                        word=(k % np.uint64(4)).astype(np.int64))
        rows = philox.mulhi(u, P).astype(np.int64)
        cnt = np.bincount(rows, minlength=P)
        acc = np.minimum(cnt, room - taken)
        taken += acc
        remaining = int(np.sum(cnt - acc))
        r += 1
    return taken.astype(np.int32), remaining


def form(row_len, ind, w, m, v, conn_bits, taken, Q: int, no_autapse: bool, seed: int, rewire_idx: int):
    """Fig. 2C.  Appends taken[i] new synapses to row i.  Returns new arrays."""
    row_len = row_len.copy()
    ind, w, m, v, conn = ind.copy(), w.copy(), m.copy(), v.copy(), conn_bits.copy()
    for i in range(len(row_len)):
        forb = n_forbidden(i, Q, no_autapse)
        for k in range(int(taken[i])):
            n_free = Q - forb - int(row_len[i])
            u = philox.draw(seed, philox.DEEPR_FORM, np.uint64(rewire_idx), np.uint64(i), np.uint64(k), 0, word=0)
            mth = int(philox.mulhi(u, n_free))
            seen = -1
            target = -1
            for j in range(Q):
                if _bit(conn, i, j) or (forb and j == i):
                    continue
                seen += 1
                if seen == mth:
                    target = j
                    break
            assert target >= 0
            s = int(row_len[i])
            ind[i, s] = target
            w[i, s] = 0.0
            m[i, s] = 0.0
            v[i, s] = 0.0
            conn[i, target >> 5] |= np.uint32(1 << (target & 31))
            row_len[i] = s + 1
    return row_len, ind, w, m, v, conn


# ------------------------------------------------------------- distance-guided formation
#
# The paper's Discussion proposes guiding DEEP R's regrowth by the distance-dependent
# formation rule of the topographic map (Tab. 1-2) instead of choosing new targets
# uniformly.  Reading: neurons of both populations sit on sites of an L x L torus; the
# k-th activation of row i picks free target j with probability proportional to the
# integer weight q[d^2] = floor(2^24 exp(-d^2 / (2 sigma^2))), d the torus distance of the
# two sites: with S the weight total over the free targets (ascending j) and the same
# draw u as uniform formation, r = mulhi(u, S) selects the first free target whose
# running weight sum exceeds r.  Integer weights make the choice exact on both sides.
# A row whose free targets all have weight 0 falls back to the uniform choice.

def guide_weights(sigma: float, L: int) -> list[int]:
    """q[d2] = floor(2^24 exp(-d2 / (2 sigma^2))) for d2 = 0 .. 2 (L // 2)^2."""
    return [int(math.exp(-d2 / (2.0 * sigma * sigma)) * 2.0 ** 24) for d2 in range(2 * (L // 2) ** 2 + 1)]


def torus_d2_sites(a: int, b: int, L: int) -> int:
    dx = abs(a % L - b % L)
    dy = abs(a // L - b // L)
    dx = min(dx, L - dx)
    dy = min(dy, L - dy)
    return dx * dx + dy * dy


def weighted_pick(weights, r: int) -> int:
    """Index of the first entry whose running sum exceeds r (0 <= r < sum(weights)); the
    running sums are exact int64."""
    c = np.cumsum(np.asarray(weights, dtype=np.int64))
    if c.size == 0 or r >= c[-1]:
        raise ValueError("r beyond the weight total")
    return int(np.searchsorted(c, r, side="right"))


def form_guided(row_len, ind, w, m, v, conn_bits, taken, Q: int, no_autapse: bool, seed: int, rewire_idx: int,
                pre_site, post_site, L: int, q):
    """Fig. 2C with distance-guided target choice (see above).  Returns new arrays."""
    row_len = row_len.copy()
    ind, w, m, v, conn = ind.copy(), w.copy(), m.copy(), v.copy(), conn_bits.copy()
    q = np.asarray(q, dtype=np.int64)
    post = np.asarray(post_site, dtype=np.int64)
    j_all = np.arange(Q)
    for i in range(len(row_len)):
        if int(taken[i]) == 0:
            continue
        forb = n_forbidden(i, Q, no_autapse)
        a = int(pre_site[i])
        dx = np.abs(post % L - a % L)
        dy = np.abs(post // L - a // L)
        dx = np.minimum(dx, L - dx)
        dy = np.minimum(dy, L - dy)
        wt_all = q[dx * dx + dy * dy]                      # weight of every target of row i
        taken_bits = np.unpackbits(conn[i].view(np.uint8), bitorder="little")[:Q].astype(bool)
        if forb:
            taken_bits[i] = True
        for k in range(int(taken[i])):
            free = j_all[~taken_bits]                      # ascending
            u = philox.draw(seed, philox.DEEPR_FORM, np.uint64(rewire_idx), np.uint64(i), np.uint64(k), 0, word=0)
            wts = wt_all[free]
            S = int(wts.sum())
            if S > 0:
                # mulhi(u, S) = floor(u S / 2^64) with S up to 2^40: exact in Python integers
                # (philox.mulhi covers n < 2^32 only)
                target = int(free[weighted_pick(wts, (int(u) * S) >> 64)])
            else:
                target = int(free[int(philox.mulhi(u, len(free)))])
            s = int(row_len[i])
            ind[i, s] = target
            w[i, s] = 0.0
            m[i, s] = 0.0
            v[i, s] = 0.0
            conn[i, target >> 5] |= np.uint32(1 << (target & 31))
            taken_bits[target] = True
            row_len[i] = s + 1
    return row_len, ind, w, m, v, conn


def rewire(row_len, ind, w, m, v, sign_bits, conn_bits, C: int, Q: int, no_autapse: bool, seed: int,
           rewire_idx: int, guide=None):
    """Elimination, redistribution and formation in one call.  guide = (pre_site,
    post_site, L, q) selects the distance-guided formation.  Returns a dict."""
    row_len, ind, w, m, v, conn, dormant = eliminate(row_len, ind, w, m, v, sign_bits, conn_bits)
    taken, overflow = distribute(row_len, dormant, C, Q, no_autapse, seed, rewire_idx)
    if guide is None:
        row_len, ind, w, m, v, conn = form(row_len, ind, w, m, v, conn, taken, Q, no_autapse, seed, rewire_idx)
    else:
        row_len, ind, w, m, v, conn = form_guided(row_len, ind, w, m, v, conn, taken, Q, no_autapse, seed,
                                                  rewire_idx, *guide)
    return {"row_len": row_len, "ind": ind, "w": w, "m": m, "v": v, "conn": conn, "dormant": dormant,
            "taken": taken, "removed": int(dormant.sum()), "formed": int(taken.sum()), "overflow": overflow}


def box_muller(w0, w1) -> np.ndarray:
    """Standard normal from two uniform 64-bit words (Box & Muller, 1958):
    u1 = ((w0 >> 11) + 1) 2^-53 in (0, 1], u2 = (w1 >> 11) 2^-53 in [0, 1) (both exact),
    nu = sqrt(-2 ln u1) cos(2 pi u2)."""
    w0 = np.asarray(w0, dtype=np.uint64)
    w1 = np.asarray(w1, dtype=np.uint64)
    u1 = ((w0 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (w1 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def langevin_normals(seed: int, noise_idx: int, row_len, C: int) -> np.ndarray:
    """nu[i, s] ~ N(0, 1) for the active slots s < row_len[i] (0 on padding): Box-Muller
    of words 0 and 1 of Philox(seed, DEEPR_NOISE; (noise_idx, i, s, 0))."""
    P = len(row_len)
    i = np.repeat(np.arange(P, dtype=np.uint64), C)
    s = np.tile(np.arange(C, dtype=np.uint64), P)
    w0 = philox.draw(seed, philox.DEEPR_NOISE, np.uint64(noise_idx), i, s, 0, word=0)
    w1 = philox.draw(seed, philox.DEEPR_NOISE, np.uint64(noise_idx), i, s, 0, word=1)
    nu = box_muller(w0, w1).reshape(P, C)
    active = np.arange(C)[None, :] < np.asarray(row_len)[:, None]
    return np.where(active, nu, 0.0)
