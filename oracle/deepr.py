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

Pins (tests/test_oracle_deepr.py): synapse count preserved; no duplicate targets;
survivors agree with their sign bits; bitfield == rows; dormant == removed; a scripted
5x4 example of Fig. 2's shape; chi-square uniformity of the chosen targets and of the
activation rows; zero-initialised state of new synapses.
"""
from __future__ import annotations

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


def rewire(row_len, ind, w, m, v, sign_bits, conn_bits, C: int, Q: int, no_autapse: bool, seed: int,
           rewire_idx: int):
    """Elimination, redistribution and formation in one call.  Returns a dict."""
    row_len, ind, w, m, v, conn, dormant = eliminate(row_len, ind, w, m, v, sign_bits, conn_bits)
    taken, overflow = distribute(row_len, dormant, C, Q, no_autapse, seed, rewire_idx)
    row_len, ind, w, m, v, conn = form(row_len, ind, w, m, v, conn, taken, Q, no_autapse, seed, rewire_idx)
    return {"row_len": row_len, "ind": ind, "w": w, "m": m, "v": v, "conn": conn, "dormant": dormant,
            "taken": taken, "removed": int(dormant.sum()), "formed": int(taken.sum()), "overflow": overflow}
