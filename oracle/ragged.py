"""Row updates of the ragged matrix — FP64 oracle (test infrastructure).

Sec. 2.1 of the paper: a custom connectivity update runs code per row of the ragged
matrix; the two listings there add the diagonal synapse (i, i) with weight 1 to every
row, and remove, from every row, the synapse to a target the host drew (if the row has
one).  Adding appends at the row's end (slot row_len) with the new synapse's other
variables at zero; removing takes the synapse out of the row.

Readings (shared with the CUDA path): one optional edit per row and call; a target
already in the row, a full row, a target outside [0, Q) or a forbidden self target
skips the add (the last two also flag an invalid state); removal keeps the order of the
remaining synapses (the paper moves the last synapse into the hole, which leaves the
same set of synapses in the row); the connectivity bitfield, where there is one, follows
the row.

Pins (tests/test_oracle_ragged.py): the diagonal and random-removal listings on small
matrices worked by hand; adds then removes of the same targets restore the rows.
"""
from __future__ import annotations

import numpy as np


def _bit(words, i, j):
    return (int(words[i, j >> 5]) >> (j & 31)) & 1


def row_add(row_len, ind, arrays, conn, targets, w_new, C: int, Q: int, no_autapse: bool = False):
    """Append synapse i -> targets[i] for every row with targets[i] >= 0.  `arrays` is a
    dict of per-slot variables; 'w' gets w_new[i] (0 if w_new is None), the others 0.
    Returns (row_len, ind, arrays, conn, added, skipped, invalid)."""
    row_len, ind = row_len.copy(), ind.copy()
    arrays = {k: v.copy() for k, v in arrays.items()}
    conn = None if conn is None else conn.copy()
    added = skipped = 0
    invalid = False
    for i in range(len(row_len)):
        t = int(targets[i])
        if t < 0:
            continue
        if t >= Q or (no_autapse and t == i):
            invalid = True
            skipped += 1
            continue
        n = int(row_len[i])
        present = t in set(int(x) for x in ind[i, :n])
        if present or n >= C:
            skipped += 1
            continue
        ind[i, n] = t
        for k, a in arrays.items():
            a[i, n] = (0.0 if w_new is None else float(w_new[i])) if k == "w" else 0.0
        if conn is not None:
            conn[i, t >> 5] |= np.uint32(1 << (t & 31))
        row_len[i] = n + 1
        added += 1
    return row_len, ind, arrays, conn, added, skipped, invalid


def row_remove(row_len, ind, arrays, conn, targets):
    """Remove synapse i -> targets[i] from every row that has it; the later synapses keep
    their order.  Returns (row_len, ind, arrays, conn, removed)."""
    row_len, ind = row_len.copy(), ind.copy()
    arrays = {k: v.copy() for k, v in arrays.items()}
    conn = None if conn is None else conn.copy()
    removed = 0
    for i in range(len(row_len)):
        t = int(targets[i])
        if t < 0:
            continue
        n = int(row_len[i])
        hits = [s for s in range(n) if int(ind[i, s]) == t]
        if not hits:
            continue
        s = hits[0]
        keep = [k for k in range(n) if k != s]
        ind[i, :n - 1] = ind[i, keep]
        for a in arrays.values():
            a[i, :n - 1] = a[i, keep]
        if conn is not None:
            conn[i, t >> 5] &= np.uint32(~(1 << (t & 31)) & 0xFFFFFFFF)
        row_len[i] = n - 1
        removed += 1
    return row_len, ind, arrays, conn, removed
