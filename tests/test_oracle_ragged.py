"""Pins of the row-update oracle: the paper's two custom connectivity update listings
(add the diagonal, remove a drawn target per row) on matrices worked by hand."""
import numpy as np

from oracle import ragged as orag


def _fig1_like():
    # 5 presynaptic rows, 4 targets, capacity 3 (out-degree 2 plus one free slot)
    row_len = np.array([2, 1, 2, 0, 2], np.int32)
    ind = np.array([[1, 3, -1], [0, -1, -1], [2, 0, -1], [-1, -1, -1], [3, 1, -1]], np.int32)
    w = np.array([[0.5, 0.25, 0], [2.0, 0, 0], [1.5, -1.0, 0], [0, 0, 0], [3.0, 4.0, 0]])
    conn = np.zeros((5, 1), np.uint32)
    for i in range(5):
        for s in range(row_len[i]):
            conn[i, 0] |= np.uint32(1 << int(ind[i, s]))
    return row_len, ind, w, conn


def test_add_diagonal_by_hand():
    row_len, ind, w, conn = _fig1_like()
    m = np.full_like(w, 7.0)
    targets = np.array([0, 1, 2, 3, 4], np.int32)        # (i, i); row 4's target 4 is outside Q = 4
    rl, ix, arr, cn, added, skipped, invalid = orag.row_add(row_len, ind, {"w": w, "m": m}, conn, targets,
                                                            np.ones(5), C=3, Q=4)
    # row 0: [1, 3] + 0; row 1: [0] + 1; row 2: [2, 0] already holds 2; row 3: [] + 3
    assert list(rl) == [3, 2, 2, 1, 2]
    assert list(ix[0, :3]) == [1, 3, 0] and list(ix[1, :2]) == [0, 1] and list(ix[3, :1]) == [3]
    assert arr["w"][0, 2] == 1.0 and arr["m"][0, 2] == 0.0 and arr["m"][0, 0] == 7.0
    assert (added, skipped, invalid) == (3, 2, True)
    assert int(cn[0, 0]) == 0b1011 and int(cn[3, 0]) == 0b1000
    # a full row skips
    rl2, _, _, _, added2, skipped2, _ = orag.row_add(rl, ix, {"w": arr["w"]}, cn, np.array([2, -1, -1, -1, -1]),
                                                     None, C=3, Q=4)
    assert rl2[0] == 3 and (added2, skipped2) == (0, 1)


def test_remove_drawn_target_by_hand():
    row_len, ind, w, conn = _fig1_like()
    targets = np.array([1, 2, 0, 1, -1], np.int32)      # row 1 has no 2, row 3 is empty
    rl, ix, arr, cn, removed = orag.row_remove(row_len, ind, {"w": w}, conn, targets)
    assert list(rl) == [1, 1, 1, 0, 2]
    assert list(ix[0, :1]) == [3] and arr["w"][0, 0] == 0.25      # later synapse moved down
    assert list(ix[2, :1]) == [2] and arr["w"][2, 0] == 1.5
    assert removed == 2
    assert int(cn[0, 0]) == 0b1000 and int(cn[2, 0]) == 0b0100


def test_add_then_remove_restores_rows():
    rng = np.random.default_rng(0)
    P, Q, C = 30, 50, 12
    row_len = rng.integers(0, 8, P).astype(np.int32)
    ind = np.full((P, C), -1, np.int32)
    w = np.zeros((P, C))
    for i in range(P):
        ind[i, :row_len[i]] = rng.choice(Q, row_len[i], replace=False)
        w[i, :row_len[i]] = rng.normal(size=row_len[i])
    targets = np.array([rng.choice([j for j in range(Q) if j not in set(ind[i, :row_len[i]])]) for i in range(P)],
                       np.int32)
    rl, ix, arr, _, added, _, _ = orag.row_add(row_len, ind, {"w": w}, None, targets, rng.normal(size=P), C, Q)
    assert added == P
    rl2, ix2, arr2, _, removed = orag.row_remove(rl, ix, arr, None, targets)
    assert removed == P
    np.testing.assert_array_equal(rl2, row_len)
    for i in range(P):
        np.testing.assert_array_equal(ix2[i, :row_len[i]], ind[i, :row_len[i]])
        np.testing.assert_array_equal(arr2["w"][i, :row_len[i]], w[i, :row_len[i]])
