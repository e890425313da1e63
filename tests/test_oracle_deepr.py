"""Pins of the DEEP R oracle: scripted Fig. 2-shaped example, invariants, uniformity."""
import math

import numpy as np
import pytest

import synth
from oracle import deepr


def _bits_of_rows(row_len, ind, P, Q):
    out = np.zeros((P, (Q + 31) // 32), dtype=np.uint32)
    for i in range(P):
        for s in range(row_len[i]):
            j = int(ind[i, s])
            out[i, j >> 5] |= np.uint32(1 << (j & 31))
    return out


def _bit(words, i, j):
    j = int(j)
    return (int(words[i, j >> 5]) >> (j & 31)) & 1


def test_init_bitfields():
    rag = synth.random_ragged(3, 40, 70, 0.2)
    sign, conn = deepr.init_bitfields(rag.row_len, rag.ind, rag.w, 70, seed=5)
    np.testing.assert_array_equal(conn, _bits_of_rows(rag.row_len, rag.ind, 40, 70))
    for i in range(40):
        for s in range(rag.row_len[i]):
            assert _bit(sign, i, rag.ind[i, s]) == int(rag.w[i, s] > 0)
    frac = np.unpackbits(sign.view(np.uint8)).mean()
    assert 0.45 < frac < 0.55


def test_fig2_shaped_scripted_example():
    """5 pre x 4 post, max out-degree 3 (Fig. 2).  Rows and sign bits are scripted;
    weights whose sign disagrees with the sign bit are removed, survivors keep order."""
    P, Q, C = 5, 4, 3
    row_len = np.array([2, 3, 1, 0, 2], np.int32)
    ind = np.array([[1, 3, -1], [0, 2, 3], [2, -1, -1], [-1, -1, -1], [0, 1, -1]], np.int32)
    w = np.array([[0.5, -0.2, 0], [-0.1, 0.3, 0.0], [-0.4, 0, 0], [0, 0, 0], [0.2, 0.7, 0]])
    m = np.arange(15, dtype=float).reshape(5, 3)
    v = m + 100
    sign = np.zeros((P, 1), np.uint32)
    pos = {(0, 1), (0, 3), (1, 2), (1, 3), (2, 2), (4, 0)}     # (0,3) and (2,2) flipped to negative weights
    for i, j in pos:
        sign[i, 0] |= np.uint32(1 << j)
    conn = _bits_of_rows(row_len, ind, P, Q)
    nl, ni, nw, nm, nv, nc, dorm = deepr.eliminate(row_len, ind, w, m, v, sign, conn)
    # row 0: (0,3) w<0 vs positive bit -> removed ; row 1: (1,0) w<0 neg bit keep, (1,2) keep,
    # (1,3) w = 0 survives ; row 2: (2,2) removed ; row 4: (4,1) w>0 vs negative bit -> removed
    assert list(nl) == [1, 3, 0, 0, 1]
    assert list(dorm) == [1, 0, 1, 0, 1]
    assert list(ni[0, :1]) == [1] and list(ni[1, :3]) == [0, 2, 3] and list(ni[4, :1]) == [0]
    assert nm[1, 2] == m[1, 2] and nv[4, 0] == v[4, 0]
    np.testing.assert_array_equal(nc, _bits_of_rows(nl, ni, P, Q))
    taken, overflow = deepr.distribute(nl, dorm, C, Q, False, seed=1, rewire_idx=0)
    assert taken.sum() == 3 and overflow == 0
    assert np.all(taken <= np.minimum(C - nl, Q - nl))
    fl, fi, fw, fm, fv, fc = deepr.form(nl, ni, nw, nm, nv, nc, taken, Q, False, seed=1, rewire_idx=0)
    assert fl.sum() == row_len.sum()
    for i in range(P):
        tg = list(fi[i, :fl[i]])
        assert len(set(tg)) == len(tg)
        for s in range(nl[i], fl[i]):
            assert fw[i, s] == 0 and fm[i, s] == 0 and fv[i, s] == 0
    np.testing.assert_array_equal(fc, _bits_of_rows(fl, fi, P, Q))


@pytest.mark.parametrize("no_autapse", [False, True])
def test_invariants_random(no_autapse):
    P = Q = 64 if no_autapse else 50
    if not no_autapse:
        Q = 80
    rag = synth.random_ragged(7, P, Q, 0.15, no_autapse=no_autapse)
    sign, conn = deepr.init_bitfields(rag.row_len, rag.ind, rag.w, Q, seed=9)
    rng = np.random.default_rng(1)
    w = rag.w + np.where(rag.ind >= 0, rng.normal(0, 0.3, rag.w.shape), 0)   # some flip sign
    m = rng.normal(size=w.shape)
    v = rng.random(w.shape)
    total = rag.row_len.sum()
    row_len, ind, conn_c = rag.row_len, rag.ind, conn
    for ridx in range(3):
        out = deepr.rewire(row_len, ind, w, m, v, sign, conn_c, rag.C, Q, no_autapse, seed=21, rewire_idx=ridx)
        assert out["overflow"] == 0
        assert out["row_len"].sum() == total
        assert out["removed"] == out["formed"] == out["dormant"].sum()
        assert np.all(out["row_len"] <= rag.C)
        np.testing.assert_array_equal(out["conn"], _bits_of_rows(out["row_len"], out["ind"], P, Q))
        el = deepr.eliminate(row_len, ind, w, m, v, sign, conn_c)
        for i in range(P):
            tg = list(out["ind"][i, :out["row_len"][i]])
            assert len(set(tg)) == len(tg)
            if no_autapse:
                assert i not in tg
            for s in range(el[0][i]):      # survivors agree with the sign bit
                sb = _bit(sign, i, el[1][i, s])
                assert not ((sb and el[2][i, s] < 0) or (not sb and el[2][i, s] > 0))
        row_len, ind, w, m, v, conn_c = out["row_len"], out["ind"], out["w"], out["m"], out["v"], out["conn"]
        w = w + np.where(np.arange(rag.C)[None] < row_len[:, None], rng.normal(0, 0.3, w.shape), 0)


def test_formation_targets_uniform_chi2():
    """One free slot per call on a row with 4 of 20 targets taken: the new target is
    uniform over the 16 free ones (chi-square, 15 dof)."""
    Q, C, n = 20, 8, 4000
    row_len = np.array([4], np.int32)
    ind = np.array([[3, 7, 11, 19, -1, -1, -1, -1]], np.int32)
    z = np.zeros((1, C))
    conn = _bits_of_rows(row_len, ind, 1, Q)
    counts = np.zeros(Q)
    for r in range(n):
        fl, fi, *_ = deepr.form(row_len, ind, z, z, z, conn, np.array([1]), Q, False, seed=4, rewire_idx=r)
        counts[fi[0, 4]] += 1
    assert counts[[3, 7, 11, 19]].sum() == 0
    free = np.delete(counts, [3, 7, 11, 19])
    chi2 = ((free - n / 16) ** 2 / (n / 16)).sum()
    assert chi2 < 37.7     # p = 0.001 for 15 dof


def test_self_target_never_chosen_without_autapses():
    Q = 6
    row_len = np.zeros(Q, np.int32)
    ind = np.full((Q, Q), -1, np.int32)
    z = np.zeros((Q, Q))
    conn = np.zeros((Q, 1), np.uint32)
    for r in range(200):
        fl, fi, *_ = deepr.form(row_len, ind, z, z, z, conn, np.full(Q, 5), Q, True, seed=2, rewire_idx=r)
        for i in range(Q):
            assert sorted(fi[i, :5]) == [j for j in range(Q) if j != i]


def test_distribution_rows_uniform_chi2():
    P, C, Q = 10, 1000, 2000
    row_len = np.zeros(P, np.int32)
    dormant = np.zeros(P, np.int32)
    dormant[0] = 5000
    taken, overflow = deepr.distribute(row_len, dormant, C, Q, False, seed=3, rewire_idx=0)
    assert overflow == 0 and taken.sum() == 5000
    chi2 = ((taken - 500) ** 2 / 500).sum()
    assert chi2 < 27.9     # p = 0.001 for 9 dof


def test_distribution_respects_room_and_reports_overflow():
    P, C, Q = 4, 3, 10
    row_len = np.array([3, 3, 2, 3], np.int32)
    dormant = np.array([0, 0, 0, 5], np.int32)      # only 1 slot free in total
    taken, overflow = deepr.distribute(row_len, dormant, C, Q, False, seed=3, rewire_idx=0)
    assert list(taken) == [0, 0, 1, 0] and overflow == 4
