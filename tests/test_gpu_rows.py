"""GPU parity of the row updates (the paper's two custom connectivity update listings):
adding the diagonal and removing a drawn target per row, against the oracle, with and
without DEEP R bitfields, FP32 and FP64."""
import numpy as np
import pytest
import torch

import synth
from oracle import deepr as od
from oracle import ragged as orag
from tests._setups import as_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _check(d, rl, ind, arrays, conn):
    from paper_2510_19764_gb300 import net
    h = d.host()
    np.testing.assert_array_equal(h["row_len"], rl)
    mask = np.arange(d.C)[None] < rl[:, None]
    np.testing.assert_array_equal(h["ind"][mask], ind[mask])
    for k, a in arrays.items():
        np.testing.assert_array_equal(h[k][mask], a[mask])
    if conn is not None:
        np.testing.assert_array_equal(net.u32_to_numpy(d.conn_bits), conn)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bitfields", [False, True])
def test_add_diagonal_then_remove_drawn_targets(dtype, bitfields):
    from paper_2510_19764_gb300 import abi, net
    P = Q = 300
    rag = synth.random_ragged(17, P, Q, 0.05, C=32)
    rag.w = as_dtype(rag.w, dtype)
    rng = np.random.default_rng(4)
    m0 = as_dtype(rng.normal(size=rag.w.shape), dtype)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype, adam=True, deepr=bitfields, seed=3,
                         m=m0, v=np.abs(m0))
    conn = net.u32_to_numpy(d.conn_bits).copy() if bitfields else None
    arrays = {"w": rag.w.copy(), "m": m0.copy(), "v": np.abs(m0)}
    rl, ind = rag.row_len.copy(), rag.ind.copy()
    # listing 1: the diagonal with weight 1 (rows already holding i, or full, skip)
    ones = torch.ones(P, dtype=torch.float32 if dtype == 0 else torch.float64, device="cuda")
    diag = torch.arange(P, dtype=torch.int32, device="cuda")
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    abi.snn_ragged_add_row(d.handle, diag, ones, stats)
    torch.cuda.synchronize()
    rl, ind, arrays, conn, added, skipped, invalid = orag.row_add(rl, ind, arrays, conn, np.arange(P), np.ones(P),
                                                                  d.C, Q)
    _check(d, rl, ind, arrays, conn)
    assert int(stats[1]) == added > 200 and int(stats[2]) == skipped and not invalid
    # listing 2: a drawn target per row, removed if present (half the rows draw a target
    # they hold), some rows without an edit
    targets = rng.integers(0, Q, P).astype(np.int32)
    for i in range(0, P, 2):
        if rl[i] > 0:
            targets[i] = ind[i, rng.integers(0, rl[i])]
    targets[5::7] = -1
    stats.zero_()
    abi.snn_ragged_remove_row(d.handle, torch.as_tensor(targets, device="cuda"), stats)
    torch.cuda.synchronize()
    rl, ind, arrays, conn, removed = orag.row_remove(rl, ind, arrays, conn, targets)
    _check(d, rl, ind, arrays, conn)
    assert int(stats[0]) == removed > 100
    assert d.status() == abi.SNN_OK
    if bitfields:
        # DEEP R still sees consistent rows: one rewiring matches the oracle
        sign = net.u32_to_numpy(d.sign_bits).copy()
        w = arrays["w"].copy()
        mask = np.arange(d.C)[None] < rl[:, None]
        w[mask & (rng.random(w.shape) < 0.1)] *= -1.0
        d.w.copy_(torch.as_tensor(w))
        stats.zero_()
        abi.snn_rewire_deepr(d.handle, 0, stats)
        torch.cuda.synchronize()
        out = od.rewire(rl, ind, w, arrays["m"], arrays["v"], sign, conn, d.C, Q, False, 3, 0)
        _check(d, out["row_len"], out["ind"], {"w": out["w"], "m": out["m"], "v": out["v"]}, out["conn"])


def test_invalid_targets_flag_the_handle():
    from paper_2510_19764_gb300 import abi, net
    rag = synth.random_ragged(18, 20, 40, 0.1, no_autapse=True)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, 40, no_autapse=True)
    t = torch.full((20,), -1, dtype=torch.int32, device="cuda")
    t[3] = 3                                            # self target of a no_autapse matrix
    t[4] = 40                                           # outside Q
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    abi.snn_ragged_add_row(d.handle, t, None, stats)
    torch.cuda.synchronize()
    assert int(stats[2]) == 2 and int(stats[1]) == 0
    assert d.status() == abi.SNN_ESTATE
    np.testing.assert_array_equal(d.host()["row_len"], rag.row_len)
