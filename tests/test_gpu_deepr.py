"""GPU parity of DEEP R rewiring: bit-exact connectivity, moved state and counts."""
import numpy as np
import pytest
import torch

import synth
from oracle import deepr as od
from tests._setups import as_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _stats():
    return torch.zeros(4, dtype=torch.int64, device="cuda")


def _compare(d, out, stats):
    from paper_2510_19764_gb300 import abi
    h = d.host()
    np.testing.assert_array_equal(h["row_len"], out["row_len"])
    mask = np.arange(d.C)[None] < out["row_len"][:, None]
    np.testing.assert_array_equal(h["ind"][mask], out["ind"][mask])
    for k in ("w", "m", "v"):
        np.testing.assert_array_equal(h[k][mask], out[k][mask])
    np.testing.assert_array_equal(h["conn_bits"], out["conn"])
    st = stats.cpu().numpy()
    assert st[0] == out["removed"] and st[1] == out["formed"] and st[2] == out["overflow"]
    assert d.status() == (abi.SNN_OK if out["overflow"] == 0 else abi.SNN_ECAPACITY)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("P,Q,p,no_aut", [(5, 4, 0.5, False), (64, 64, 0.2, True), (700, 1024, 0.1, False),
                                          (1024, 1024, 0.1, True), (33, 1000, 0.05, False)])
def test_rewire_bit_exact(dtype, P, Q, p, no_aut):
    from paper_2510_19764_gb300 import abi, net
    rag = synth.random_ragged(11, P, Q, p, no_autapse=no_aut)
    rag.w = as_dtype(rag.w, dtype)
    rng = np.random.default_rng(5)
    m0 = as_dtype(rng.normal(size=rag.w.shape), dtype)
    v0 = as_dtype(rng.random(rag.w.shape), dtype)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype, no_autapse=no_aut, adam=True, deepr=True,
                         seed=99, m=m0, v=v0)
    sign = net.u32_to_numpy(d.sign_bits).copy()
    conn = net.u32_to_numpy(d.conn_bits).copy()
    state = (rag.row_len.copy(), rag.ind.copy(), rag.w.copy(), m0.copy(), v0.copy())
    for ridx in range(3):
        # drift weights so that a fraction of them flips sign (some land exactly on 0)
        rl, ind, w, m, v = state
        mask = np.arange(rag.C)[None] < rl[:, None]
        w = as_dtype(np.where(mask, w + rng.normal(0, 0.15, w.shape), w), dtype)
        w[mask & (rng.random(w.shape) < 0.02)] = 0.0
        d.w.copy_(torch.as_tensor(w))
        stats = _stats()
        abi.snn_rewire_deepr(d.handle, ridx, stats)
        torch.cuda.synchronize()
        out = od.rewire(rl, ind, w, m, v, sign, conn, rag.C, Q, no_aut, 99, ridx)
        assert out["removed"] > 0
        _compare(d, out, stats)
        state = (out["row_len"], out["ind"], out["w"], out["m"], out["v"])
        conn = out["conn"]


def test_fig2_shaped_scripted_example():
    """5 pre x 4 post, out-degree 3 with scripted sign bits (Fig. 2 shape)."""
    from paper_2510_19764_gb300 import abi, net
    P, Q, C = 5, 4, 3
    row_len = np.array([2, 3, 1, 0, 2], np.int32)
    ind = np.array([[1, 3, -1], [0, 2, 3], [2, -1, -1], [-1, -1, -1], [0, 1, -1]], np.int32)
    w = np.array([[0.5, -0.2, 0], [-0.1, 0.3, 0.0], [-0.4, 0, 0], [0, 0, 0], [0.2, 0.7, 0]])
    sign = np.zeros((P, 1), np.uint32)
    for i, j in {(0, 1), (0, 3), (1, 2), (1, 3), (2, 2), (4, 0)}:
        sign[i, 0] |= np.uint32(1 << j)
    d = net.DeviceRagged(row_len, ind, w, Q, dtype=1, adam=True, deepr=True, seed=1, sign_bits=sign)
    stats = _stats()
    abi.snn_rewire_deepr(d.handle, 0, stats)
    torch.cuda.synchronize()
    conn = np.zeros((P, 1), np.uint32)
    for i in range(P):
        for s in range(row_len[i]):
            conn[i, 0] |= np.uint32(1 << int(ind[i, s]))
    out = od.rewire(row_len, ind, w, np.zeros_like(w), np.zeros_like(w), sign, conn, C, Q, False, 1, 0)
    assert out["removed"] == 3
    _compare(d, out, stats)


def test_capacity_overflow_reported():
    """1000 full rows (every target taken) and one dormant synapse: its activation has
    to land on the one row with room, which 64 uniform rounds usually miss.  The kernel
    must agree with the oracle on where (if anywhere) it lands, count the leftover in
    the stats and report SNN_ECAPACITY in the status word (no device trap)."""
    from paper_2510_19764_gb300 import abi, net
    P, Q, C = 1000, 4, 4
    row_len = np.full(P, 4, np.int32)
    ind = np.tile(np.arange(4, dtype=np.int32), (P, 1))
    w = np.ones((P, C))
    d = net.DeviceRagged(row_len, ind, w, Q, dtype=1, adam=True, deepr=True, seed=3)
    sign = net.u32_to_numpy(d.sign_bits).copy()
    conn = net.u32_to_numpy(d.conn_bits).copy()
    w2 = w.copy()
    w2[7, 0] = -1.0
    d.w.copy_(torch.as_tensor(w2))
    overflowed = 0
    for ridx in range(4):
        stats = _stats()
        d.row_len.copy_(torch.as_tensor(row_len))
        d.ind.copy_(torch.as_tensor(ind))
        d.w.copy_(torch.as_tensor(w2))
        d.conn_bits.copy_(torch.as_tensor(conn.view(np.int32)))
        abi.snn_rewire_deepr(d.handle, ridx, stats)
        torch.cuda.synchronize()
        out = od.rewire(row_len, ind, w2, np.zeros_like(w), np.zeros_like(w), sign, conn, C, Q, False, 3, ridx)
        _compare(d, out, stats)
        overflowed += out["overflow"]
    assert overflowed > 0


def _guide(P, Q, L, sigma, seed):
    """Sites of both populations on an L x L torus: targets in grid order (Q <= L^2),
    sources spread over the grid by a seeded permutation."""
    from paper_2510_19764_gb300 import abi
    rng = np.random.default_rng(seed)
    pre = (rng.permutation(L * L)[:P] if P <= L * L else rng.integers(0, L * L, P)).astype(np.int32)
    post = np.arange(Q, dtype=np.int32) % (L * L)
    g = abi.DeeprGuide()
    g.L, g.reserved, g.sigma = L, 0, sigma
    pre_t = torch.as_tensor(pre, device="cuda")
    post_t = torch.as_tensor(post, device="cuda")
    g.pre_site, g.post_site = abi.ptr(pre_t), abi.ptr(post_t)
    return g, (pre_t, post_t), (pre, post, L, od.guide_weights(sigma, L))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("P,Q,p,no_aut,L,sigma", [(64, 64, 0.2, True, 8, 1.5), (700, 1024, 0.1, False, 32, 3.0),
                                                  (1024, 1024, 0.1, True, 32, 2.0), (33, 1000, 0.05, False, 32, 40.0),
                                                  (200, 256, 0.3, False, 16, 0.3)])
def test_guided_rewire_bit_exact(dtype, P, Q, p, no_aut, L, sigma):
    """Distance-guided formation (the Discussion's proposal) against the oracle: rows,
    moved state, bitfields and counts bit for bit, over three rewirings; sigma = 0.3
    leaves most rows' free targets weightless (uniform fallback)."""
    from paper_2510_19764_gb300 import abi, net
    rag = synth.random_ragged(12, P, Q, p, no_autapse=no_aut)
    rag.w = as_dtype(rag.w, dtype)
    rng = np.random.default_rng(6)
    z = np.zeros_like(rag.w)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype, no_autapse=no_aut, adam=True, deepr=True,
                         seed=77)
    g, keep, oguide = _guide(P, Q, L, sigma, 3)
    abi.snn_ragged_set_deepr_guide(d.handle, g)
    sign = net.u32_to_numpy(d.sign_bits).copy()
    conn = net.u32_to_numpy(d.conn_bits).copy()
    state = (rag.row_len.copy(), rag.ind.copy(), rag.w.copy(), z.copy(), z.copy())
    formed = 0
    for ridx in range(3):
        rl, ind, w, m, v = state
        mask = np.arange(rag.C)[None] < rl[:, None]
        w = as_dtype(np.where(mask, w + rng.normal(0, 0.15, w.shape), w), dtype)
        d.w.copy_(torch.as_tensor(w))
        stats = _stats()
        abi.snn_rewire_deepr(d.handle, ridx, stats)
        torch.cuda.synchronize()
        out = od.rewire(rl, ind, w, m, v, sign, conn, rag.C, Q, no_aut, 77, ridx, guide=oguide)
        _compare(d, out, stats)
        formed += out["formed"]
        state = (out["row_len"], out["ind"], out["w"], out["m"], out["v"])
        conn = out["conn"]
    assert formed > 0
    # detaching restores the uniform rule
    abi.snn_ragged_set_deepr_guide(d.handle, None)
    rl, ind, w, m, v = state
    mask = np.arange(rag.C)[None] < rl[:, None]
    w = as_dtype(np.where(mask, -w, w), dtype)              # every synapse turns dormant
    d.w.copy_(torch.as_tensor(w))
    stats = _stats()
    abi.snn_rewire_deepr(d.handle, 3, stats)
    torch.cuda.synchronize()
    _compare(d, od.rewire(rl, ind, w, m, v, sign, conn, rag.C, Q, no_aut, 77, 3), stats)


def test_guide_rejects_bad_sites_and_arguments():
    from paper_2510_19764_gb300 import abi, net
    rag = synth.random_ragged(13, 40, 64, 0.2)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, 64, adam=True, deepr=True, seed=1)
    g, keep, _ = _guide(40, 64, 8, 2.0, 1)
    keep[1][5] = 64                                   # outside the 8 x 8 grid
    with pytest.raises(abi.SnnError) as e:
        abi.snn_ragged_set_deepr_guide(d.handle, g)
    assert e.value.status == abi.SNN_ESTATE
    keep[1][5] = 5
    g.sigma = 0.0
    with pytest.raises(abi.SnnError):
        abi.snn_ragged_set_deepr_guide(d.handle, g)
    g.sigma = 2.0
    abi.snn_ragged_set_deepr_guide(d.handle, g)
    assert d.status() == abi.SNN_OK


def test_rows_rewritten_between_calls():
    """The handle caches each slot's sign bit tagged with its target.  A caller that
    reorders rows, moves synapses to other targets and shortens rows between rewirings
    (keeping the bitfields consistent) gets the oracle's result bit for bit."""
    from paper_2510_19764_gb300 import abi, net
    P, Q = 300, 700
    rag = synth.random_ragged(21, P, Q, 0.08, no_autapse=False)
    rng = np.random.default_rng(8)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=0, adam=True, deepr=True, seed=55)
    sign = net.u32_to_numpy(d.sign_bits).copy()
    rl, ind, w = rag.row_len.copy(), rag.ind.copy(), rag.w.copy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    conn = net.u32_to_numpy(d.conn_bits).copy()
    for ridx in range(4):
        mask = np.arange(rag.C)[None] < rl[:, None]
        w = as_dtype(np.where(mask, w + rng.normal(0, 0.1, w.shape), w), 0)
        if ridx > 0:
            # caller-side edits: shuffle every row, retarget one synapse of every third
            # row to a free target, drop the last synapse of every fifth row
            for i in range(P):
                n = int(rl[i])
                if n == 0:
                    continue
                perm = rng.permutation(n)
                for arr in (ind, w, m, v):
                    arr[i, :n] = arr[i, :n][perm]
                if i % 3 == 0:
                    taken = set(int(x) for x in ind[i, :n])
                    new = int(rng.choice([j for j in range(Q) if j not in taken]))
                    old = int(ind[i, 0])
                    conn[i, old >> 5] &= np.uint32(~(1 << (old & 31)) & 0xFFFFFFFF)
                    conn[i, new >> 5] |= np.uint32(1 << (new & 31))
                    ind[i, 0] = new
                if i % 5 == 0:
                    last = int(ind[i, n - 1])
                    conn[i, last >> 5] &= np.uint32(~(1 << (last & 31)) & 0xFFFFFFFF)
                    rl[i] = n - 1
            d.row_len.copy_(torch.as_tensor(rl))
            d.ind.copy_(torch.as_tensor(np.where(ind >= 0, ind, 0).astype(np.int32)))
            d.m.copy_(torch.as_tensor(m, dtype=torch.float32))
            d.v.copy_(torch.as_tensor(v, dtype=torch.float32))
            d.conn_bits.copy_(torch.as_tensor(conn.view(np.int32)))
        d.w.copy_(torch.as_tensor(w, dtype=torch.float32))
        stats = _stats()
        abi.snn_rewire_deepr(d.handle, ridx, stats)
        torch.cuda.synchronize()
        out = od.rewire(rl, ind, w, m, v, sign, conn, rag.C, Q, False, 55, ridx)
        assert out["removed"] > 0
        _compare(d, out, stats)
        rl, ind, w, m, v, conn = out["row_len"], out["ind"], out["w"], out["m"], out["v"], out["conn"]


@pytest.mark.parametrize("no_aut", [False, True])
def test_rewire_bit_exact_wide_rows(no_aut):
    """Rows of 65536 potential targets (64 chunks of 1024: two per lane in the
    register-resident formation), three sign flips per row, against the oracle."""
    from paper_2510_19764_gb300 import abi, net
    P, Q = 48, 65536
    rag = synth.random_ragged(31, P, Q, 0.003, C=384, no_autapse=no_aut)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=0, no_autapse=no_aut, adam=True, deepr=True, seed=9)
    sign = net.u32_to_numpy(d.sign_bits).copy()
    conn = net.u32_to_numpy(d.conn_bits).copy()
    rl, ind = rag.row_len.copy(), rag.ind.copy()
    w = as_dtype(rag.w, 0)
    z = np.zeros_like(w)
    rng = np.random.default_rng(2)
    for ridx in range(2):
        for i in range(P):
            for s in rng.choice(int(rl[i]), size=min(3, int(rl[i])), replace=False):
                w[i, s] = -w[i, s]
        d.w.copy_(torch.as_tensor(w, dtype=torch.float32))
        stats = _stats()
        abi.snn_rewire_deepr(d.handle, ridx, stats)
        torch.cuda.synchronize()
        out = od.rewire(rl, ind, w, z, z, sign, conn, rag.C, Q, no_aut, 9, ridx)
        assert out["formed"] > 0
        _compare(d, out, stats)
        rl, ind, w, conn = out["row_len"], out["ind"], out["w"], out["conn"]


def test_refused_rewire_leaves_matrix_untouched():
    """A rewiring whose formation table would not fit (Q > ~1.57 M targets) is refused
    with SNN_EINVAL before any kernel runs: row lengths, targets and bitfields stay as
    they were, so the synapse count is not left pruned without regrowth."""
    from paper_2510_19764_gb300 import abi, net
    P, Q, C = 2, 1_700_000, 4
    ind = np.array([[5, 1_600_000, -1, -1], [7, 9, 11, -1]], dtype=np.int32)
    row_len = np.array([2, 3], dtype=np.int32)
    w = np.array([[0.5, -0.25, 0, 0], [0.1, 0.2, -0.3, 0]])
    d = net.DeviceRagged(row_len, ind, w, Q, adam=True, deepr=True, seed=3)
    d.w.neg_()                                     # every synapse now opposes its sign bit
    before = {k: getattr(d, k).clone() for k in ("row_len", "ind", "w", "conn_bits")}
    with pytest.raises(abi.SnnError) as e:
        abi.snn_rewire_deepr(d.handle, 0, _stats())
    assert e.value.status == abi.SNN_EINVAL
    torch.cuda.synchronize()
    for k, t in before.items():
        assert torch.equal(getattr(d, k), t), k
    assert d.status() == abi.SNN_OK
