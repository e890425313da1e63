"""GPU parity: Philox, ragged validation, DEEP R bitfield init, spike propagation."""
import numpy as np
import pytest
import torch

import synth
from oracle import classifier as oc
from oracle import deepr as od
from oracle import philox as oph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def test_philox_bit_exact():
    from paper_2510_19764_gb300 import abi, net
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 63, size=(n, 4), dtype=np.uint64)
    ctr[:5] = [[0, 0, 0, 0], [1, 0, 0, 0], [2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1], [7, 3, 1, 0],
               [12345, 678, 9, 1]]
    dctr = net._u64_tensor(ctr, "cuda")
    out = torch.empty((n, 4), dtype=torch.int64, device="cuda")
    for seed, purpose in ((0, 0), (2 ** 64 - 1, 9), (123456789, oph.INPUT)):
        abi.snn_philox(seed, purpose, dctr, n, out)
        got = net.u64_to_numpy(out)
        ref = np.stack(oph.philox4x64(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed, purpose), axis=1)
        np.testing.assert_array_equal(got, ref)


def test_create_rejects_invalid_rows():
    from paper_2510_19764_gb300 import abi, net
    row_len = np.array([2, 1], np.int32)
    for ind, no_aut in ((np.array([[1, 1], [0, 0]]), False),       # duplicate target
                        (np.array([[0, 5], [1, 0]]), False),       # target out of range
                        (np.array([[0, 1], [1, 0]]), True)):       # self target
        with pytest.raises(abi.SnnError) as e:
            net.DeviceRagged(row_len, ind, np.ones((2, 2)), 3, no_autapse=no_aut)
        assert e.value.status == abi.SNN_ESTATE
    with pytest.raises(abi.SnnError) as e:
        net.DeviceRagged(np.array([3, 0], np.int32), np.zeros((2, 2), np.int32), np.ones((2, 2)), 3)
    assert e.value.status == abi.SNN_ESTATE
    ok = net.DeviceRagged(row_len, np.array([[2, 0], [1, 0]]), np.ones((2, 2)), 3)
    assert ok.status() == abi.SNN_OK


@pytest.mark.parametrize("P,Q,no_aut", [(40, 70, False), (64, 64, True), (700, 1024, False)])
def test_deepr_bitfield_init_bit_exact(P, Q, no_aut):
    from paper_2510_19764_gb300 import net
    rag = synth.random_ragged(3, P, Q, 0.1, no_autapse=no_aut)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, no_autapse=no_aut, adam=True, deepr=True, seed=77)
    sign, conn = od.init_bitfields(rag.row_len, rag.ind, rag.w.astype(np.float32), Q, 77)
    np.testing.assert_array_equal(net.u32_to_numpy(d.sign_bits), sign)
    np.testing.assert_array_equal(net.u32_to_numpy(d.conn_bits), conn)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("P,Q,C,B", [(1, 1, 1, 1), (37, 53, 8, 3), (700, 1024, 288, 4), (1024, 1024, 64, 2)])
def test_propagate_matches_oracle(dtype, P, Q, C, B):
    from paper_2510_19764_gb300 import abi, net
    from tests._setups import as_dtype
    rag = synth.random_ragged(5, P, Q, min(0.5, C / (2.0 * Q)), C=C)
    rag.w = as_dtype(rag.w, dtype)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype)
    rng = np.random.default_rng(1)
    spikes = rng.random((B, P)) < 0.3
    spikes[0, :] = spikes[0, :] | (np.arange(P) == P - 1)            # ragged tail row
    bits = np.zeros((B, net.words(P)), np.uint32)
    for b in range(B):
        for i in np.nonzero(spikes[b])[0]:
            bits[b, i >> 5] |= np.uint32(1 << (i & 31))
    acc = torch.zeros((B, Q), dtype=torch.int64, device="cuda")
    abi.snn_propagate(d.handle, net._u32_tensor(bits, "cuda"), B, acc)
    got = acc.cpu().numpy().astype(np.float64) * 2.0 ** -abi.SNN_FIXED_FRAC_BITS
    for b in range(B):
        ref = oc.propagate(rag.row_len, rag.ind, rag.w, spikes[b], Q)
        # fixed-point quantisation: at most 2^-41 per addend
        np.testing.assert_allclose(got[b], ref, rtol=0, atol=P * 2.0 ** -40 + 1e-15)


def _spike_bits(rng, B, P, rate):
    from paper_2510_19764_gb300 import net
    spikes = rng.random((B, P)) < rate
    spikes[0, :] = spikes[0, :] | (np.arange(P) == P - 1)            # ragged tail row
    bits = np.zeros((B, net.words(P)), np.uint32)
    for b in range(B):
        for i in np.nonzero(spikes[b])[0]:
            bits[b, i >> 5] |= np.uint32(1 << (i & 31))
    return spikes, net._u32_tensor(bits, "cuda")


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("P,Q,C,B,max_B", [(1, 1, 1, 1, 1), (37, 53, 8, 3, 3), (700, 1024, 288, 4, 16),
                                           (1024, 1024, 64, 20, 20), (3000, 9000, 96, 17, 32)])
def test_propagate_tiled_equals_propagate(dtype, P, Q, C, B, max_B):
    """The target-tiled propagation adds the same int64 fixed-point sums as the row-major
    one (exact integers, order-free), for one and several instance groups, and matches
    the oracle; an unpacked plan adds nothing."""
    from paper_2510_19764_gb300 import abi, net
    from tests._setups import as_dtype
    rag = synth.random_ragged(6, P, Q, min(0.5, C / (2.0 * Q)), C=C)
    rag.w = as_dtype(rag.w, dtype)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype)
    spikes, bits = _spike_bits(np.random.default_rng(2), B, P, 0.3)
    plan = abi.snn_create_prop_plan(d.handle, max_B)
    try:
        acc = torch.zeros((B, Q), dtype=torch.int64, device="cuda")
        abi.snn_propagate_tiled(plan, bits, B, acc)
        torch.cuda.synchronize()
        assert int(acc.abs().sum()) == 0
        abi.snn_prop_plan_pack(plan)
        abi.snn_propagate_tiled(plan, bits, B, acc)
        ref = torch.zeros_like(acc)
        abi.snn_propagate(d.handle, bits, B, ref)
        torch.cuda.synchronize()
        assert torch.equal(acc, ref)
        got = acc.cpu().numpy().astype(np.float64) * 2.0 ** -abi.SNN_FIXED_FRAC_BITS
        for b in range(B):
            want = oc.propagate(rag.row_len, rag.ind, rag.w, spikes[b], Q)
            np.testing.assert_allclose(got[b], want, rtol=0, atol=P * 2.0 ** -40 + 1e-15)
        # accumulates into the caller's array
        abi.snn_propagate_tiled(plan, bits, B, acc)
        torch.cuda.synchronize()
        assert torch.equal(acc, 2 * ref)
        with pytest.raises(abi.SnnError):
            abi.snn_propagate_tiled(plan, bits, max_B + 1, acc)
        assert d.status() == abi.SNN_OK
    finally:
        abi.snn_destroy_prop_plan(plan)


def test_propagate_tiled_after_rewiring_and_large_weights():
    """Re-packing after a DEEP R rewiring follows the new synapses; weights near the
    fixed-point range (sums that carry across the 32-bit halves, both signs) stay exact."""
    from paper_2510_19764_gb300 import abi, net
    P, Q = 2048, 4096
    rag = synth.random_ragged(8, P, Q, 0.05, C=256)
    rng = np.random.default_rng(3)
    rag.w = np.where(rag.ind >= 0, rng.uniform(-3000.0, 3000.0, rag.w.shape), 0.0).astype(np.float32)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, adam=True, deepr=True, seed=9)
    _, bits = _spike_bits(rng, 16, P, 0.5)
    plan = abi.snn_create_prop_plan(d.handle, 16)
    try:
        for rep in range(2):
            if rep:
                live = torch.arange(d.C, device="cuda")[None, :] < d.row_len[:, None].long()
                flip = live & (torch.rand(d.w.shape, device="cuda") < 0.1)
                d.w[flip] = -d.w[flip]
                abi.snn_rewire_deepr(d.handle, 0)
            abi.snn_prop_plan_pack(plan)
            acc = torch.zeros((16, Q), dtype=torch.int64, device="cuda")
            ref = torch.zeros_like(acc)
            abi.snn_propagate_tiled(plan, bits, 16, acc)
            abi.snn_propagate(d.handle, bits, 16, ref)
            torch.cuda.synchronize()
            assert torch.equal(acc, ref)
            assert int((ref.abs() > 2 ** 51).sum()) > 0     # the high words carry real sums
        assert d.status() == abi.SNN_OK
    finally:
        abi.snn_destroy_prop_plan(plan)
