"""Edge and degenerate cases of the CUDA path against the oracle: sizes that are not
multiples of 32 (ragged tail words) and that select each adjoint kernel (N % 4 == 0,
N even, N odd), the library's size limits, rows longer than one gather slot group,
split step windows, per-trial lengths, a silent network, empty propagation and a
rewiring with nothing dormant."""
import numpy as np
import pytest
import torch

import synth
from oracle import classifier as oc
from oracle import deepr as od
from tests import _setups

pytestmark = pytest.mark.gpu

F32, F64 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _forward(s, B, T, seed=0, record_state=True, trial_T=None, windows=None):
    from paper_2510_19764_gb300 import abi, net
    tb = synth.trial_batch(s.task, seed, 0, B)
    batch = net.DeviceBatch(s.dev, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=record_state,
                            trial_T=trial_T)
    for t0, n in (windows or [(0, T)]):
        abi.snn_step_neurons(s.dev.handle, batch.desc, t0, n)
    torch.cuda.synchronize()
    return tb, batch


def _host(batch, n_in, N):
    from paper_2510_19764_gb300 import net
    return {"x": net.spikes_from_bits(net.u32_to_numpy(batch.x_rec), n_in).astype(np.float64),
            "z": net.spikes_from_bits(net.u32_to_numpy(batch.z_rec), N).astype(np.float64),
            "psi": batch.psi_rec.double().cpu().numpy(), "d": batch.d_rec.double().cpu().numpy()}


def _grad_check(s, batch, B, tol):
    from paper_2510_19764_gb300 import abi
    abi.snn_eprop_update(s.dev.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
    torch.cuda.synchronize()
    g = _host(batch, s.onet.n_in, s.onet.N)
    Gi, Gr = np.zeros(s.in_rag.w.shape), np.zeros(s.rec_rag.w.shape)
    Go, Gb = np.zeros((s.onet.K, s.onet.N)), np.zeros(s.onet.K)
    for b in range(B):
        a, r_, o, bb = oc.eprop_gradients(s.onet, g["x"][b], g["z"][b], g["psi"][b], g["d"][b])
        Gi, Gr, Go, Gb = Gi + a, Gr + r_, Go + o, Gb + bb
    for got, ref, rag in ((s.dev.w_in.grad, Gi, s.in_rag), (s.dev.w_rec.grad, Gr, s.rec_rag)):
        got = got.double().cpu().numpy()
        mask = np.arange(rag.C)[None] < rag.row_len[:, None]
        scale = max(np.abs(ref[mask]).max(), 1e-30)
        np.testing.assert_allclose(got[mask], ref[mask], rtol=0, atol=tol * scale)
    np.testing.assert_allclose(s.dev.G_out.double().cpu().numpy(), Go, rtol=0, atol=tol * max(np.abs(Go).max(), 1e-30))
    np.testing.assert_allclose(s.dev.G_b.double().cpu().numpy(), Gb, rtol=0, atol=tol * max(1.0, np.abs(Gb).max()))
    return g


@pytest.mark.parametrize("N", [100, 98, 99])
def test_ragged_sizes_and_each_adjoint_kernel(N):
    """n_in = 45, K = 1 and N = 100 / 98 / 99 (tail words; the bulk-copy, packed and
    scalar FP32 adjoint kernels): FP64 rasters exact, FP32 gradients within 2e-5."""
    T, B, n_in = 90, 3, 45
    s64 = _setups.classifier(seed=11, dtype=F64, lif=False, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=1,
                             n_classes=1, n_bins=3, spoken=True, p_in=0.25, p_rec=0.15, w_scale=1.5)
    tb, batch = _forward(s64, B, T)
    g = _host(batch, n_in, N)
    for b in range(B):
        r = oc.forward_trial(s64.onet, s64.task.thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], s64.in_seed, T)
        np.testing.assert_array_equal(g["x"][b], r["x"])
        np.testing.assert_array_equal(g["z"][b], r["z"])
        np.testing.assert_allclose(g["d"][b], r["d"], rtol=1e-9, atol=1e-9)
    assert g["z"].sum() > 10
    s32 = _setups.classifier(seed=11, dtype=F32, lif=False, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=1,
                             n_classes=1, n_bins=3, spoken=True, p_in=0.25, p_rec=0.15, w_scale=1.5)
    _, batch32 = _forward(s32, B, T, record_state=False)
    _grad_check(s32, batch32, B, 2e-5)


def test_size_limits_one_step_parity():
    """The largest sizes the library accepts (n_in 1024, N 2048, K 32): each FP32 step
    from the kernel's own state matches one oracle step."""
    T, B, n_in, N, K = 12, 2, 1024, 2048, 32
    s = _setups.classifier(seed=5, dtype=F32, lif=False, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=K,
                           n_classes=4, n_bins=2, spoken=True, p_in=0.05, p_rec=0.05, w_scale=2.0)
    tb, batch = _forward(s, B, T)
    g = _host(batch, n_in, N)
    v, a, y = (t.double().cpu().numpy() for t in (batch.v_rec, batch.a_rec, batch.y_rec))
    for b in range(B):
        for t in range(1, T):
            st = {"v": v[b, t - 1], "a": a[b, t - 1], "z": g["z"][b, t - 1], "x": g["x"][b, t - 1], "y": y[b, t - 1]}
            r = oc.forward_trial(s.onet, s.task.thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], s.in_seed, 1,
                                 state=st, t0=t)
            np.testing.assert_array_equal(g["x"][b, t], r["x"][0])
            np.testing.assert_allclose(v[b, t], r["v"][0], rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(g["d"][b, t], r["d"][0], rtol=1e-5, atol=1e-6)
    assert g["z"].sum() > 0


def test_long_rows_span_several_gather_groups():
    """Recurrent rows of ~300 synapses (slots beyond 128 and 256 go to further gather
    CTAs): FP64 gradients equal the trace form within 1e-9."""
    T, B, n_in, N = 60, 2, 40, 512
    s = _setups.classifier(seed=13, dtype=F64, lif=True, v_thr=1.0, T=T, max_B=B, n_in=n_in, N=N, K=3,
                           p_in=0.3, p_rec=0.6, w_scale=0.3, rate_hz=60.0)
    assert s.rec_rag.row_len.max() > 256
    _, batch = _forward(s, B, T, record_state=False)
    g = _grad_check(s, batch, B, 1e-9)
    assert g["z"].sum() > 0


def test_split_windows_equal_one_call():
    """Steps run as three windows ([0,37), [37,38), [38,T)) give bit-identical records
    and state to one call."""
    T, B = 120, 4
    s = _setups.classifier(seed=6, dtype=F32, lif=False, v_thr=0.6, T=T, max_B=B, n_in=50, N=96, K=4,
                           n_classes=3, n_bins=3, spoken=True, p_in=0.2, p_rec=0.15, w_scale=1.5)
    _, one = _forward(s, B, T)
    _, split = _forward(s, B, T, windows=[(0, 37), (37, 1), (38, T - 38)])
    for k in ("x_rec", "z_rec", "psi_rec", "d_rec", "v_rec", "a_rec", "y_rec", "ysum", "v", "a", "y",
              "x_bits", "z_bits"):
        assert torch.equal(getattr(one, k), getattr(split, k)), k


def test_per_trial_lengths():
    """With trial_T, trial b runs exactly trial_T[b] steps: its records over those steps
    and its final readout sum equal a run of that trial alone for trial_T[b] steps."""
    from paper_2510_19764_gb300 import abi, net
    T, B = 100, 3
    lens = np.array([100, 37, 1], dtype=np.int32)
    s = _setups.classifier(seed=8, dtype=F32, lif=False, v_thr=0.6, T=T, max_B=B, n_in=50, N=96, K=4,
                           n_classes=3, n_bins=3, spoken=True, p_in=0.2, p_rec=0.15, w_scale=1.5)
    tb, mixed = _forward(s, B, T, trial_T=lens)
    for b in range(B):
        one = net.DeviceBatch(s.dev, tb.labels[b:b + 1], tb.bin_len[b:b + 1], tb.trial_ids[b:b + 1], int(lens[b]))
        abi.snn_step_neurons(s.dev.handle, one.desc, 0, int(lens[b]))
        torch.cuda.synchronize()
        n = int(lens[b])
        for k in ("x_rec", "z_rec", "psi_rec", "d_rec"):
            assert torch.equal(getattr(mixed, k)[b, :n], getattr(one, k)[0, :n]), (b, k)
        assert torch.equal(mixed.ysum[b], one.ysum[0])


def test_silent_network_has_only_bias_gradient():
    """All synaptic weights zero and no input: no hidden spike, so the ragged and
    readout-weight gradients are exactly zero and the bias gradient is sum_t d."""
    from paper_2510_19764_gb300 import abi
    T, B = 50, 2
    s = _setups.classifier(seed=3, dtype=F64, lif=True, v_thr=1.0, T=T, max_B=B, n_in=40, N=64, K=3,
                           w_scale=0.0, rate_hz=0.0)
    _, batch = _forward(s, B, T, record_state=False)
    abi.snn_eprop_update(s.dev.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
    torch.cuda.synchronize()
    g = _host(batch, 40, 64)
    assert g["z"].sum() == 0 and g["x"].sum() == 0
    assert torch.count_nonzero(s.dev.w_in.grad) == 0 and torch.count_nonzero(s.dev.w_rec.grad) == 0
    assert torch.count_nonzero(s.dev.G_out) == 0
    np.testing.assert_allclose(s.dev.G_b.double().cpu().numpy(), g["d"].sum(axis=(0, 1)), rtol=1e-12, atol=1e-12)


def test_propagate_empty_rows_and_tail_word():
    """P = 45 (a 13-bit tail word), an instance with no spikes, spiking rows of length 0:
    accumulators equal the oracle's dense masked sum, the silent instance stays zero."""
    from paper_2510_19764_gb300 import abi, net
    P, Q, B = 45, 70, 3
    rag = synth.random_ragged(21, P, Q, 0.2)
    rag.row_len[[3, 17, 44]] = 0
    r = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=F64)
    rng = np.random.default_rng(2)
    spk = rng.random((B, P)) < 0.5
    spk[1] = False
    spk[:, [3, 17, 44]] = True
    words = np.zeros((B, 2), dtype=np.uint32)
    for b in range(B):
        for i in np.nonzero(spk[b])[0]:
            words[b, i >> 5] |= np.uint32(1 << (i & 31))
    pre = torch.from_numpy(words.view(np.int32)).cuda()
    acc = torch.zeros((B, Q), dtype=torch.int64, device="cuda")
    abi.snn_propagate(r.handle, pre, B, acc)
    torch.cuda.synchronize()
    got = acc.double().cpu().numpy() / 2.0 ** 40
    for b in range(B):
        ref = oc.propagate(rag.row_len, rag.ind, rag.w, spk[b].astype(float), Q)
        np.testing.assert_allclose(got[b], ref, rtol=0, atol=1e-10)
    assert not got[1].any()


def test_rewire_with_nothing_dormant_is_a_no_op():
    """Every weight agrees with its sign bit: DEEP R removes and forms nothing and leaves
    every array bit for bit as it was."""
    from paper_2510_19764_gb300 import abi, net
    P, Q = 70, 90
    rag = synth.random_ragged(31, P, Q, 0.2)
    r = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=F32, adam=True, deepr=True, seed=5)
    torch.cuda.synchronize()
    before = r.host()
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    abi.snn_rewire_deepr(r.handle, 3, stats)
    torch.cuda.synchronize()
    after = r.host()
    assert stats.tolist() == [0, 0, 0, 0]
    for k in before:
        np.testing.assert_array_equal(before[k], after[k], err_msg=k)
    assert r.status() == abi.SNN_OK


def test_bounded_wait_gives_up_with_a_status_and_the_context_survives():
    """Failure detection without a fault: a bounded mbarrier wait on a barrier nothing
    completes gives up, the handle reports SNN_ETIMEOUT, and the GPU keeps working
    (a Philox draw afterwards equals the oracle's); the same wait on a completed barrier
    reports nothing."""
    import torch
    from oracle import philox as oph
    from paper_2510_19764_gb300 import abi, net
    rag = synth.random_ragged(3, 16, 32, 0.2)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, 32)
    abi.snn_test_wait_timeout(d.handle, True, 1 << 20)
    assert d.status() == abi.SNN_OK
    abi.snn_test_wait_timeout(d.handle, False, 1 << 16)
    assert d.status() == abi.SNN_ETIMEOUT
    assert d.status() == abi.SNN_OK                    # reading the status clears it
    ctr = torch.tensor([[7, 1, 2, 3]], dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    abi.snn_philox(5, 1, ctr, 1, out)
    got = net.u64_to_numpy(out)
    want = [int(oph.draw(5, 1, np.uint64(7), np.uint64(1), np.uint64(2), np.uint64(3), word=q)) for q in range(4)]
    assert [int(x) for x in got] == want


@pytest.mark.parametrize("where", ["one_weight", "input_column", "readout_column", "below_limit"])
def test_fixed_point_range_is_flagged(where):
    """The forward's sums are exact in fixed point while |sum| < 2^11.  A neuron or
    readout whose incoming |weight| sum reaches 2^11 (one oversized weight, many input
    weights onto one neuron, a readout's column of W_out) is reported as SNN_ESTATE;
    a sum just below the limit is not."""
    from paper_2510_19764_gb300 import abi, net
    s = _setups.classifier(seed=3, dtype=abi.SNN_F32, T=20, max_B=2, n_in=32, N=64, K=4, p_in=1.0)
    d = s.dev
    if where == "one_weight":
        d.w_in.w[0, 0] = 3000.0
    elif where == "input_column":
        # target of slot 0 of every input row: all 32 rows reach every target (p_in = 1)
        tgt = int(d.w_in.ind[0, 0])
        mask = d.w_in.ind == tgt
        d.w_in.w[mask] = 64.5                      # 32 x 64.5 = 2064 >= 2048
        assert int(mask.sum()) == 32
    elif where == "readout_column":
        d.W_out[1, :] = 32.5                       # 64 x 32.5 = 2080
    else:
        d.W_out[1, :] = 31.5                       # 64 x 31.5 = 2016 < 2048
    tb = synth.trial_batch(s.task, 0, 0, 2)
    batch = net.DeviceBatch(d, tb.labels, tb.bin_len, tb.trial_ids, 20)
    abi.snn_step_neurons(d.handle, batch.desc, 0, 20)
    torch.cuda.synchronize()
    want = abi.SNN_OK if where == "below_limit" else abi.SNN_ESTATE
    assert d.w_in.status() == want
