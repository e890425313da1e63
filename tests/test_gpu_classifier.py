"""GPU parity of the classifier path: forward (raster, voltages, readout), e-prop
gradient, L1 + Adam, and a full e-prop + DEEP R training run against the FP64 oracle."""
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


def _run_forward(s, B, T, seed=0, batch_idx=0, record_state=True):
    from paper_2510_19764_gb300 import abi, net
    tb = synth.trial_batch(s.task, seed, batch_idx, B)
    batch = net.DeviceBatch(s.dev, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=record_state)
    abi.snn_step_neurons(s.dev.handle, batch.desc, 0, T)
    torch.cuda.synchronize()
    return tb, batch


def _host(batch, s):
    from paper_2510_19764_gb300 import net
    n_in, N = s.onet.n_in, s.onet.N
    out = {"x": net.spikes_from_bits(net.u32_to_numpy(batch.x_rec), n_in).astype(np.float64),
           "z": net.spikes_from_bits(net.u32_to_numpy(batch.z_rec), N).astype(np.float64),
           "psi": batch.psi_rec.double().cpu().numpy(), "d": batch.d_rec.double().cpu().numpy(),
           "ysum": batch.ysum.double().cpu().numpy()}
    if batch.v_rec is not None:
        out.update(v=batch.v_rec.double().cpu().numpy(), a=batch.a_rec.double().cpu().numpy(),
                   y=batch.y_rec.double().cpu().numpy())
    return out


@pytest.mark.parametrize("lif", [True, False])
def test_forward_f64_raster_exact(lif):
    """FP64 build: input and hidden rasters identical to the oracle's, continuous
    records equal up to the fixed-point accumulator quantisation."""
    T, B = 200, 4
    s = _setups.classifier(seed=0, dtype=F64, lif=lif, v_thr=1.0 if lif else 0.6, T=T, max_B=B)
    tb, batch = _run_forward(s, B, T)
    g = _host(batch, s)
    total = 0
    for b in range(B):
        r = oc.forward_trial(s.onet, s.task.thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], s.in_seed, T)
        np.testing.assert_array_equal(g["x"][b], r["x"])
        np.testing.assert_array_equal(g["z"][b], r["z"])
        for k in ("v", "a", "psi", "y", "d"):
            np.testing.assert_allclose(g[k][b], r[k], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(g["ysum"][b], r["ysum"], rtol=1e-9, atol=1e-9)
        total += r["z"].sum()
    assert total > 0


@pytest.mark.parametrize("lif", [True, False])
def test_forward_f32_per_step(lif):
    """FP32: from the kernel's own state at t-1, one oracle step reproduces step t:
    input spikes exactly, v, a, y, psi, d within 1e-5 relative, spikes except where the
    margin to threshold is below the FP32 error."""
    T, B, n_in, N, K = 80, 3, 100, 128, 8
    s = _setups.classifier(seed=4, dtype=F32, lif=lif, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=K,
                           n_classes=5, n_bins=4, spoken=True, p_in=0.2, p_rec=0.1, w_scale=1.5)
    tb, batch = _run_forward(s, B, T)
    g = _host(batch, s)
    flips = 0
    for b in range(B):
        for t in range(1, T):
            st = {"v": g["v"][b, t - 1], "a": g["a"][b, t - 1], "z": g["z"][b, t - 1], "x": g["x"][b, t - 1],
                  "y": g["y"][b, t - 1]}
            r = oc.forward_trial(s.onet, s.task.thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], s.in_seed, 1,
                                 state=st, t0=t)
            np.testing.assert_array_equal(g["x"][b, t], r["x"][0])
            for k in ("v", "a", "psi", "y", "d"):
                np.testing.assert_allclose(g[k][b, t], r[k][0], rtol=1e-5, atol=1e-6)
            A = s.onet.neuron.v_thr + s.onet.neuron.beta * r["a"][0]
            differ = g["z"][b, t] != r["z"][0]
            assert np.all(np.abs(r["v"][0] - A)[differ] < 1e-5)
            flips += differ.sum()
    assert flips <= 2
    assert g["z"].sum() > 50


@pytest.mark.parametrize("dtype,lif", [(F64, True), (F64, False), (F32, False)])
def test_eprop_gradient_matches_trace_form(dtype, lif):
    """The adjoint/event form on the GPU equals the oracle's forward-trace e-prop
    gradients computed from the same records, summed over trials."""
    from paper_2510_19764_gb300 import abi
    T, B, n_in, N, K = 120, 5, 60, 96, 6
    s = _setups.classifier(seed=9, dtype=dtype, lif=lif, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=K,
                           n_classes=3, n_bins=3, spoken=True, p_in=0.2, p_rec=0.15, w_scale=1.5)
    tb, batch = _run_forward(s, B, T, record_state=False)
    abi.snn_eprop_update(s.dev.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
    torch.cuda.synchronize()
    g = _host(batch, s)
    Gi = np.zeros(s.in_rag.w.shape)
    Gr = np.zeros(s.rec_rag.w.shape)
    Go = np.zeros((K, N))
    Gb = np.zeros(K)
    for b in range(B):
        a, r_, o, bb = oc.eprop_gradients(s.onet, g["x"][b], g["z"][b], g["psi"][b], g["d"][b])
        Gi += a
        Gr += r_
        Go += o
        Gb += bb
    tol = 1e-9 if dtype == F64 else 2e-5
    for got, ref, rag in ((s.dev.w_in.grad, Gi, s.in_rag), (s.dev.w_rec.grad, Gr, s.rec_rag)):
        got = got.double().cpu().numpy()
        mask = np.arange(rag.C)[None] < rag.row_len[:, None]
        scale = np.abs(ref[mask]).max()
        assert scale > 0
        np.testing.assert_allclose(got[mask], ref[mask], rtol=0, atol=tol * scale)
    np.testing.assert_allclose(s.dev.G_out.double().cpu().numpy(), Go, rtol=0, atol=tol * np.abs(Go).max())
    np.testing.assert_allclose(s.dev.G_b.double().cpu().numpy(), Gb, rtol=0, atol=tol * max(1.0, np.abs(Gb).max()))


@pytest.mark.parametrize("dtype", [F32, F64])
def test_adam_l1_apply(dtype):
    from paper_2510_19764_gb300 import abi, net
    s = _setups.classifier(seed=2, dtype=dtype, lif=False, T=10, max_B=1, n_in=50, N=70, K=5)
    rng = np.random.default_rng(3)
    host = {}
    for name, d, rag in (("in", s.dev.w_in, s.in_rag), ("rec", s.dev.w_rec, s.rec_rag)):
        G = _setups.as_dtype(rng.normal(0, 1, rag.w.shape), dtype)
        m0 = _setups.as_dtype(rng.normal(0, 0.1, rag.w.shape), dtype)
        v0 = _setups.as_dtype(rng.random(rag.w.shape) * 0.01, dtype)
        d.grad.copy_(torch.as_tensor(G))
        d.m.copy_(torch.as_tensor(m0))
        d.v.copy_(torch.as_tensor(v0))
        host[name] = (G, m0, v0, net.u32_to_numpy(d.sign_bits), rag)
    Go = _setups.as_dtype(rng.normal(size=(5, 70)), dtype)
    Gb = _setups.as_dtype(rng.normal(size=5), dtype)
    s.dev.G_out.copy_(torch.as_tensor(Go))
    s.dev.G_b.copy_(torch.as_tensor(Gb))
    W0 = s.dev.W_out.double().cpu().numpy()
    b0 = s.dev.b_out.double().cpu().numpy()
    ad = net.adam_params(1e-3, 3, l1=1e-2)
    abi.snn_eprop_update(s.dev.handle, None, abi.SNN_EPROP_APPLY, ad)
    torch.cuda.synchronize()
    # FP32: each stored value is within a few float32 ulps of the FP64 update; moments
    # that cancel towards zero keep the absolute error of their terms (|m|, |v| <~ 1)
    rtol, atol = (1e-6, 1e-7) if dtype == F32 else (1e-13, 1e-15)
    for name, d in (("in", s.dev.w_in), ("rec", s.dev.w_rec)):
        G, m0, v0, sign, rag = host[name]
        Gl = oc.l1_on_sign(G, rag.row_len, rag.ind, sign, 1e-2)
        w, m, v = oc.adam_ragged(rag.w, m0, v0, Gl, rag.row_len, 1e-3, oc.adam_bias(0.9, 3),
                                 oc.adam_bias(0.999, 3))
        mask = np.arange(rag.C)[None] < rag.row_len[:, None]
        for got, ref in ((d.w, w), (d.m, m), (d.v, v)):
            np.testing.assert_allclose(got.double().cpu().numpy()[mask], ref[mask], rtol=rtol, atol=atol)
    w, m, v = oc.adam(W0, 0 * W0, 0 * W0, Go, 1e-3, oc.adam_bias(0.9, 3), oc.adam_bias(0.999, 3))
    np.testing.assert_allclose(s.dev.W_out.double().cpu().numpy(), w, rtol=rtol, atol=atol)
    w, m, v = oc.adam(b0, 0 * b0, 0 * b0, Gb, 1e-3, oc.adam_bias(0.9, 3), oc.adam_bias(0.999, 3))
    np.testing.assert_allclose(s.dev.b_out.double().cpu().numpy(), w, rtol=rtol, atol=atol)


def test_adam_step_from_device_memory_equals_host_step():
    """The Adam step count read from device memory (graph replay) gives the same update,
    bit for bit, as the count passed by value: steps 1, 2, then a jump to 7 and back to 3
    (the library re-forms the running products), in FP32 and FP64."""
    from paper_2510_19764_gb300 import abi, net
    for dtype in (F32, F64):
        a = _setups.classifier(seed=8, dtype=dtype, lif=False, T=10, max_B=1, n_in=40, N=64, K=3)
        b = _setups.classifier(seed=8, dtype=dtype, lif=False, T=10, max_B=1, n_in=40, N=64, K=3)
        rng = np.random.default_rng(1)
        t_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        for step in (1, 2, 7, 3):
            for x, y in ((a.dev.w_in, b.dev.w_in), (a.dev.w_rec, b.dev.w_rec)):
                G = torch.as_tensor(rng.normal(size=x.w.shape), dtype=x.w.dtype, device="cuda")
                x.grad.copy_(G)
                y.grad.copy_(G)
            Go = torch.as_tensor(rng.normal(size=a.dev.G_out.shape), dtype=a.dev.G_out.dtype, device="cuda")
            for c in (a.dev, b.dev):
                c.G_out.copy_(Go)
                c.G_b.fill_(0.25)
            t_dev.fill_(step)
            abi.snn_eprop_update(a.dev.handle, None, abi.SNN_EPROP_APPLY, net.adam_params(1e-2, step, l1=1e-3))
            abi.snn_eprop_update(b.dev.handle, None, abi.SNN_EPROP_APPLY,
                                 net.adam_params(1e-2, 1, l1=1e-3, step_dev=t_dev))
            torch.cuda.synchronize()
            for x, y in ((a.dev.w_in, b.dev.w_in), (a.dev.w_rec, b.dev.w_rec)):
                assert torch.equal(x.w, y.w) and torch.equal(x.m, y.m) and torch.equal(x.v, y.v)
            assert torch.equal(a.dev.W_out, b.dev.W_out) and torch.equal(a.dev.b_out, b.dev.b_out)
        assert a.dev.w_in.status() == abi.SNN_OK and b.dev.w_in.status() == abi.SNN_OK


@pytest.mark.parametrize("dtype", [F32, F64])
def test_adam_noise_apply(dtype):
    """DEEP R's noise term: after the Adam step every active ragged weight adds
    sqrt(2 lr T) nu with the oracle's Box-Muller normals (host counter, then the device
    counter); the dense readout gets no noise; padding slots stay untouched."""
    from paper_2510_19764_gb300 import abi, net
    s = _setups.classifier(seed=4, dtype=dtype, lif=False, T=10, max_B=1, n_in=40, N=90, K=3)
    rng = np.random.default_rng(5)
    lr, temp = 1e-3, 2e-3
    idx_dev = torch.tensor([7], dtype=torch.int64, device="cuda")
    for step, (noise_idx, dev_idx) in enumerate(((5, None), (0, idx_dev)), start=1):
        host = {}
        for name, d in (("in", s.dev.w_in), ("rec", s.dev.w_rec)):
            G = _setups.as_dtype(rng.normal(0, 1, d.w.shape), dtype)
            d.grad.copy_(torch.as_tensor(G))
            host[name] = (G, d.host())
        Go = np.zeros((3, 90))
        s.dev.G_out.copy_(torch.as_tensor(Go))
        s.dev.G_b.zero_()
        W0 = s.dev.W_out.double().cpu().numpy()
        ad = net.adam_params(lr, step, temperature=temp, noise_idx=noise_idx, noise_idx_dev=dev_idx)
        abi.snn_eprop_update(s.dev.handle, None, abi.SNN_EPROP_APPLY, ad)
        torch.cuda.synchronize()
        rtol, atol = (1e-6, 1e-7) if dtype == F32 else (1e-13, 1e-15)
        k = 7 if dev_idx is not None else noise_idx
        for name, d in (("in", s.dev.w_in), ("rec", s.dev.w_rec)):
            G, h = host[name]
            nu = od.langevin_normals(d.desc.seed, k, h["row_len"], d.C)
            w, m, v = oc.adam_ragged(h["w"], h["m"], h["v"], G, h["row_len"], lr, oc.adam_bias(0.9, step),
                                     oc.adam_bias(0.999, step), temperature=temp, nu=nu)
            got = d.host()
            np.testing.assert_allclose(got["w"], w, rtol=rtol, atol=atol)       # padding included
            np.testing.assert_allclose(got["m"], m, rtol=rtol, atol=atol)
            assert np.abs(nu).max() > 1.0
        # readout: plain Adam on a zero gradient leaves W_out unchanged
        np.testing.assert_array_equal(s.dev.W_out.double().cpu().numpy(), W0)
    with pytest.raises(abi.SnnError):
        abi.snn_eprop_update(s.dev.handle, None, abi.SNN_EPROP_APPLY, net.adam_params(lr, 1, temperature=-1.0))


def _oracle_train(s, batches, lr, l1, T, temperature=0.0):
    """Oracle training run: per batch forward all trials, sum gradients, L1 + Adam,
    DEEP R on both projections (bitfields from the oracle's own init)."""
    n = s.onet
    seed_in, seed_rec = s.dev.w_in.desc.seed, s.dev.w_rec.desc.seed
    sign_in = od.init_bitfields(n.in_len, n.in_ind, n.w_in, n.N, seed_in)[0]
    sign_rec = od.init_bitfields(n.rec_len, n.rec_ind, n.w_rec, n.N, seed_rec)[0]
    st = {"in": [n.in_len.copy(), n.in_ind.copy(), n.w_in.copy(), np.zeros_like(n.w_in), np.zeros_like(n.w_in)],
          "rec": [n.rec_len.copy(), n.rec_ind.copy(), n.w_rec.copy(), np.zeros_like(n.w_rec), np.zeros_like(n.w_rec)]}
    conn = {"in": od.init_bitfields(n.in_len, n.in_ind, n.w_in, n.N, 0)[1],
            "rec": od.init_bitfields(n.rec_len, n.rec_ind, n.w_rec, n.N, 0)[1]}
    sign = {"in": sign_in, "rec": sign_rec}
    W, b = n.W_out.copy(), n.b_out.copy()
    mW, vW, mb, vb = np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)
    b1t = b2t = 1.0
    rasters, preds = [], []
    for bi, tb in enumerate(batches):
        net_b = oc.ClassifierNet(n.n_in, n.N, n.K, st["in"][0], st["in"][1], st["in"][2], st["rec"][0],
                                 st["rec"][1], st["rec"][2], W, b, n.neuron)
        G = {"in": 0, "rec": 0}
        Go, Gb = 0, 0
        for k in range(len(tb.labels)):
            r = oc.forward_trial(net_b, s.task.thr, tb.labels[k], tb.bin_len[k], tb.trial_ids[k], s.in_seed, T)
            rasters.append(r["z"])
            preds.append(r["pred"])
            gi, gr, go, gb = oc.eprop_gradients(net_b, r["x"], r["z"], r["psi"], r["d"])
            G["in"] = G["in"] + gi
            G["rec"] = G["rec"] + gr
            Go, Gb = Go + go, Gb + gb
        b1t *= 0.9
        b2t *= 0.999
        for name in ("in", "rec"):
            rl, ind, w, m, v = st[name]
            Gl = oc.l1_on_sign(G[name], rl, ind, sign[name], l1)
            nu = od.langevin_normals(seed_in if name == "in" else seed_rec, bi, rl, w.shape[1]) \
                if temperature > 0 else None
            w, m, v = oc.adam_ragged(w, m, v, Gl, rl, lr, b1t, b2t, temperature=temperature, nu=nu)
            out = od.rewire(rl, ind, w, m, v, sign[name], conn[name], w.shape[1], n.N, name == "rec",
                            seed_in if name == "in" else seed_rec, bi)
            st[name] = [out["row_len"], out["ind"], out["w"], out["m"], out["v"]]
            conn[name] = out["conn"]
        W, mW, vW = oc.adam(W, mW, vW, Go, lr, b1t, b2t)
        b, mb, vb = oc.adam(b, mb, vb, Gb, lr, b1t, b2t)
    return st, conn, W, b, rasters, preds


@pytest.mark.parametrize("dtype,temperature", [(F64, 0.0), (F32, 0.0), (F64, 1e-6)])
def test_training_run_tiny_config(dtype, temperature):
    """32 Poisson inputs -> 64 LIF (v_thr 1) -> 4 readouts, 200 steps, 10 trials of batch
    1 with e-prop, L1 1e-5, Adam lr 1e-3 and DEEP R after every trial, without and with
    DEEP R's noise term at temperature 1e-6.  FP64: every raster and the final
    connectivity equal the oracle's exactly; FP32: >= 99.9 % spike agreement and
    identical predictions."""
    from paper_2510_19764_gb300 import abi, net
    T, n_trials, lr, l1 = 200, 10, 1e-3, 1e-5
    s = _setups.classifier(seed=0, dtype=dtype, lif=True, v_thr=1.0, T=T, max_B=1, w_scale=1.5)
    batches = [synth.trial_batch(s.task, 0, i, 1) for i in range(n_trials)]
    g_rasters, g_preds = [], []
    batch = net.DeviceBatch(s.dev, batches[0].labels, batches[0].bin_len, batches[0].trial_ids, T)
    for i, tb in enumerate(batches):
        batch.set_trials(tb.labels, tb.bin_len, tb.trial_ids)
        net.train_batch(s.dev, batch, net.adam_params(lr, i + 1, l1=l1, temperature=temperature), i)
        torch.cuda.synchronize()
        g_rasters.append(net.spikes_from_bits(net.u32_to_numpy(batch.z_rec[0]), s.onet.N).astype(np.float64))
        g_preds.append(int(np.argmax(batch.ysum[0].double().cpu().numpy())))
    assert s.dev.w_in.status() == abi.SNN_OK and s.dev.w_rec.status() == abi.SNN_OK
    st, conn, W, b, rasters, preds = _oracle_train(s, batches, lr, l1, T, temperature)
    total = sum(r.sum() for r in rasters)
    assert total > 100
    if dtype == F64:
        for gr, r in zip(g_rasters, rasters):
            np.testing.assert_array_equal(gr, r)
        for name, d in (("in", s.dev.w_in), ("rec", s.dev.w_rec)):
            h = d.host()
            rl = st[name][0]
            np.testing.assert_array_equal(h["row_len"], rl)
            mask = np.arange(d.C)[None] < rl[:, None]
            np.testing.assert_array_equal(h["ind"][mask], st[name][1][mask])
            np.testing.assert_allclose(h["w"][mask], st[name][2][mask], rtol=1e-9, atol=1e-12)
            np.testing.assert_array_equal(h["conn_bits"], conn[name])
        np.testing.assert_allclose(s.dev.W_out.cpu().numpy(), W, rtol=1e-9, atol=1e-12)
    else:
        agree = np.mean([np.mean(gr == r) for gr, r in zip(g_rasters, rasters)])
        assert agree >= 0.999
    assert abs(np.mean(np.array(g_preds) == np.array([tb.labels[0] for tb in batches]))
               - np.mean(np.array(preds) == np.array([tb.labels[0] for tb in batches]))) <= 0.005 + 1e-12


def test_predrawn_inputs_give_identical_records():
    """snn_draw_inputs (on another stream) + snn_step_neurons_ex(INPUTS_READY) give the
    same records, bit for bit, as snn_step_neurons drawing its own inputs; so does
    SNN_STEP_PACKED_READY after snn_classifier_pack; unknown flag bits are rejected."""
    from paper_2510_19764_gb300 import abi, net
    T, B = 300, 6
    s = _setups.classifier(seed=3, n_in=64, N=128, K=4, lif=False, v_thr=0.6, T=T, max_B=B, spoken=True,
                           n_bins=5, n_classes=4)
    tb = synth.trial_batch(s.task, 3, 0, B)
    ref = net.DeviceBatch(s.dev, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=True)
    abi.snn_step_neurons(s.dev.handle, ref.desc, 0, T)
    got = net.DeviceBatch(s.dev, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=True)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    abi.snn_draw_inputs(s.dev.handle, got.desc, 0, T, side)
    side.synchronize()
    abi.snn_step_neurons_ex(s.dev.handle, got.desc, 0, T, abi.SNN_STEP_INPUTS_READY)
    torch.cuda.synchronize()
    for k in ("x_rec", "z_rec", "psi_rec", "d_rec", "v_rec", "a_rec", "y_rec", "ysum", "v", "a"):
        assert torch.equal(getattr(ref, k), getattr(got, k)), k
    assert int(net.spikes_from_bits(net.u32_to_numpy(got.z_rec), 128).sum()) > 0
    packed = net.DeviceBatch(s.dev, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=True)
    abi.snn_classifier_pack(s.dev.handle)
    abi.snn_draw_inputs(s.dev.handle, packed.desc, 0, T)
    abi.snn_step_neurons_ex(s.dev.handle, packed.desc, 0, T, abi.SNN_STEP_INPUTS_READY | abi.SNN_STEP_PACKED_READY)
    torch.cuda.synchronize()
    for k in ("x_rec", "z_rec", "psi_rec", "d_rec", "v_rec", "a_rec", "y_rec", "ysum", "v", "a"):
        assert torch.equal(getattr(ref, k), getattr(packed, k)), k
    with pytest.raises(abi.SnnError):
        abi.snn_step_neurons_ex(s.dev.handle, got.desc, 0, T, 4)


def test_gradient_of_a_split_batch_is_the_sum_of_its_halves():
    """The classifier's data-parallel split (trials across ranks, then one sum of the
    gradients): the gradient of a batch equals the sum of the gradients of its two
    halves computed separately from the same weights (FP64; only the summation order
    differs)."""
    from paper_2510_19764_gb300 import abi, net
    T, B = 100, 6
    s = _setups.classifier(seed=11, dtype=F64, lif=False, v_thr=0.6, T=T, max_B=B, n_in=50, N=80, K=4,
                           n_classes=3, n_bins=2, spoken=True, p_in=0.2, p_rec=0.15, w_scale=1.5)
    tb = synth.trial_batch(s.task, 0, 0, B)

    def grads(idx):
        batch = net.DeviceBatch(s.dev, tb.labels[idx], tb.bin_len[idx], tb.trial_ids[idx], T)
        abi.snn_step_neurons(s.dev.handle, batch.desc, 0, T)
        abi.snn_eprop_update(s.dev.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
        torch.cuda.synchronize()
        return [t.double().cpu().numpy().copy() for t in (s.dev.w_in.grad, s.dev.w_rec.grad, s.dev.G_out, s.dev.G_b)]

    full = grads(np.arange(B))
    halves = [grads(np.arange(0, B // 2)), grads(np.arange(B // 2, B))]
    for k, (f, a, b) in enumerate(zip(full, *halves)):
        scale = max(np.abs(f).max(), 1e-300)
        assert scale > 0 or k == 3
        np.testing.assert_allclose(a + b, f, rtol=0, atol=1e-12 * scale)
