"""Oracle parity over whole runs and at the shapes of the batched and served forms:
a multi-batch training run of a reduced spoken-digit classifier (FP32: spike agreement
and accuracy; FP64: identical rasters and connectivity), one training iteration of a
batched-form instance at its largest shape (hidden 2048, 20 % connectivity, 1000
steps) in the plain and the persistent-kernel paths, and served requests."""
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
    _setups.oracle_pool()                 # spawned before this module's first GPU call
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _arrays(n, st, W, b):
    return (n.n_in, n.N, n.K, st["in"][0], st["in"][1], st["in"][2], st["rec"][0], st["rec"][1], st["rec"][2], W, b)


def _oracle_update(st, sign, conn, W, b, mom, G, i, lr, l1, seeds, N):
    """L1 + Adam on both projections and the readout, then DEEP R (rewire index i)."""
    b1t, b2t = oc.adam_bias(0.9, i + 1), oc.adam_bias(0.999, i + 1)
    post = {}
    for name, Gm in (("in", G[0]), ("rec", G[1])):
        rl, ind, w, m, v = st[name]
        Gl = oc.l1_on_sign(Gm, rl, ind, sign[name], l1)
        w, m, v = oc.adam_ragged(w, m, v, Gl, rl, lr, b1t, b2t)
        post[name] = (w, m, v)
        out = od.rewire(rl, ind, w, m, v, sign[name], conn[name], w.shape[1], N, name == "rec", seeds[name], i)
        st[name] = [out["row_len"], out["ind"], out["w"], out["m"], out["v"]]
        conn[name] = out["conn"]
    W, mom[0], mom[1] = oc.adam(W, mom[0], mom[1], G[2], lr, b1t, b2t)
    b, mom[2], mom[3] = oc.adam(b, mom[2], mom[3], G[3], lr, b1t, b2t)
    return W, b, post


@pytest.mark.parametrize("dtype", [F32, F64])
def test_training_run_reduced_classifier(dtype):
    """700 inputs -> 128 ALIF -> 20 readouts, 10 %, 400 steps, batch 16, 20 batches of
    e-prop + L1 + Adam + DEEP R (320 trials).

    FP64: the oracle trained from the same start on its own (its trials in parallel
    processes, gradients summed in trial order) gives every raster, every prediction and
    the final connectivity exactly.

    FP32: judged batch by batch from the GPU's own state (the oracle takes the GPU's
    weights, moments and connectivity before each batch): >= 99.9 % of all spikes of the
    run agree (each trial simulated by the oracle on its own from the GPU's weights), the
    accuracy over the run is within 0.5 points, each batch's gradient agrees with the
    oracle's from the GPU's records within the gradient tolerance, L1 + Adam from the
    GPU's gradient within FP32 rounding, and DEEP R from the GPU's post-Adam state
    bit-exactly.
    (Adam's first steps divide by |g|, so gradients near its eps would magnify the FP32
    gradient error; the update is compared from the same gradient, as for a single step.)
    (Trained on its own, the FP64 oracle drifts from the FP32 run once a sign test or a
    threshold crossing is decided differently by rounding: in the measured run, all
    spikes agreed for 10 batches, then agreement fell to ~92 %; every step from the same
    state agreed.)"""
    from paper_2510_19764_gb300 import abi, net
    T, B, n_batches, lr, l1 = 400, 16, 20, 1e-3, 1e-5
    s = _setups.classifier(seed=5, n_in=700, N=128, K=20, lif=False, v_thr=0.6, T=T, n_classes=20, n_bins=10,
                           spoken=True, max_B=B, dtype=dtype)
    batches = [synth.trial_batch(s.task, 5, i, B) for i in range(n_batches)]
    batch = net.DeviceBatch(s.dev, batches[0].labels, batches[0].bin_len, batches[0].trial_ids, T)
    n, pool, dev = s.onet, _setups.oracle_pool(), s.dev
    seeds = {"in": dev.w_in.desc.seed, "rec": dev.w_rec.desc.seed}
    st = {"in": [n.in_len.copy(), n.in_ind.copy(), n.w_in.copy(), 0 * n.w_in, 0 * n.w_in],
          "rec": [n.rec_len.copy(), n.rec_ind.copy(), n.w_rec.copy(), 0 * n.w_rec, 0 * n.w_rec]}
    sign, conn = {}, {}
    for name, (rl, ind, w) in (("in", (n.in_len, n.in_ind, n.w_in)), ("rec", (n.rec_len, n.rec_ind, n.w_rec))):
        sign[name], conn[name] = od.init_bitfields(rl, ind, w, n.N, seeds[name])
    W, b = n.W_out.copy(), n.b_out.copy()
    mom = [0 * W, 0 * W, 0 * b, 0 * b]
    agree, total_spikes, g_preds, o_preds, rewired = [], 0, [], [], 0
    for i, tb in enumerate(batches):
        if dtype == F32:            # the oracle starts the batch from the GPU's state
            for name, d in (("in", dev.w_in), ("rec", dev.w_rec)):
                h = d.host()
                st[name] = [h["row_len"], h["ind"], h["w"], h["m"], h["v"]]
                conn[name] = h["conn_bits"]
            W, b = dev.W_out.double().cpu().numpy(), dev.b_out.double().cpu().numpy()
            mom = [t.double().cpu().numpy() for t in (dev.W_out_m, dev.W_out_v, dev.b_m, dev.b_v)]
        batch.set_trials(tb.labels, tb.bin_len, tb.trial_ids)
        abi.snn_step_neurons(dev.handle, batch.desc, 0, T)
        abi.snn_eprop_update(dev.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
        abi.snn_eprop_update(dev.handle, batch.desc, abi.SNN_EPROP_APPLY, net.adam_params(lr, i + 1, l1=l1))
        torch.cuda.synchronize()
        g_post = {name: d.host() for name, d in (("in", dev.w_in), ("rec", dev.w_rec))}
        stats = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
        abi.snn_rewire_deepr(dev.w_in.handle, i, stats[0])
        abi.snn_rewire_deepr(dev.w_rec.handle, i, stats[1])
        torch.cuda.synchronize()
        rewired += int(stats[:, 0].sum())
        z = net.spikes_from_bits(net.u32_to_numpy(batch.z_rec), 128).astype(np.uint8)
        g_preds += list(np.argmax(batch.ysum.double().cpu().numpy(), axis=1))
        arrays = _arrays(n, st, W, b)
        if dtype == F32:
            # the oracle's gradient from the GPU's own records (a trial whose raster a
            # rounding flip sent elsewhere would otherwise compare different spikes)
            x = net.spikes_from_bits(net.u32_to_numpy(batch.x_rec), 700).astype(np.float64)
            psi, dd = batch.psi_rec.double().cpu().numpy(), batch.d_rec.double().cpu().numpy()
            g_jobs = [(arrays, n.neuron, x[k], z[k].astype(np.float64), psi[k], dd[k]) for k in range(B)]
            G_rec = [0, 0, 0, 0]
            for g in pool.map(_setups.oracle_grad_from_records, g_jobs):
                G_rec = [a + c for a, c in zip(G_rec, g)]
        jobs = [(arrays, n.neuron, s.task.thr, tb.labels[k], tb.bin_len[k], tb.trial_ids[k], s.in_seed, T)
                for k in range(B)]
        G = [0, 0, 0, 0]
        for k, (zo, pred, _, g) in enumerate(pool.map(_setups.oracle_trial, jobs)):
            o_preds.append(pred)
            G = [a + c for a, c in zip(G, g)]
            total_spikes += int(zo.sum())
            if dtype == F64:
                np.testing.assert_array_equal(z[k], zo, err_msg=f"batch {i} trial {k}")
            agree.append((z[k] == zo).ravel())
        pre_w = {name: [a.copy() for a in st[name]] for name in ("in", "rec")}
        W, b, post = _oracle_update(st, sign, conn, W, b, mom, G, i, lr, l1, seeds, n.N)
        for k_, (name, d) in enumerate((("in", dev.w_in), ("rec", dev.w_rec))):
            live = np.arange(d.C)[None] < g_post[name]["row_len"][:, None]
            if dtype == F32:
                # the batch's gradient (summed over its trials) against the oracle's from the
                # same records.  Each entry sums ~10^2 adjoint values of either sign, each
                # carrying up to T x 2^-24 relative FP32 error from the reverse-time scan; an
                # entry that cancels keeps the absolute error of its terms, hence the
                # absolute term (of the largest entry, whose terms rarely cancel)
                Gg, Go = g_post[name]["grad"][live], G_rec[k_][live]
                gmax = np.abs(Go).max()
                bound = 2e-5 * np.maximum(np.abs(Go), 1e-3 * gmax) + 5e-6 * gmax
                worst = int(np.argmax(np.abs(Gg - Go) / bound))
                assert np.all(np.abs(Gg - Go) <= bound), (i, name, Gg[worst], Go[worst], gmax)
                # L1 + Adam from the GPU's own gradient: FP32 rounding of the FP64 update
                rl, ind, w0, m0, v0 = pre_w[name]
                Gl = oc.l1_on_sign(g_post[name]["grad"], rl, ind, sign[name], l1)
                w1, _, _ = oc.adam_ragged(w0, m0, v0, Gl, rl, lr, oc.adam_bias(0.9, i + 1), oc.adam_bias(0.999, i + 1))
                np.testing.assert_allclose(g_post[name]["w"][live], w1[live], rtol=1e-6, atol=1e-7)
                # DEEP R from the GPU's own post-Adam state: bit-exact
                h = g_post[name]
                out = od.rewire(h["row_len"], h["ind"], h["w"], h["m"], h["v"], h["sign_bits"], h["conn_bits"], d.C,
                                n.N, name == "rec", seeds[name], i)
                got = d.host()
                np.testing.assert_array_equal(got["row_len"], out["row_len"])
                live2 = np.arange(d.C)[None] < out["row_len"][:, None]
                np.testing.assert_array_equal(got["ind"][live2], out["ind"][live2])
                np.testing.assert_array_equal(got["w"][live2], out["w"][live2])
                np.testing.assert_array_equal(got["conn_bits"], out["conn"])
    assert dev.w_in.status() == abi.SNN_OK and dev.w_rec.status() == abi.SNN_OK
    assert total_spikes > 1000 and rewired > 0
    labels = np.concatenate([tb.labels for tb in batches])
    acc_g = np.mean(np.array(g_preds) == labels)
    acc_o = np.mean(np.array(o_preds) == labels)
    frac = float(np.mean(np.concatenate(agree)))
    assert frac >= 0.999, frac
    assert abs(acc_g - acc_o) <= 0.005 + 1e-12, (acc_g, acc_o)
    if dtype == F64:
        assert g_preds == o_preds
        for name, d in (("in", dev.w_in), ("rec", dev.w_rec)):
            h = d.host()
            rl = st[name][0]
            np.testing.assert_array_equal(h["row_len"], rl)
            mask = np.arange(d.C)[None] < rl[:, None]
            np.testing.assert_array_equal(h["ind"][mask], st[name][1][mask])
            np.testing.assert_allclose(h["w"][mask], st[name][2][mask], rtol=1e-9, atol=1e-12)
            np.testing.assert_array_equal(h["conn_bits"], conn[name])


def test_batched_instance_at_largest_shape():
    """One training iteration of a batched-form instance with hidden 2048, 20 %
    connectivity and 1000 steps (the largest of the batched workload): records of
    sampled steps from the kernel's own state (FP32 1e-5), sampled synapses' gradients
    against the oracle's trace form, L1 + Adam, and DEEP R on both projections bit-exact
    against the oracle from the post-Adam state; the persistent kernel then gives the
    same records, weights and connectivity as these per-call steps, bit for bit."""
    from paper_2510_19764_gb300 import abi, net, sched
    N, T, p = 2048, 1000, 0.2
    task = synth.spoken_digit_task(3, n_in=sched.N_IN, n_classes=sched.N_CLASSES, T=1000, n_bins=sched.N_BINS)
    spec = sched.InstanceSpec(N, T, p, 4)
    a = sched.Instance(spec, task)
    bt = net.DeviceBatch(a.cls, [0], [int(a.bin_table[0])], [0], T, record_state=True)
    h0 = {"in": a.d_in.host(), "rec": a.d_rec.host()}
    W0, b0 = a.cls.W_out.double().cpu().numpy(), a.cls.b_out.double().cpu().numpy()
    abi.snn_step_neurons(a.cls.handle, bt.desc, 0, T)
    abi.snn_eprop_update(a.cls.handle, bt.desc, abi.SNN_EPROP_GRAD, None)
    torch.cuda.synchronize()
    onet = oc.ClassifierNet(sched.N_IN, N, sched.K_OUT, h0["in"]["row_len"], h0["in"]["ind"], h0["in"]["w"],
                            h0["rec"]["row_len"], h0["rec"]["ind"], h0["rec"]["w"], W0, b0, oc.NeuronParams())
    label, bin_len, seed = 0, int(a.bin_table[0]), a.cls.desc.in_seed
    z = net.spikes_from_bits(net.u32_to_numpy(bt.z_rec[0]), N).astype(np.float64)
    x = net.spikes_from_bits(net.u32_to_numpy(bt.x_rec[0]), sched.N_IN).astype(np.float64)
    assert z.mean() > 1e-3
    rng = np.random.default_rng(7)
    for t in rng.integers(1, T, 6):
        t = int(t)
        stt = {"v": bt.v_rec[0, t - 1].double().cpu().numpy(), "a": bt.a_rec[0, t - 1].double().cpu().numpy(),
               "z": z[t - 1], "x": x[t - 1], "y": bt.y_rec[0, t - 1].double().cpu().numpy()}
        r = oc.forward_trial(onet, task.thr, label, bin_len, 0, seed, 1, state=stt, t0=t)
        np.testing.assert_array_equal(x[t], r["x"][0])
        for key, ref in (("v_rec", r["v"][0]), ("a_rec", r["a"][0]), ("psi_rec", r["psi"][0]), ("y_rec", r["y"][0]),
                         ("d_rec", r["d"][0])):
            np.testing.assert_allclose(getattr(bt, key)[0, t].double().cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
        A = 0.6 + 0.0174 * r["a"][0]
        assert np.all(np.abs(r["v"][0] - A)[z[t] != r["z"][0]] < 1e-5)
    d = bt.d_rec[0].double()
    Wd = a.cls.W_out.double()
    for proj, h, grad, bits in (("in", h0["in"], a.d_in.grad, x), ("rec", h0["rec"], a.d_rec.grad, z)):
        G = grad.double().cpu().numpy()
        live = np.arange(G.shape[1])[None] < h["row_len"][:, None]
        for _ in range(8):
            i = int(rng.integers(0, len(h["row_len"])))
            while h["row_len"][i] == 0:
                i = int(rng.integers(0, len(h["row_len"])))
            s = int(rng.integers(0, h["row_len"][i]))
            j = int(h["ind"][i, s])
            ref = oc.eprop_synapse(bits[None, :, i], bt.psi_rec[0, :, j].double().cpu().numpy()[None],
                                   (d @ Wd[:, j]).cpu().numpy()[None], onet.neuron)
            scale = max(abs(ref), 1e-3 * np.abs(G[live]).max())
            assert abs(G[i, s] - ref) <= 2e-5 * scale, (proj, i, s, G[i, s], ref)
    pre = {"in": a.d_in.host(), "rec": a.d_rec.host()}
    abi.snn_eprop_update(a.cls.handle, bt.desc, abi.SNN_EPROP_APPLY, net.adam_params(a.lr, 1, l1=a.l1))
    torch.cuda.synchronize()
    post = {"in": a.d_in.host(), "rec": a.d_rec.host()}
    for name in ("in", "rec"):
        h = pre[name]
        Gl = oc.l1_on_sign(h["grad"], h["row_len"], h["ind"], h["sign_bits"], a.l1)
        w, m, v = oc.adam_ragged(h["w"], h["m"], h["v"], Gl, h["row_len"], a.lr, oc.adam_bias(0.9, 1),
                                 oc.adam_bias(0.999, 1))
        live = np.arange(w.shape[1])[None] < h["row_len"][:, None]
        np.testing.assert_allclose(post[name]["w"][live], w[live], rtol=1e-6, atol=1e-7)
    stats = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
    abi.snn_rewire_deepr(a.d_in.handle, 0, stats[0])
    abi.snn_rewire_deepr(a.d_rec.handle, 0, stats[1])
    torch.cuda.synchronize()
    for k, (name, d_, no_aut) in enumerate((("in", a.d_in, False), ("rec", a.d_rec, True))):
        h = post[name]
        out = od.rewire(h["row_len"], h["ind"], h["w"], h["m"], h["v"], h["sign_bits"], h["conn_bits"], d_.C, N,
                        no_aut, d_.desc.seed, 0)
        got = d_.host()
        np.testing.assert_array_equal(got["row_len"], out["row_len"])
        live = np.arange(d_.C)[None] < out["row_len"][:, None]
        for key in ("ind", "w", "m", "v"):
            np.testing.assert_array_equal(got[key][live], out[key][live])
        np.testing.assert_array_equal(got["conn_bits"], out["conn"])
        assert int(stats[k, 0]) == out["removed"] and int(stats[k, 1]) == out["formed"]
    assert int(stats[:, 0].sum()) > 0
    # the same iteration in the persistent kernel
    b = sched.Instance(spec, task)
    mr = sched.MultiRunner([b])
    mr.iterate()
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_OK and int(b.step.item()) == 1
    for key in ("x_rec", "z_rec", "psi_rec", "d_rec", "ysum"):
        assert torch.equal(getattr(bt, key), getattr(b.batch, key)), key
    for da, db in ((a.d_in, b.d_in), (a.d_rec, b.d_rec)):
        assert torch.equal(da.row_len, db.row_len) and torch.equal(da.conn_bits, db.conn_bits)
        live = torch.arange(da.C, device="cuda")[None] < da.row_len[:, None]
        for key in ("ind", "w", "m", "v"):
            assert torch.equal(getattr(da, key)[live], getattr(db, key)[live]), key
    assert torch.equal(a.cls.W_out, b.cls.W_out) and torch.equal(a.cls.b_out, b.cls.b_out)


def test_served_requests_match_the_oracle():
    """Inference and fine-tuning requests through the serving loop: each result (sum of
    the readout over the request's steps, from the model's resident weights) equals the
    oracle's forward of the same request within 1e-5."""
    from paper_2510_19764_gb300 import serve
    task = synth.spoken_digit_task(1, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX,
                                   n_bins=serve.N_BINS)
    model = serve.Model(0, 256, task, max_batch=8)
    eng = serve.Engine([model], max_batch=8, slots_per_model=2, n_streams=4)
    reqs = [serve.Request(i, 0, lab, T, max(1, round(w * T / serve.N_BINS)), ft)
            for i, (lab, T, w, ft) in enumerate([(3, 120, 1.0, False), (7, 250, 0.9, False), (11, 180, 1.1, True),
                                                 (0, 300, 1.2, False), (19, 150, 0.8, True)])]
    res = {r.rid: r for r in eng.run(reqs, realtime=False)}
    onet = oc.ClassifierNet(serve.N_IN, 256, serve.K_OUT, model.host_in.row_len, model.host_in.ind,
                            np.float32(model.host_in.w).astype(np.float64), model.host_rec.row_len, model.host_rec.ind,
                            np.float32(model.host_rec.w).astype(np.float64),
                            np.float32(model.W_out).astype(np.float64), np.float32(model.b).astype(np.float64),
                            oc.NeuronParams())
    for q in reqs:
        r = oc.forward_trial(onet, task.thr, q.label, q.bin_len, q.rid, model.in_seed, q.T)
        np.testing.assert_allclose(res[q.rid].ysum, r["ysum"], rtol=1e-5, atol=1e-5 * np.abs(r["ysum"]).max())
        assert res[q.rid].finetune == q.finetune
