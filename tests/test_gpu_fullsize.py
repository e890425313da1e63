"""Full-size parity in the benchmark's launch configuration (512 trials x 1000 steps,
700 inputs -> 1024 ALIF -> 20 readouts, 10 % ragged connectivity, capacity 288), on
outputs the oracle can compute one by one, plus the 32 x 32 topographic map after
thousands of steps."""
import numpy as np
import pytest
import torch

import synth
from oracle import classifier as oc
from oracle import deepr as od
from oracle import philox as oph
from oracle import topo as ot

pytestmark = pytest.mark.gpu

B, T, N_IN, N, K = 512, 1000, 700, 1024, 20


@pytest.fixture(scope="module")
def full():
    from paper_2510_19764_gb300 import abi, build, net
    build.build()
    abi.load()
    seed = 0
    task = synth.spoken_digit_task(seed, n_in=N_IN, n_classes=20, T=T, n_bins=10)
    in_rag = synth.random_ragged(seed + 1, N_IN, N, 0.1)
    rec_rag = synth.random_ragged(seed + 2, N, N, 0.1, no_autapse=True)
    for r in (in_rag, rec_rag):
        r.w = r.w.astype(np.float32).astype(np.float64)
    W_out, b = synth.dense_readout(seed + 3, K, N)
    W_out = W_out.astype(np.float32).astype(np.float64)
    d_in = net.DeviceRagged(in_rag.row_len, in_rag.ind, in_rag.w, N, adam=True, grad=True, deepr=True, seed=100)
    d_rec = net.DeviceRagged(rec_rag.row_len, rec_rag.ind, rec_rag.w, N, no_autapse=True, adam=True, grad=True,
                             deepr=True, seed=101)
    ncfg = net.NeuronCfg(tau_m=20.0, v_thr=0.6, beta=0.0174, tau_a=2000.0)
    cls = net.DeviceClassifier(N_IN, N, K, d_in, d_rec, W_out, b, task.thr, 7, ncfg, max_B=B, max_T=T)
    tb = synth.trial_batch(task, seed, 0, B)
    batch = net.DeviceBatch(cls, tb.labels, tb.bin_len, tb.trial_ids, T, record_state=True)
    abi.snn_step_neurons(cls.handle, batch.desc, 0, T)
    abi.snn_eprop_update(cls.handle, batch.desc, abi.SNN_EPROP_GRAD, None)
    torch.cuda.synchronize()
    onet = oc.ClassifierNet(N_IN, N, K, in_rag.row_len, in_rag.ind, in_rag.w, rec_rag.row_len, rec_rag.ind,
                            rec_rag.w, W_out, b, oc.NeuronParams(tau_m=20.0, v_thr=0.6, beta=0.0174, tau_a=2000.0))
    return {"task": task, "in": in_rag, "rec": rec_rag, "cls": cls, "batch": batch, "tb": tb, "onet": onet,
            "net": net, "abi": abi}


def test_input_spikes_sampled_bit_exact(full):
    net, bt, tb = full["net"], full["batch"], full["tb"]
    rng = np.random.default_rng(0)
    for b, t in zip(rng.integers(0, B, 12), rng.integers(0, T, 12)):
        got = net.spikes_from_bits(net.u32_to_numpy(bt.x_rec[b, t]), N_IN).astype(bool)
        ref = oc.poisson_input(full["task"].thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], int(t), 7)
        np.testing.assert_array_equal(got, ref)


def test_forward_steps_sampled(full):
    """From the kernel's own state at t-1, one oracle step reproduces step t."""
    net, bt, tb, onet = full["net"], full["batch"], full["tb"], full["onet"]
    rng = np.random.default_rng(1)
    spikes = 0
    for b, t in zip(rng.integers(0, B, 8), rng.integers(1, T, 8)):
        b, t = int(b), int(t)
        zb = net.spikes_from_bits(net.u32_to_numpy(bt.z_rec[b]), N).astype(np.float64)
        xb = net.spikes_from_bits(net.u32_to_numpy(bt.x_rec[b]), N_IN).astype(np.float64)
        st = {"v": bt.v_rec[b, t - 1].double().cpu().numpy(), "a": bt.a_rec[b, t - 1].double().cpu().numpy(),
              "z": zb[t - 1], "x": xb[t - 1], "y": bt.y_rec[b, t - 1].double().cpu().numpy()}
        r = oc.forward_trial(onet, full["task"].thr, tb.labels[b], tb.bin_len[b], tb.trial_ids[b], 7, 1, state=st,
                             t0=t)
        for k, ref in (("v", r["v"][0]), ("a", r["a"][0]), ("psi", r["psi"][0])):
            got = getattr(bt, {"v": "v_rec", "a": "a_rec", "psi": "psi_rec"}[k])[b, t].double().cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(bt.y_rec[b, t].double().cpu().numpy(), r["y"][0], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(bt.d_rec[b, t].double().cpu().numpy(), r["d"][0], rtol=1e-5, atol=1e-6)
        A = 0.6 + 0.0174 * r["a"][0]
        differ = zb[t] != r["z"][0]
        assert np.all(np.abs(r["v"][0] - A)[differ] < 1e-5)
        spikes += zb[t].sum()
    assert spikes > 0


def test_gradient_sampled_synapses_over_all_trials(full):
    """G of sampled synapses, summed over all 512 trials, against the oracle's trace
    recursion for that synapse (vectorised over trials) from the same records."""
    net, bt, cls, onet = full["net"], full["batch"], full["cls"], full["onet"]
    p = onet.neuron
    d = bt.d_rec.double()                                            # [B, T, K]
    W = cls.W_out.double()
    rng = np.random.default_rng(2)
    for proj, rag, grad, bits, n_pre in (("in", full["in"], cls.w_in.grad, bt.x_rec, N_IN),
                                        ("rec", full["rec"], cls.w_rec.grad, bt.z_rec, N)):
        G = grad.double().cpu().numpy()
        for _ in range(6):
            i = int(rng.integers(0, n_pre))
            while rag.row_len[i] == 0:
                i = int(rng.integers(0, n_pre))
            s = int(rng.integers(0, rag.row_len[i]))
            j = int(rag.ind[i, s])
            words = bits[:, :, i >> 5].cpu().numpy().view(np.uint32)
            pre = ((words >> np.uint32(i & 31)) & 1).astype(np.float64)       # [B, T]
            psi_j = bt.psi_rec[:, :, j].double().cpu().numpy()
            L_j = (d @ W[:, j]).cpu().numpy()                              # [B, T]
            ref = oc.eprop_synapse(pre, psi_j, L_j, p)
            scale = max(abs(ref), 1e-3 * np.abs(G[:rag.P]).max())
            assert abs(G[i, s] - ref) <= 2e-5 * scale + 1e-6 * np.abs(G).max(), (proj, i, s, G[i, s], ref)


def test_adam_and_deepr_full_size_bit_exact(full):
    """L1 + Adam on the full gradient, then DEEP R on both 700/1024 x 1024 projections:
    row lengths, targets, moved weights/moments and connectivity identical to the
    oracle run on the same post-Adam state."""
    net, abi, cls = full["net"], full["abi"], full["cls"]
    pre = {name: d.host() for name, d in (("in", cls.w_in), ("rec", cls.w_rec))}
    abi.snn_eprop_update(cls.handle, None, abi.SNN_EPROP_APPLY, net.adam_params(1e-3, 1, l1=1e-5))
    torch.cuda.synchronize()
    for name, d, no_aut, seed in (("in", cls.w_in, False, 100), ("rec", cls.w_rec, True, 101)):
        h0 = pre[name]
        h = d.host()
        Gl = oc.l1_on_sign(h0["grad"], h0["row_len"], h0["ind"], h0["sign_bits"], 1e-5)
        w, m, v = oc.adam_ragged(h0["w"], h0["m"], h0["v"], Gl, h0["row_len"], 1e-3, 0.9, 0.999)
        mask = np.arange(d.C)[None] < h0["row_len"][:, None]
        np.testing.assert_allclose(h["w"][mask], w[mask], rtol=1e-6, atol=1e-7)
        # DEEP R from the device's post-Adam state
        stats = torch.zeros(4, dtype=torch.int64, device="cuda")
        abi.snn_rewire_deepr(d.handle, 0, stats)
        torch.cuda.synchronize()
        out = od.rewire(h["row_len"], h["ind"], h["w"], h["m"], h["v"], h["sign_bits"], h["conn_bits"], d.C, N,
                        no_aut, seed, 0)
        h2 = d.host()
        np.testing.assert_array_equal(h2["row_len"], out["row_len"])
        mk = np.arange(d.C)[None] < out["row_len"][:, None]
        np.testing.assert_array_equal(h2["ind"][mk], out["ind"][mk])
        for k in ("w", "m", "v"):
            np.testing.assert_array_equal(h2[k][mk], out[k][mk])
        np.testing.assert_array_equal(h2["conn_bits"], out["conn"])
        st = stats.cpu().numpy()
        assert (st[0], st[1], st[2]) == (out["removed"], out["formed"], out["overflow"])


def test_row_schedules_give_identical_results(full):
    """The forward's row schedule (4, 8 or 16 warps per trial) changes nothing but speed."""
    net, abi, cls, tb = full["net"], full["abi"], full["cls"], full["tb"]
    outs = []
    for warps in (8, 16, 4):
        abi.snn_classifier_set_schedule(cls.handle, warps)
        bt = net.DeviceBatch(cls, tb.labels[:64], tb.bin_len[:64], tb.trial_ids[:64], T, workspace=False)
        abi.snn_step_neurons(cls.handle, bt.desc, 0, T)
        torch.cuda.synchronize()
        outs.append((bt.z_rec.cpu().numpy(), bt.psi_rec.cpu().numpy(), bt.ysum.cpu().numpy()))
    abi.snn_classifier_set_schedule(cls.handle, 8)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def test_topographic_map_after_thousands_of_steps():
    """32 x 32 sheets, C = 64, 40 attempts every 10 steps: run 3000 steps, then check
    one more step (propagation, neurons, STDP) and one rewiring against the oracle from
    the device state."""
    from paper_2510_19764_gb300 import abi, build, net
    build.build()
    L, C = 32, 64
    Np = L * L
    p = ot.TopoParams(L=L, n_att=40)
    ff = synth.topo_initial(1, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
    lat = synth.topo_initial(2, L, p.p_form_lat, p.sigma_lat, C, p.g_max)
    dff = net.DeviceRagged(ff.row_len, ff.ind, ff.w, Np, seed=11)
    dlat = net.DeviceRagged(lat.row_len, lat.ind, lat.w, Np, seed=12)
    tp = net.topo_params(L=L)
    rw_ff = net.topo_rewire(L, p.p_form_ff, p.sigma_ff, 40)
    rw_lat = net.topo_rewire(L, p.p_form_lat, p.sigma_lat, 40)
    st = net.DeviceTopoState(Np, p.V_rest)
    t0 = 3000
    abi.snn_topo_run(tp, st.desc, dff.handle, dlat.handle, rw_ff, rw_lat, 5, 10, 0, t0)
    torch.cuda.synchronize()
    cur, prv = t0 & 1, (t0 & 1) ^ 1
    o = {k: getattr(st, k).double().cpu().numpy() for k in ("V", "gs", "x_src", "x_tgt", "y")}
    o["ref"] = st.ref.cpu().numpy().astype(np.int64)
    s_prev = net.spikes_from_bits(net.u32_to_numpy(st.src_bits[prv]), Np).astype(bool)
    z_prev = net.spikes_from_bits(net.u32_to_numpy(st.tgt_bits[prv]), Np).astype(bool)
    hff, hlat = dff.host(), dlat.host()
    assert hff["row_len"].sum() != ff.row_len.sum() or hlat["row_len"].sum() != lat.row_len.sum()
    abi.snn_topo_input(tp, st.desc, 5, t0)
    abi.snn_propagate(dff.handle, st.src_bits[prv], 1, st.acc)
    abi.snn_propagate(dlat.handle, st.tgt_bits[prv], 1, st.acc)
    abi.snn_topo_neurons(tp, st.desc, t0)
    abi.snn_stdp_update(dff.handle, tp, st.src_bits[cur], st.tgt_bits[cur], st.x_src, st.ydec)
    abi.snn_stdp_update(dlat.handle, tp, st.tgt_bits[cur], st.tgt_bits[cur], st.x_tgt, st.ydec)
    torch.cuda.synchronize()
    s = ot.input_spikes(5, t0, p)
    np.testing.assert_array_equal(net.spikes_from_bits(net.u32_to_numpy(st.src_bits[cur]), Np).astype(bool), s)
    I = ot.propagate_rows((hff["row_len"], hff["ind"], hff["w"]), s_prev, Np)
    I += ot.propagate_rows((hlat["row_len"], hlat["ind"], hlat["w"]), z_prev, Np)
    V, gs, ref, z = ot.neuron_step(o["V"], o["gs"], o["ref"], I, p)
    np.testing.assert_allclose(st.gs.double().cpu().numpy(), gs, rtol=1e-5, atol=1e-6)
    zg = net.spikes_from_bits(net.u32_to_numpy(st.tgt_bits[cur]), Np).astype(bool)
    assert (zg != z).sum() <= 1
    pff = [hff["row_len"], hff["ind"], hff["w"].copy()]
    plat = [hlat["row_len"], hlat["ind"], hlat["w"].copy()]
    ot.stdp_step([tuple(pff), tuple(plat)], [o["x_src"], o["x_tgt"]], o["y"], [s, zg], zg, p)
    for dev, ref_p in ((dff, pff), (dlat, plat)):
        mask = np.arange(C)[None] < ref_p[0][:, None]
        np.testing.assert_allclose(dev.w.double().cpu().numpy()[mask], ref_p[2][mask], rtol=0, atol=2e-7)
    ridx = (t0 + 10) // 10 - 1
    for dev, rw, pf, sg, seed in ((dff, rw_ff, p.p_form_ff, p.sigma_ff, 11),
                                  (dlat, rw_lat, p.p_form_lat, p.sigma_lat, 12)):
        h = dev.host()
        abi.snn_rewire_topo(dev.handle, rw, ridx)
        torch.cuda.synchronize()
        out = ot.rewire(h["row_len"], h["ind"], h["w"], C, Np, L, seed, ridx, 40, oph.threshold(p.p_elim_dep),
                        oph.threshold(p.p_elim_pot), float(np.float32(p.g_theta)), ot.form_thresholds(pf, sg, L),
                        float(np.float32(p.g_max)))
        h2 = dev.host()
        np.testing.assert_array_equal(h2["row_len"], out["row_len"])
        mask = np.arange(C)[None] < out["row_len"][:, None]
        np.testing.assert_array_equal(h2["ind"][mask], out["ind"][mask])
        np.testing.assert_array_equal(h2["w"][mask], out["g"][mask])
