"""GPU parity of the topographic map: rewiring bit-exact, and each simulation step
(input, conductance LIF, propagation, STDP) against the oracle from the same state."""
import numpy as np
import pytest
import torch

import synth
from oracle import philox as oph
from oracle import topo as ot
from tests._setups import as_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _rewire_args(p, L, name):
    pf, sg = (p.p_form_ff, p.sigma_ff) if name == "ff" else (p.p_form_lat, p.sigma_lat)
    return pf, sg


@pytest.mark.parametrize("L,C,n_att,name", [(16, 16, 60, "ff"), (16, 16, 60, "lat"), (32, 64, 40, "ff"),
                                            (32, 64, 40, "lat"), (8, 6, 500, "ff"), (16, 8, 3000, "lat"),
                                            # many attempts, and a map too large for one CTA's
                                            # shared memory: rows spread over the grid
                                            (16, 8, 5000, "lat"), (64, 16, 6000, "ff"),
                                            (256, 8, 20000, "lat")])
def test_rewire_bit_exact(L, C, n_att, name):
    from paper_2510_19764_gb300 import abi, net
    p = ot.TopoParams(L=L, n_att=n_att)
    pf, sg = _rewire_args(p, L, name)
    rag = synth.topo_initial(4, L, pf, sg, C, p.g_max)
    rng = np.random.default_rng(1)
    g = as_dtype(np.where(rag.ind >= 0, rng.uniform(0, p.g_max, rag.w.shape), 0.0), 0)
    d = net.DeviceRagged(rag.row_len, rag.ind, g, L * L, dtype=0, seed=2024)
    rw = net.topo_rewire(L, pf, sg, n_att, g_max=p.g_max)
    state = (rag.row_len.copy(), rag.ind.copy(), g.copy())
    changes = 0
    for ridx in range(3 if L >= 256 else 10):
        stats = torch.zeros(4, dtype=torch.int64, device="cuda")
        abi.snn_rewire_topo(d.handle, rw, ridx, stats)
        torch.cuda.synchronize()
        out = ot.rewire(*state, C, L * L, L, 2024, ridx, n_att, oph.threshold(p.p_elim_dep),
                        oph.threshold(p.p_elim_pot), float(np.float32(p.g_theta)),
                        ot.form_thresholds(pf, sg, L), float(np.float32(p.g_max)))
        h = d.host()
        np.testing.assert_array_equal(h["row_len"], out["row_len"])
        mask = np.arange(C)[None] < out["row_len"][:, None]
        np.testing.assert_array_equal(h["ind"][mask], out["ind"][mask])
        np.testing.assert_array_equal(h["w"][mask], out["g"][mask])
        st = stats.cpu().numpy()
        assert (st[0], st[1], st[2], st[3]) == (out["removed"], out["formed"], out["overflow"],
                                                int(out["attempts"].sum()))
        changes += out["removed"] + out["formed"]
        state = (out["row_len"], out["ind"], out["g"])
        assert d.status() == abi.SNN_OK
    assert changes > 0


def _device_params(p):
    """The library's parameter structs for an oracle TopoParams."""
    from paper_2510_19764_gb300 import net
    return net.topo_params(L=p.L, L_f=p.L_f, radius=p.radius, t_stim=p.t_stim, dt=p.dt, tau_ref=p.tau_ref,
                           f_base=p.f_base, f_in=p.f_in, sigma_stim=p.sigma_stim)


@pytest.mark.parametrize("setting", ["disc", "paper"])
def test_steps_match_oracle_from_same_state(setting):
    """Each step t of the GPU's granular calls against one oracle.topo.step from the
    GPU's state after step t-1.  disc: the 1 ms workload (disc input, 40/200 Hz); paper:
    Tab. 1-2 as printed (h = 0.1 ms, Gaussian input, 20 ms stimulus interval, rewiring
    every 1 ms).  g_max is the float32 value the device holds, so g_theta = g_max / 2
    and new synapses' weights are the same numbers on both sides."""
    from paper_2510_19764_gb300 import abi, net
    L, C = 16, 32
    N = L * L
    g32 = float(np.float32(0.2))
    if setting == "disc":
        T = 60
        p = ot.TopoParams(L=L, n_att=10, f_base=40.0, f_in=200.0, g_max=g32)
    else:
        T = 300
        p = ot.paper_setting(L, g_max=g32)
    ff = synth.topo_initial(1, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
    lat = synth.topo_initial(2, L, p.p_form_lat, p.sigma_lat, C, p.g_max)
    for r in (ff, lat):
        r.w = as_dtype(r.w, 0)
    dff = net.DeviceRagged(ff.row_len, ff.ind, ff.w, N, dtype=0, seed=11)
    dlat = net.DeviceRagged(lat.row_len, lat.ind, lat.w, N, dtype=0, seed=12)
    tp = _device_params(p)
    rw_ff = net.topo_rewire(L, p.p_form_ff, p.sigma_ff, p.n_att)
    rw_lat = net.topo_rewire(L, p.p_form_lat, p.sigma_lat, p.n_att)
    st = net.DeviceTopoState(N, p.V_rest)
    seeds = {"input": 5, "ff": 11, "lat": 12}
    spikes = flips = rewirings = 0
    for t in range(T):
        cur, prv = t & 1, (t & 1) ^ 1
        # the oracle's state = the GPU's state after step t-1
        hff, hlat = dff.host(), dlat.host()
        o = {k: getattr(st, k).double().cpu().numpy() for k in ("V", "gs", "x_src", "x_tgt", "y")}
        ost = ot.TopoState([hff["row_len"], hff["ind"], hff["w"]], [hlat["row_len"], hlat["ind"], hlat["w"]],
                           o["V"], o["gs"], st.ref.cpu().numpy().astype(np.int64), o["x_src"], o["x_tgt"], o["y"],
                           net.spikes_from_bits(net.u32_to_numpy(st.src_bits[prv]), N).astype(bool),
                           net.spikes_from_bits(net.u32_to_numpy(st.tgt_bits[prv]), N).astype(bool))
        # GPU step t: the granular calls in the order snn_topo_run documents
        abi.snn_topo_input(tp, st.desc, seeds["input"], t)
        abi.snn_propagate(dff.handle, st.src_bits[prv], 1, st.acc)
        abi.snn_propagate(dlat.handle, st.tgt_bits[prv], 1, st.acc)
        abi.snn_topo_neurons(tp, st.desc, t)
        abi.snn_stdp_update(dff.handle, tp, st.src_bits[cur], st.tgt_bits[cur], st.x_src, st.ydec)
        abi.snn_stdp_update(dlat.handle, tp, st.tgt_bits[cur], st.tgt_bits[cur], st.x_tgt, st.ydec)
        rewire = (t + 1) % p.rewire_every == 0
        rst = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
        if rewire:
            ridx = (t + 1) // p.rewire_every - 1
            abi.snn_rewire_topo(dff.handle, rw_ff, ridx, rst[0])
            abi.snn_rewire_topo(dlat.handle, rw_lat, ridx, rst[1])
        torch.cuda.synchronize()
        # oracle step t (input, propagation, neurons, STDP, rewiring) from that state
        out = ot.step(ost, t, p, seeds, C)
        np.testing.assert_array_equal(net.spikes_from_bits(net.u32_to_numpy(st.src_bits[cur]), N).astype(bool),
                                      out["s"])
        zg = net.spikes_from_bits(net.u32_to_numpy(st.tgt_bits[cur]), N).astype(bool)
        differ = zg != out["z"]
        flips += differ.sum()
        spikes += out["z"].sum()
        np.testing.assert_allclose(st.gs.double().cpu().numpy(), ost.gs, rtol=1e-5, atol=1e-6)
        ok = ~differ
        np.testing.assert_allclose(st.V.double().cpu().numpy()[ok], ost.V[ok], rtol=1e-5, atol=1e-4)
        if differ.any():
            continue          # a threshold decided by rounding: STDP and rewiring follow it differently
        np.testing.assert_allclose(st.x_src.double().cpu().numpy(), ost.x_src, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(st.x_tgt.double().cpu().numpy(), ost.x_tgt, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(st.y.double().cpu().numpy(), ost.y, rtol=1e-6, atol=1e-6)
        for dev, proj in ((dff, ost.ff), (dlat, ost.lat)):
            h = dev.host()
            np.testing.assert_array_equal(h["row_len"], proj[0])
            mask = np.arange(C)[None] < proj[0][:, None]
            np.testing.assert_array_equal(h["ind"][mask], proj[1][mask])
            np.testing.assert_allclose(h["w"][mask], proj[2][mask], rtol=0, atol=2e-7)
        if rewire:
            rewirings += 1
            for k, name in enumerate(("ff", "lat")):
                assert rst[k, :3].tolist() == [out[name]["removed"], out[name]["formed"], out[name]["overflow"]]
    assert spikes > 20
    assert flips <= 2
    assert rewirings >= T // p.rewire_every - 2


@pytest.mark.parametrize("L,C,T,n_att,paper", [(16, 32, 40, 10, False), (32, 64, 200, 40, False),
                                               (112, 64, 30, 490, False), (16, 32, 400, 10, True),
                                               (32, 64, 300, 40, True)])
def test_topo_run_matches_granular_calls(L, C, T, n_att, paper):
    """snn_topo_run (the fused cluster loop) equals the same sequence of granular calls,
    bit for bit: connectivity, conductances, neuron state and traces; also in the
    printed setting (h = 0.1 ms, Gaussian input, replicated foci at 32 x 32)."""
    from paper_2510_19764_gb300 import abi, net
    N = L * L
    p = ot.paper_setting(L) if paper else ot.TopoParams(L=L, n_att=n_att)
    res = []
    for mode in ("run", "granular"):
        ff = synth.topo_initial(1, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
        lat = synth.topo_initial(2, L, p.p_form_lat, p.sigma_lat, C, p.g_max)
        dff = net.DeviceRagged(ff.row_len, ff.ind, ff.w, N, dtype=0, seed=11)
        dlat = net.DeviceRagged(lat.row_len, lat.ind, lat.w, N, dtype=0, seed=12)
        tp = _device_params(p)
        rw_ff = net.topo_rewire(L, p.p_form_ff, p.sigma_ff, p.n_att)
        rw_lat = net.topo_rewire(L, p.p_form_lat, p.sigma_lat, p.n_att)
        st = net.DeviceTopoState(N, p.V_rest)
        if mode == "run":
            abi.snn_topo_run(tp, st.desc, dff.handle, dlat.handle, rw_ff, rw_lat, 5, 10, 0, T)
        else:
            for t in range(T):
                cur, prv = t & 1, (t & 1) ^ 1
                abi.snn_topo_input(tp, st.desc, 5, t)
                abi.snn_propagate(dff.handle, st.src_bits[prv], 1, st.acc)
                abi.snn_propagate(dlat.handle, st.tgt_bits[prv], 1, st.acc)
                abi.snn_topo_neurons(tp, st.desc, t)
                abi.snn_stdp_update(dff.handle, tp, st.src_bits[cur], st.tgt_bits[cur], st.x_src, st.ydec)
                abi.snn_stdp_update(dlat.handle, tp, st.tgt_bits[cur], st.tgt_bits[cur], st.x_tgt, st.ydec)
                if (t + 1) % 10 == 0:
                    abi.snn_rewire_topo(dff.handle, rw_ff, (t + 1) // 10 - 1)
                    abi.snn_rewire_topo(dlat.handle, rw_lat, (t + 1) // 10 - 1)
        torch.cuda.synchronize()
        res.append((dff.host(), dlat.host(),
                    {k: getattr(st, k).cpu().numpy().copy()
                     for k in ("V", "gs", "ref", "x_src", "x_tgt", "y", "ydec", "acc", "src_bits", "tgt_bits")}))
    for a, b in zip(res[0][:2], res[1][:2]):
        assert a["row_len"].sum() > 0
        for k in ("row_len", "ind", "w"):
            np.testing.assert_array_equal(a[k], b[k])
    for k in res[0][2]:
        np.testing.assert_array_equal(res[0][2][k], res[1][2][k], err_msg=k)
    assert res[0][2]["tgt_bits"].any() or res[0][2]["y"].max() > 0


@pytest.mark.parametrize("L", [16, 32])
def test_gaussian_input_bit_exact(L):
    """snn_topo_input with Tab. 1's Gaussian profile at h = 0.1 ms (replicated 16 x 16
    foci at 32 x 32) equals the oracle's spikes over several stimulus intervals; a
    profile too wide for the threshold table is rejected."""
    from paper_2510_19764_gb300 import abi, net
    p = ot.paper_setting(L, t_stim=7)
    tp = _device_params(p)
    st = net.DeviceTopoState(p.N, p.V_rest)
    fired = 0
    for t in range(40):
        abi.snn_topo_input(tp, st.desc, 9, t)
        torch.cuda.synchronize()
        got = net.spikes_from_bits(net.u32_to_numpy(st.src_bits[t & 1]), p.N).astype(bool)
        want = ot.input_spikes(9, t, p)
        np.testing.assert_array_equal(got, want)
        fired += want.sum()
    assert fired > 10
    # one 64 x 64 focus tile: squared distances up to 2048 exceed the 1024-entry table;
    # sigma_stim = 2 has decayed to f_base's rounding by then, sigma_stim = 40 has not
    big = net.DeviceTopoState(64 * 64, p.V_rest)
    abi.snn_topo_input(_device_params(ot.paper_setting(64, L_f=None)), big.desc, 9, 0)
    with pytest.raises(abi.SnnError):
        abi.snn_topo_input(_device_params(ot.paper_setting(64, L_f=None, sigma_stim=40.0)), big.desc, 9, 0)
    torch.cuda.synchronize()
