"""GPU parity of the connectivity-evolution analysis of the topographic map (Sec. 3.2,
Figs. 8-9): elimination / formation histograms by squared distance recorded by the
rewiring (granular and fused paths), and the displacement / in-degree profile."""
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


@pytest.mark.parametrize("L,C,n_att,name", [(16, 16, 300, "ff"), (32, 64, 400, "lat"), (8, 6, 500, "ff")])
def test_rewire_event_histograms_match_oracle(L, C, n_att, name):
    from paper_2510_19764_gb300 import abi, net
    p = ot.TopoParams(L=L, n_att=n_att)
    pf, sg = (p.p_form_ff, p.sigma_ff) if name == "ff" else (p.p_form_lat, p.sigma_lat)
    rag = synth.topo_initial(7, L, pf, sg, C, p.g_max)
    rng = np.random.default_rng(2)
    g = as_dtype(np.where(rag.ind >= 0, rng.uniform(0, p.g_max, rag.w.shape), 0.0), 0)
    d = net.DeviceRagged(rag.row_len, rag.ind, g, L * L, dtype=0, seed=77)
    rw = net.topo_rewire(L, pf, sg, n_att, g_max=p.g_max)
    elim, form = net.attach_event_histograms(rw, L)
    state = (rag.row_len.copy(), rag.ind.copy(), g.copy())
    want_e = np.zeros(elim.numel(), np.int64)
    want_f = np.zeros(form.numel(), np.int64)
    for ridx in range(8):
        abi.snn_rewire_topo(d.handle, rw, ridx)
        out = ot.rewire(*state, C, L * L, L, 77, ridx, n_att, oph.threshold(p.p_elim_dep),
                        oph.threshold(p.p_elim_pot), float(np.float32(p.g_theta)),
                        ot.form_thresholds(pf, sg, L), float(np.float32(p.g_max)))
        want_e += ot.d2_histogram(out["removed_d2"], L)
        want_f += ot.d2_histogram(out["formed_d2"], L)
        state = (out["row_len"], out["ind"], out["g"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(elim.cpu().numpy(), want_e)
        np.testing.assert_array_equal(form.cpu().numpy(), want_f)
    assert want_e.sum() > 0 and want_f.sum() > 0
    # the histograms are only added to: zeroing them between time bins is the caller's
    elim.zero_()
    abi.snn_rewire_topo(d.handle, rw, 8)
    out = ot.rewire(*state, C, L * L, L, 77, 8, n_att, oph.threshold(p.p_elim_dep), oph.threshold(p.p_elim_pot),
                    float(np.float32(p.g_theta)), ot.form_thresholds(pf, sg, L), float(np.float32(p.g_max)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(elim.cpu().numpy(), ot.d2_histogram(out["removed_d2"], L))
    assert d.status() == abi.SNN_OK


@pytest.mark.parametrize("L,C,T,n_att", [(16, 32, 100, 40), (32, 64, 400, 40), (112, 64, 40, 490)])
def test_fused_run_records_the_same_events_as_granular_calls(L, C, T, n_att):
    """snn_topo_run (one cluster launch) fills the histograms exactly as the per-step
    calls do, and the connectivity profile of the final state matches the oracle's."""
    from paper_2510_19764_gb300 import abi, net
    N = L * L
    p = ot.TopoParams(L=L, n_att=n_att)
    res = []
    for mode in ("run", "granular"):
        ff = synth.topo_initial(1, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
        lat = synth.topo_initial(2, L, p.p_form_lat, p.sigma_lat, C, p.g_max)
        dff = net.DeviceRagged(ff.row_len, ff.ind, ff.w, N, dtype=0, seed=11)
        dlat = net.DeviceRagged(lat.row_len, lat.ind, lat.w, N, dtype=0, seed=12)
        tp = net.topo_params(L=L)
        rw_ff = net.topo_rewire(L, p.p_form_ff, p.sigma_ff, p.n_att)
        rw_lat = net.topo_rewire(L, p.p_form_lat, p.sigma_lat, p.n_att)
        h_ff = net.attach_event_histograms(rw_ff, L)
        h_lat = net.attach_event_histograms(rw_lat, L)
        st = net.DeviceTopoState(N, p.V_rest)
        stats = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
        if mode == "run":
            abi.snn_topo_run(tp, st.desc, dff.handle, dlat.handle, rw_ff, rw_lat, 5, 10, 0, T, stats[0], stats[1])
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
                    abi.snn_rewire_topo(dff.handle, rw_ff, (t + 1) // 10 - 1, stats[0])
                    abi.snn_rewire_topo(dlat.handle, rw_lat, (t + 1) // 10 - 1, stats[1])
        torch.cuda.synchronize()
        hist = [h.cpu().numpy() for h in h_ff + h_lat]
        st_h = stats.cpu().numpy()
        # every recorded event is one of the counted ones
        assert hist[0].sum() == st_h[0, 0] and hist[1].sum() == st_h[0, 1]
        assert hist[2].sum() == st_h[1, 0] and hist[3].sum() == st_h[1, 1]
        prof = [tuple(x.cpu().numpy() for x in net.topo_connectivity(r, L)) for r in (dff, dlat)]
        res.append((hist, prof, dff.host(), dlat.host()))
    for a, b in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, b)
    assert sum(h.sum() for h in res[0][0]) > 0
    for (count, wsum, indeg), host in zip(res[0][1], res[0][2:]):
        oc, ow, oi = ot.connectivity_profile(host["row_len"], host["ind"], host["w"], L)
        np.testing.assert_array_equal(count, oc)
        np.testing.assert_array_equal(indeg, oi)
        # float32 weights summed in double by atomics: order-dependent rounding only
        np.testing.assert_allclose(wsum, ow, rtol=1e-12, atol=1e-15)


def test_connectivity_profile_large_and_edge_cases():
    """A 112 x 112 map (many CTAs), an empty matrix, the no-output call, and the
    argument checks."""
    from paper_2510_19764_gb300 import abi, net
    L, C = 112, 64
    p = ot.TopoParams(L=L)
    rag = synth.topo_initial(5, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
    rng = np.random.default_rng(4)
    g = as_dtype(np.where(rag.ind >= 0, rng.uniform(0, p.g_max, rag.w.shape), 0.0), 0)
    d = net.DeviceRagged(rag.row_len, rag.ind, g, L * L, dtype=0, seed=1)
    count, wsum, indeg = (x.cpu().numpy() for x in net.topo_connectivity(d, L))
    oc, ow, oi = ot.connectivity_profile(rag.row_len, rag.ind, g, L)
    np.testing.assert_array_equal(count, oc)
    np.testing.assert_array_equal(indeg, oi)
    np.testing.assert_allclose(wsum, ow, rtol=1e-12, atol=1e-15)
    # outputs are overwritten, not added to
    count2 = net.topo_connectivity(d, L)[0].cpu().numpy()
    np.testing.assert_array_equal(count2, oc)
    abi.snn_topo_connectivity(d.handle, L)           # no outputs: nothing to do
    # empty matrix
    Le = 8
    e = net.DeviceRagged(np.zeros(Le * Le, np.int32), np.full((Le * Le, 4), -1, np.int32),
                         np.zeros((Le * Le, 4)), Le * Le, dtype=0)
    for x in net.topo_connectivity(e, Le):
        assert not x.cpu().numpy().any()
    with pytest.raises(abi.SnnError):
        abi.snn_topo_connectivity(d.handle, L + 1)
    d64 = net.DeviceRagged(np.zeros(64, np.int32), np.full((64, 4), -1, np.int32), np.zeros((64, 4)), 64,
                           dtype=abi.SNN_F64)
    with pytest.raises(abi.SnnError):
        abi.snn_topo_connectivity(d64.handle, 8)
    torch.cuda.synchronize()
