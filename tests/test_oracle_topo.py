"""Pins of the topographic-map oracle: analytic neuron solution, STDP pair rule,
Fig. 3's worked example, closed-form formation rates, input statistics."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import philox
from oracle import topo


def test_exponential_euler_is_exact_for_constant_conductance():
    p = topo.TopoParams(tau_s=float("inf"), V_theta=1e9)
    N = 3
    V = np.array([-70.0, -60.0, -20.0])
    gs = np.array([0.0, 0.35, 2.0])
    ref = np.zeros(N, np.int64)
    V0 = V.copy()
    for t in range(1, 200):
        V, gs, ref, z = topo.neuron_step(V, gs, ref, np.zeros(N), p)
        Vinf = (p.V_rest + gs * p.E_exc) / (1 + gs)
        exact = Vinf + (V0 - Vinf) * np.exp(-t * p.dt * (1 + gs) / p.tau_m)
        np.testing.assert_allclose(V, exact, rtol=0, atol=1e-12)


def test_refractory_hold_and_conductance_decay():
    p = topo.TopoParams()
    V, gs, ref = np.array([-55.0]), np.array([0.0]), np.zeros(1, np.int64)
    V, gs, ref, z = topo.neuron_step(V, gs, ref, np.array([5.0]), p)   # strong kick -> spike
    assert z[0] and V[0] == p.V_reset and ref[0] == p.n_ref
    for k in range(p.n_ref):
        V, gs, ref, z = topo.neuron_step(V, gs, ref, np.zeros(1), p)
        assert V[0] == p.V_reset and not z[0]
    np.testing.assert_allclose(gs[0], 5.0 * math.exp(-p.dt / p.tau_s) ** p.n_ref, rtol=1e-12)
    V, gs, ref, z = topo.neuron_step(V, gs, ref, np.zeros(1), p)
    assert V[0] > p.V_reset


@pytest.mark.parametrize("lag", [1, 3, 10])
def test_stdp_pair_rule(lag):
    """One synapse 0 -> 0 starting mid-range: a pre spike then a post spike lag steps
    later changes g by +A_+ exp(-lag dt / tau_+); post then pre by -A_- exp(-lag dt / tau_-)."""
    p = topo.TopoParams()
    for order in ("pre_post", "post_pre"):
        proj = (np.array([1]), np.array([[0]]), np.array([[0.1]]))
        x, y = np.zeros(1), np.zeros(1)
        for t in range(lag + 1):
            pre = np.array([t == (0 if order == "pre_post" else lag)])
            post = np.array([t == (lag if order == "pre_post" else 0)])
            xs, y = topo.stdp_step([proj], [x], y, [pre], post, p)
            x = xs[0]
        dg = proj[2][0, 0] - 0.1
        if order == "pre_post":
            np.testing.assert_allclose(dg, p.A_plus * math.exp(-lag * p.dt / p.tau_plus), rtol=1e-12)
        else:
            np.testing.assert_allclose(dg, -p.A_minus * math.exp(-lag * p.dt / p.tau_minus), rtol=1e-12)


def test_fig3_worked_example_as_sets():
    """Fig. 3: six attempts on s0 (t0, t2), s2 (t2) and s4 (t2, t3, t0).  (s0,t0) is
    strong and stays, (s0,t2) and (s4,t2) are eliminated, (s4,t3) stays, (s2,t2) is
    formed and (s4,t0) is not."""
    P, Q, C = 5, 4, 3
    row_len = np.array([2, 1, 0, 2, 2], np.int32)
    ind = np.array([[0, 2, -1], [1, -1, -1], [-1, -1, -1], [3, 1, -1], [2, 3, -1]], np.int32)
    g_max, g_theta = 0.2, 0.1
    g = np.array([[0.18, 0.05, 0], [0.15, 0, 0], [0, 0, 0], [0.02, 0.19, 0], [0.03, 0.04, 0]])
    lo, hi = 0, 2 ** 64 - 1
    draws = topo.Draws(attempts=np.array([2, 0, 1, 0, 3]),
                       candidates={0: [0, 2], 2: [2], 4: [2, 3, 0]},
                       R={(0, 0): hi, (0, 2): lo, (4, 2): lo, (4, 3): hi, (2, 2): lo, (4, 0): hi})
    thr_form = [philox.threshold(0.5)] * 20
    out = topo.rewire(row_len, ind, g, C, Q, 4, seed=0, rewire_idx=0, n_att=6,
                      thr_dep=philox.threshold(0.5), thr_pot=philox.threshold(0.01), g_theta=g_theta,
                      thr_form=thr_form, g_new=g_max, draws=draws)
    rows = [set(out["ind"][i, :out["row_len"][i]]) for i in range(P)]
    assert rows == [{0}, {1}, {2}, {3, 1}, {3}]
    assert list(out["row_len"]) == [1, 1, 1, 2, 1]
    assert out["removed"] == 2 and out["formed"] == 1 and out["overflow"] == 0
    assert out["g"][2, 0] == g_max and out["g"][0, 0] == 0.18


def test_formation_rate_on_empty_rows_matches_gaussian_closed_form():
    L, n_att, calls = 16, 200, 150
    P = Q = L * L
    p_form, sigma = 0.16, 2.5
    thr_form = topo.form_thresholds(p_form, sigma, L)
    empty = (np.zeros(P, np.int32), np.full((P, 8), -1, np.int32), np.zeros((P, 8)))
    formed = 0
    shell = {}
    for r in range(calls):
        out = topo.rewire(*empty, 8, Q, L, seed=31, rewire_idx=r, n_att=n_att, thr_dep=0, thr_pot=0,
                          g_theta=0.1, thr_form=thr_form, g_new=0.2)
        formed += out["formed"]
        for d2 in out["formed_d2"]:
            shell[d2] = shell.get(d2, 0) + 1
    d2_all = synth.torus_d2(np.zeros(Q, np.int64), np.arange(Q), L)
    p_bar = np.mean(p_form * np.exp(-d2_all / (2 * sigma ** 2)))
    n = n_att * calls
    assert abs(formed - n * p_bar) < 5 * math.sqrt(n * p_bar * (1 - p_bar))
    # per distance shell: binomial with p = (#targets at d2 / Q) * p_form exp(-d2 / 2 sigma^2)
    for d2 in (0, 1, 2, 4, 5, 8):
        ps = np.sum(d2_all == d2) / Q * p_form * math.exp(-d2 / (2 * sigma ** 2))
        assert abs(shell.get(d2, 0) - n * ps) < 5 * math.sqrt(n * ps * (1 - ps)) + 1


def test_depressed_full_rows_lose_every_selected_synapse():
    P = Q = 9
    C = Q
    row_len = np.full(P, Q, np.int32)
    rng = np.random.default_rng(0)
    ind = np.array([rng.permutation(Q) for _ in range(P)], np.int32)
    g = np.full((P, C), 0.05)
    for r in range(5):
        out = topo.rewire(row_len, ind, g, C, Q, 3, seed=8, rewire_idx=r, n_att=12,
                          thr_dep=philox.threshold(2.45e-2 * 50), thr_pot=0, g_theta=0.1,
                          thr_form=[2 ** 64 - 1] * 10, g_new=0.2)
        assert out["removed"] == out["attempts"].sum() == 12
        assert out["formed"] == 0
        for i in range(P):
            kept = [j for j in ind[i] if j in set(out["ind"][i, :out["row_len"][i]])]
            assert list(out["ind"][i, :out["row_len"][i]]) == kept     # stable order


def test_full_row_formation_counts_overflow():
    P = Q = 4
    C = 1
    row_len = np.ones(P, np.int32)
    ind = np.array([[0], [1], [2], [3]], np.int32)
    g = np.full((P, 1), 0.2)
    draws = topo.Draws(attempts=np.array([2, 0, 0, 0]), candidates={0: [0, 3]},
                       R={(0, 0): 2 ** 64 - 1, (0, 3): 0})
    out = topo.rewire(row_len, ind, g, C, Q, 2, 0, 0, 2, 0, 0, 0.1, [2 ** 64 - 1] * 5, 0.2, draws=draws)
    assert out["overflow"] == 1 and out["formed"] == 0 and out["removed"] == 0


def test_input_rates_and_focus():
    p = topo.TopoParams(L=16)
    seed = 5
    T = 4000
    inside_cnt = outside_cnt = 0
    inside_n = outside_n = 0
    foci = []
    for t in range(T):
        s = topo.input_spikes(seed, t, p)
        fx, fy = topo.focus(seed, t // p.t_stim, p.L)
        if t % p.t_stim == 0:
            foci.append(fx + p.L * fy)
        c = np.arange(p.N)
        d2 = synth.torus_d2(np.full(p.N, fx + p.L * fy), c, p.L)
        ins = d2 <= p.radius ** 2
        inside_cnt += s[ins].sum()
        outside_cnt += s[~ins].sum()
        inside_n += ins.sum()
        outside_n += (~ins).sum()
    for cnt, n, prob in ((inside_cnt, inside_n, 0.1), (outside_cnt, outside_n, 0.02)):
        assert abs(cnt - n * prob) < 5 * math.sqrt(n * prob * (1 - prob))
    assert len(set(foci)) > 100


def test_initial_degree_matches_lattice_sum():
    L, p_form, sigma = 32, 0.16, 2.5
    rag = synth.topo_initial(3, L, p_form, sigma, 64, 0.2)
    d2 = synth.torus_d2(np.zeros(L * L, np.int64), np.arange(L * L), L)
    K = p_form * np.exp(-d2 / (2 * sigma ** 2)).sum()
    assert abs(K - 2 * math.pi * p_form * sigma ** 2) < 0.01        # the paper's K, read as 2 pi p sigma^2
    var = (p_form * np.exp(-d2 / (2 * sigma ** 2)) * (1 - p_form * np.exp(-d2 / (2 * sigma ** 2)))).sum()
    assert abs(rag.row_len.mean() - K) < 5 * math.sqrt(var / (L * L))


def test_short_run_invariants():
    p = topo.TopoParams(L=8, n_att=10)
    ff = synth.topo_initial(1, p.L, p.p_form_ff, p.sigma_ff, 16, p.g_max)
    lat = synth.topo_initial(2, p.L, p.p_form_lat, p.sigma_lat, 16, p.g_max)
    st = topo.initial_state([ff.row_len, ff.ind, ff.w], [lat.row_len, lat.ind, lat.w], p)
    seeds = {"input": 1, "ff": 2, "lat": 3}
    spikes = 0
    for t in range(60):
        out = topo.step(st, t, p, seeds, 16)
        spikes += out["z"].sum()
        for proj in (st.ff, st.lat):
            assert np.all(proj[0] <= 16)
            for i in range(p.N):
                tg = list(proj[1][i, :proj[0][i]])
                assert len(set(tg)) == len(tg)
                assert np.all((proj[2][i, :proj[0][i]] >= 0) & (proj[2][i, :proj[0][i]] <= p.g_max))
    assert spikes > 0


def _paper_tables():
    rows = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "topo_parameter_tables.txt")
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        fields, src = line.split(";", 1)
        name, value = fields.split()[:2]
        rows[name] = (float(value), "reading" in src)
    return rows


def test_parameters_match_paper_tables():
    """TopoParams' defaults are the printed table values (apart from the lines the
    fixture marks as readings), and the derived quantities follow the printed formulas:
    A+ = 0.1 g_max, A- = B A+ tau+ / tau-, g_theta = g_max / 2."""
    tab = _paper_tables()
    p = topo.TopoParams()
    direct = {"tau_m": p.tau_m, "V_rest": p.V_rest, "E_exc": p.E_exc, "V_theta": p.V_theta,
              "V_reset": p.V_reset, "tau_ref": p.tau_ref, "tau_s": p.tau_s, "t_stim": p.t_stim,
              "g_max": p.g_max, "B_ratio": p.B_ratio, "tau_plus": p.tau_plus, "tau_minus": p.tau_minus,
              "p_form_ff": p.p_form_ff, "sigma_ff": p.sigma_ff, "p_form_lat": p.p_form_lat,
              "sigma_lat": p.sigma_lat, "p_elim_dep": p.p_elim_dep, "p_elim_pot": p.p_elim_pot,
              "A_plus_over_g_max": p.A_plus / p.g_max, "g_theta_over_g_max": p.g_theta / p.g_max}
    for name, got in direct.items():
        value, reading = tab[name]
        assert not reading, name
        assert got == pytest.approx(value, rel=1e-12), name
    assert p.A_minus == pytest.approx(1.2 * 0.1 * 0.2 * 20.0 / 64.0, rel=1e-12)
    # the scaled sheet: L = L0 s with s = 2 for the 32 x 32 workload
    assert p.L == 2 * int(tab["L0"][0])
    # reading lines are the documented replacements, not silent changes
    assert all(tab[n][1] for n in ("t_d", "C_m", "f_base", "f_peak", "sigma_stim", "N_attempts", "h", "t_rewiring"))
    # rewiring every t_rewiring / h steps, as printed (10), at the oracle's 1 ms step
    assert p.rewire_every == round(tab["t_rewiring"][0] / tab["h"][0])


# --------------------------------------------------------------------- connectivity analysis

def _row_sets(row_len, ind):
    return [set(int(j) for j in ind[i, :row_len[i]]) for i in range(len(row_len))]


def test_event_histograms_equal_the_row_set_differences_of_each_call():
    """Within one rewiring call a candidate is either eliminated or formed, never both,
    so the call's eliminations are exactly the synapses missing afterwards and its
    formations the ones that are new; their squared-distance histograms must equal the
    ones the rewiring records."""
    L, C = 16, 16
    p = topo.TopoParams(L=L, n_att=400)
    rag = synth.topo_initial(6, L, p.p_form_ff, p.sigma_ff, C, p.g_max)
    rng = np.random.default_rng(3)
    g = np.where(rag.ind >= 0, rng.uniform(0, p.g_max, rag.w.shape), 0.0)
    state = (rag.row_len, rag.ind, g)
    tot_rm = tot_fm = 0
    for r in range(6):
        out = topo.rewire(*state, C, L * L, L, 17, r, p.n_att, philox.threshold(p.p_elim_dep),
                          philox.threshold(p.p_elim_pot), p.g_theta,
                          topo.form_thresholds(p.p_form_ff, p.sigma_ff, L), p.g_max)
        before, after = _row_sets(state[0], state[1]), _row_sets(out["row_len"], out["ind"])
        gone = [topo.torus_d2(i, j, L) for i in range(L * L) for j in before[i] - after[i]]
        new = [topo.torus_d2(i, j, L) for i in range(L * L) for j in after[i] - before[i]]
        np.testing.assert_array_equal(topo.d2_histogram(out["removed_d2"], L), topo.d2_histogram(gone, L))
        np.testing.assert_array_equal(topo.d2_histogram(out["formed_d2"], L), topo.d2_histogram(new, L))
        tot_rm += len(gone)
        tot_fm += len(new)
        state = (out["row_len"], out["ind"], out["g"])
    assert tot_rm > 20 and tot_fm > 20


def test_unit_distance_bins_by_hand():
    # L = 4: squared distances 0..8; d = 0 -> bin 0; 1, sqrt2, sqrt3 -> 1; 2 .. sqrt8 -> 2
    h = np.arange(1, 10, dtype=np.int64)                     # h[d2] = d2 + 1
    np.testing.assert_array_equal(topo.unit_distance_bins(h), [1, 2 + 3 + 4, 5 + 6 + 7 + 8 + 9])
    # L = 8: d2 = 9 (d = 3) opens bin 3, d2 = 16 (d = 4) bin 4, d2 = 32 is the largest
    h = np.zeros(33, dtype=np.int64)
    h[[8, 9, 15, 16, 32]] = 1
    np.testing.assert_array_equal(topo.unit_distance_bins(h), [0, 0, 1, 2, 1, 1])


def test_connectivity_profile_by_hand():
    # 3 x 3 torus; x = index % 3, y = index // 3
    L = 3
    row_len = np.zeros(9, np.int32)
    ind = np.full((9, 3), -1, np.int32)
    g = np.zeros((9, 3))
    def put(i, js, ws):
        row_len[i] = len(js)
        ind[i, :len(js)] = js
        g[i, :len(js)] = ws
    put(0, [1, 3, 8], [0.5, 0.25, 0.125])    # (0,0) -> (1,0), (0,1), (2,2)
    put(4, [0, 4], [1.0, 2.0])               # (1,1) -> (0,0) = (-1,-1) = (2,2); itself (0,0)
    put(7, [1], [4.0])                       # (1,2) -> (1,0): dy = -2 = 1
    count, wsum, indeg = topo.connectivity_profile(row_len, ind, g, L)
    want_c = np.zeros(9, np.int64)
    want_w = np.zeros(9)
    for (dx, dy), w in (((1, 0), 0.5), ((0, 1), 0.25), ((2, 2), 0.125), ((2, 2), 1.0), ((0, 0), 2.0),
                        ((0, 1), 4.0)):
        want_c[dy * L + dx] += 1
        want_w[dy * L + dx] += w
    np.testing.assert_array_equal(count, want_c)
    np.testing.assert_array_equal(wsum, want_w)
    np.testing.assert_array_equal(indeg, [1, 2, 0, 1, 1, 0, 0, 0, 1])


def test_connectivity_profile_of_initial_maps_follows_the_formation_law():
    """Pairwise-Bernoulli initial connectivity: the synapses at displacement (dx, dy)
    number Binomial(N, p_form exp(-d^2 / 2 sigma^2)); in- and out-degrees sum to the
    synapse count and have the lattice-sum mean."""
    L, p_form, sigma = 32, 0.16, 2.5
    N = L * L
    rag = synth.topo_initial(9, L, p_form, sigma, 64, 0.2)
    rng = np.random.default_rng(1)
    g = np.where(rag.ind >= 0, rng.uniform(0, 0.2, rag.w.shape), 0.0)
    count, wsum, indeg = topo.connectivity_profile(rag.row_len, rag.ind, g, L)
    assert count.sum() == indeg.sum() == rag.row_len.sum()
    d2 = synth.torus_d2(np.zeros(N, np.int64), np.arange(N), L)      # displacement k = (k % L, k // L)
    pk = p_form * np.exp(-d2 / (2 * sigma ** 2))
    assert np.all(np.abs(count - N * pk) <= 5 * np.sqrt(N * pk * (1 - pk)) + 1)
    # weights U[0, 0.2): the mean weight of each well-populated displacement is near 0.1
    big = count > 100
    assert np.all(np.abs(wsum[big] / count[big] - 0.1) < 5 * 0.2 / math.sqrt(12) / np.sqrt(count[big]))
    assert abs(indeg.mean() - pk.sum()) < 5 * math.sqrt((pk * (1 - pk)).sum() / N)


# ------------------------------------------------------------- the paper's own setting

def test_paper_setting_matches_the_printed_tables():
    """oracle.topo.paper_setting reproduces the printed time step, delay, input and
    rewiring-interval lines that the default workload replaces by readings."""
    tab = _paper_tables()
    p = topo.paper_setting(16)
    assert p.dt == tab["h"][0] == tab["t_d"][0]                      # delay = one step
    assert p.f_base == tab["f_base"][0] and p.f_in == tab["f_peak"][0]
    assert p.sigma_stim == tab["sigma_stim"][0]
    assert p.t_stim * p.dt == pytest.approx(tab["t_stim"][0])
    assert p.rewire_every * p.dt == pytest.approx(tab["t_rewiring"][0])
    assert p.n_att == tab["N_attempts"][0]
    assert topo.paper_setting(32).n_att == 4 * tab["N_attempts"][0]  # scaled with s^2
    assert p.n_ref * p.dt == pytest.approx(tab["tau_ref"][0])


def test_gaussian_input_rates_follow_the_profile():
    """With the focus held (one stimulus interval), channel firing counts in each
    squared-distance shell are binomial with p = (5 + 152.8 exp(-d^2/8)) Hz x 0.1 ms."""
    p = topo.paper_setting(16, t_stim=10 ** 9)
    seed, T = 3, 3000
    fx, fy = topo.focus(seed, 0, p.L)
    d2 = synth.torus_d2(np.full(p.N, fx + p.L * fy), np.arange(p.N), p.L)
    cnt = np.zeros(p.N)
    for t in range(T):
        cnt += topo.input_spikes(seed, t, p)
    for shell in (0, 1, 2, 4, 5, 8, 9, 10, 13, 25, 50, 128):
        m = d2 == shell
        if not m.any():
            continue
        prob = (5.0 + 152.8 * math.exp(-shell / 8.0)) * 1e-4
        n = T * m.sum()
        assert abs(cnt[m].sum() - n * prob) < 5 * math.sqrt(n * prob * (1 - prob)) + 1, shell
    # the profile's threshold at the focus in closed form
    assert philox.threshold((5.0 + 152.8) * 0.1 * 1e-3) == int((5.0 + 152.8) * 0.1 * 1e-3 * 2.0 ** 64)


# --------------------------------------------------------- composition of one step
#
# Tab. 2 fixes the synaptic delay t_d at one time step h, the exponential synapse
# (g decays with tau_s, each spike adds its weight) and the rewiring period; Tab. 1
# fixes the pair-based STDP rule.  These scripted networks pin how topo.step() puts
# the parts together: a source spike of step t reaches the conductance at step t + 1,
# after that step's decay; the membrane then integrates the new conductance; STDP runs
# after the neuron update with the depression seeing y before the step's post spikes
# and the potentiation seeing x after the step's pre spikes; propagation at t + 1 uses
# the weights STDP left at t; rewiring follows STDP after steps with
# (t + 1) % rewire_every == 0.  A zero-delay, jump-before-decay, swapped-STDP or
# off-by-one-cadence version of step() fails one of them.

def _scripted(L, C, syn, **kw):
    """Topographic state with feed-forward synapses `syn` = [(i, j, w), ...], no lateral
    ones, silent Poisson input (inputs are scripted per step)."""
    p = topo.TopoParams(L=L, n_att=kw.pop("n_att", 0), f_base=0.0, f_in=0.0, **kw)
    N = p.N
    ff = [np.zeros(N, np.int32), np.full((N, C), -1, np.int32), np.zeros((N, C))]
    for i, j, w in syn:
        s = int(ff[0][i])
        ff[1][i, s], ff[2][i, s] = j, w
        ff[0][i] = s + 1
    lat = [np.zeros(N, np.int32), np.full((N, C), -1, np.int32), np.zeros((N, C))]
    return p, topo.initial_state(ff, lat, p)


def _run(st, p, C, script, t_end):
    """Steps 0 .. t_end - 1; script[t] = source neurons spiking at step t.  Returns the
    state arrays recorded after every step."""
    rec = []
    for t in range(t_end):
        s = np.zeros(p.N, bool)
        s[list(script.get(t, ()))] = True
        out = topo.step(st, t, p, {"input": 1, "ff": 2, "lat": 3}, C, inputs=s)
        rec.append({"gs": st.gs.copy(), "V": st.V.copy(), "z": out["z"].copy(), "w": st.ff[2].copy(),
                    "x": st.x_src.copy(), "y": st.y.copy(), "rewired": "ff" in out, "out": out})
    return rec


def _cond_lif_exact(V0, g, p, dt):
    """Membrane equation tau_m dV/dt = (V_rest - V) + g/g_leak (E_exc - V) with g held
    over the step, integrated numerically (an independent check of the closed form)."""
    from scipy.integrate import solve_ivp
    f = lambda _t, V: [((p.V_rest - V[0]) + g / p.g_leak * (p.E_exc - V[0])) / p.tau_m]  # noqa: E731
    return solve_ivp(f, (0.0, dt), [V0], rtol=1e-12, atol=1e-12, method="DOP853").y[0, -1]


def test_source_spike_reaches_the_conductance_one_step_later_after_the_decay():
    w = 0.05
    p, st = _scripted(2, 4, [(0, 1, w)])
    rec = _run(st, p, 4, {3: [0]}, 7)
    for t in range(4):
        assert rec[t]["gs"][1] == 0.0, t                   # nothing before the delay has passed
        assert rec[t]["V"][1] == p.V_rest, t
    assert rec[4]["gs"][1] == w                            # 0 * decay + w: decay first, then the jump
    assert rec[5]["gs"][1] == pytest.approx(w * math.exp(-p.dt / p.tau_s), rel=1e-15)
    assert rec[6]["gs"][1] == pytest.approx(w * math.exp(-2 * p.dt / p.tau_s), rel=1e-15)
    assert np.all(rec[6]["gs"][[0, 2, 3]] == 0.0)          # only the target receives it


def test_membrane_integrates_the_conductance_of_its_own_step():
    w = 0.05
    p, st = _scripted(2, 4, [(0, 1, w)])
    rec = _run(st, p, 4, {3: [0]}, 6)
    V4 = _cond_lif_exact(p.V_rest, w, p, p.dt)
    assert rec[4]["V"][1] == pytest.approx(V4, abs=1e-9)
    assert rec[4]["V"][1] > p.V_rest + 1e-3                # the jump of step 4 is already felt
    V5 = _cond_lif_exact(rec[4]["V"][1], w * math.exp(-p.dt / p.tau_s), p, p.dt)
    assert rec[5]["V"][1] == pytest.approx(V5, abs=1e-9)
    assert rec[5]["V"][0] == p.V_rest


def test_stdp_within_a_step_and_propagation_of_the_updated_weight():
    """Source 0 drives target 1 over threshold (its spike of step 3 arrives at step 4);
    source 2 fires at step 4 too, so synapse 2 -> 1 sees a pre and a post spike in the
    same step: no depression (y before the post spike is 0), potentiation by A+ x with
    x = 1 (this step's pre spike counted).  Source 2 fires again at step 7: depression
    by A- y with y decayed over three steps.  Its spike of step 4 arrives at step 5 with
    the weight STDP left at step 4."""
    w_drive, w0 = 50.0, 0.05
    p, st = _scripted(2, 4, [(0, 1, w_drive), (2, 1, w0)])
    rec = _run(st, p, 4, {3: [0], 4: [2], 7: [2]}, 8)
    assert not rec[3]["z"].any() and rec[4]["z"][1] and rec[4]["z"].sum() == 1
    assert rec[4]["x"][2] == 1.0 and rec[4]["y"][1] == 1.0
    w_after4 = w0 + p.A_plus * 1.0
    assert rec[4]["w"][2, 0] == pytest.approx(w_after4, rel=1e-15)
    assert rec[4]["w"][0, 0] == p.g_max                    # 50 + A+ e^{-1/20} clamped
    assert rec[5]["gs"][1] == pytest.approx(w_drive * math.exp(-p.dt / p.tau_s) + w_after4, rel=1e-15)
    for t in (5, 6):
        assert rec[t]["w"][2, 0] == pytest.approx(w_after4, rel=1e-15)
    assert not rec[5]["z"].any() and not rec[6]["z"].any() and not rec[7]["z"].any()   # refractory
    y7 = math.exp(-3 * p.dt / p.tau_minus)
    assert rec[7]["w"][2, 0] == pytest.approx(w_after4 - p.A_minus * y7, rel=1e-14)


def test_rewiring_runs_after_steps_with_t_plus_1_multiple_of_the_period_after_stdp():
    """4 x 4 sheets, every target a candidate of every row (2000 attempts).  The
    network is silent except for a scripted pair that potentiates synapse 5 -> 6 from
    below g_theta to above it in step 9 itself: rewiring after STDP sees it potentiated
    and (with this seed's draw) keeps it, where a depressed synapse is always removed
    (p_elim_dep clamps to 1).  Rewiring happens after steps 9 and 19 only, with rewire
    indices 0 and 1."""
    L, C = 4, 16
    g_theta = 0.5 * 0.2
    w56 = g_theta - 0.01
    p, st = _scripted(L, C, [(0, 6, 50.0), (5, 6, w56), (3, 9, 0.15)], n_att=2000)
    assert p.rewire_every == 10
    seed_ff = 2
    R = philox.draw(seed_ff, philox.TOPO_DRAW, np.uint64(0), np.uint64(5), np.uint64(6), 0, word=0)
    assert int(R) >= philox.threshold(p.p_elim_pot)        # kept if potentiated
    rec = _run(st, p, C, {7: [5], 8: [0]}, 20)
    assert [t for t in range(20) if rec[t]["rewired"]] == [9, 19]
    assert rec[9]["z"][6]                                   # post spike of step 9
    assert rec[8]["w"][5, 0] == w56
    # the rewiring of step 9 starts from the state after step 9's STDP
    pre = rec[9]["out"]["ff"]
    assert 6 in set(pre["ind"][5, :pre["row_len"][5]].tolist())
    # the same call on the pre-STDP weights (a rewiring placed before STDP) removes it
    w_pre = rec[8]["w"].copy()
    ff_len = np.array([1 if i in (0, 5, 3) else 0 for i in range(p.N)], np.int32)
    ind0 = np.full((p.N, C), -1, np.int32)
    ind0[0, 0], ind0[5, 0], ind0[3, 0] = 6, 6, 9
    early = topo.rewire(ff_len, ind0, w_pre, C, p.N, L, seed_ff, 0, p.n_att, philox.threshold(p.p_elim_dep),
                        philox.threshold(p.p_elim_pot), p.g_theta, topo.form_thresholds(p.p_form_ff, p.sigma_ff, L),
                        p.g_max)
    assert 6 not in set(early["ind"][5, :early["row_len"][5]].tolist())
    # index 1 at step 19: the draws of rewire index 1 (attempt histogram) were used
    att1 = np.bincount(philox.mulhi(philox.draw(seed_ff, philox.TOPO_ATT, np.uint64(1),
                                                np.arange(p.n_att, dtype=np.uint64) // np.uint64(4), 0, 0,
                                                word=(np.arange(p.n_att) % 4).astype(np.int64)), p.N).astype(np.int64),
                       minlength=p.N)
    np.testing.assert_array_equal(rec[19]["out"]["ff"]["attempts"], np.minimum(att1, p.N))
