"""Topographic map with STDP and parallel rewiring — FP64 oracle (test infrastructure).

Sec. 2.1.3 (rewiring algorithm, Fig. 3) and Sec. 2.2.2 (model, Tab. 1-2) of the paper.

Per step t (dt = h):
 1. source layer: Poisson spikes; channel c fires with probability rate(c) dt where,
    with d the torus distance to the stimulus centre, the rate is either Tab. 1's
    Gaussian f_base + f_peak exp(-d^2 / (2 sigma_stim^2)) (sigma_stim > 0, f_in = f_peak)
    or a disc: f_in for d <= r, f_base outside (the 32 x 32 workload's profile); the
    centre is re-drawn every t_stim steps.  Replicated foci: the centre lives on a tile
    of side L_f and repeats on every tile (Sec. 2.2.2, s^2 stimulus locations when
    scaling).
 2. conductance: g_i <- g_i exp(-dt/tau_s) + sum of weights of spikes of step t-1
    (delay = one step, Tab. 2 t_d = h).
 3. conductance LIF (Tab. 1): in refractory steps V is held at V_reset; otherwise
    exponential Euler with g held over the step, which is the exact solution for
    constant g:  g_eff = g/g_leak, V_inf = (V_rest + g_eff E_exc)/(1 + g_eff),
    V <- V_inf + (V - V_inf) exp(-dt (1 + g_eff)/tau_m);  spike iff V >= V_theta, then
    V = V_reset for the next tau_ref/dt steps.
 4. all-to-all STDP (Tab. 1): traces decay (x with tau_+, y with tau_-); for each pre
    spike of t, every synapse of its row is depressed g <- max(0, g - A_- y_post) with y
    before the post spikes of t are counted; pre traces x += 1; for each post spike of t
    every synapse onto it is potentiated g <- min(g_max, g + A_+ x_pre) with the updated
    x; post traces y += 1.
 5. every `rewire_every` steps (after step t with (t+1) % rewire_every == 0), the
    rewiring of Sec. 2.1.3 on each projection, rewire index (t+1)/rewire_every - 1:
    N_att attempts distributed uniformly over rows with replacement; per row a_r
    distinct candidate targets (without replacement); existing synapses on candidates
    are eliminated with probability p_elim_dep (g < g_theta) or p_elim_pot; remaining
    candidates (empty slots) are formed with probability p_form exp(-d^2/(2 sigma^2))
    with g = g_max, no multapses; a full row skips the formation and counts overflow.

Units: conductances in units of g_leak (g_leak = 1), i.e. g_max = 0.2 means
0.2 x g_leak; the paper's "0.2 mS" with C_m = 20 nF would give g_max/g_leak = 200,
which saturates every neuron (parity unpinned for this reading; sanity-checked by
firing rates).  p_elim_dep = 2.45e-2 x 50 > 1 clamps to 1.

Pins (tests/test_oracle_topo.py): exponential Euler = analytic solution for constant
g; refractory hold; STDP pair rule for a single pre/post pair at lag Delta; Fig. 3's
worked example with scripted draws (compared as row sets); formation rate on empty
rows = (1/Q) p_form sum_j exp(-d^2/2 sigma^2) (binomial bound); all-depressed rows
lose every selected synapse; Poisson counts binomial; focus uniform.  The composition
of step() on scripted two- to four-neuron networks: a source spike reaches g one step
later (Tab. 2 delay t_d = h) after that step's decay; V then follows the numerically
integrated membrane equation for that g; a same-step pre/post pair is potentiated by
A+ (no depression), a later pre spike depressed by A- y with y decayed in between;
propagation uses the weights STDP left; rewiring follows STDP after steps with
(t + 1) % rewire_every == 0 only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox


@dataclass
class TopoParams:
    L: int = 32
    dt: float = 1.0
    # neuron (Tab. 2D; conductances in units of g_leak)
    tau_m: float = 20.0
    V_rest: float = -70.0
    E_exc: float = 0.0
    V_theta: float = -54.0
    V_reset: float = -70.0
    tau_ref: float = 5.0
    tau_s: float = 5.0
    g_leak: float = 1.0
    # input
    f_base: float = 20.0
    f_in: float = 100.0
    radius: int = 3
    t_stim: int = 20
    L_f: int | None = None      # focus tile side (None -> L: a single focus)
    sigma_stim: float = 0.0     # > 0: Gaussian profile f_base + f_in exp(-d^2/2 sigma^2) (Tab. 1 "Input")
    # STDP (Tab. 2F)
    g_max: float = 0.2
    tau_plus: float = 20.0
    tau_minus: float = 64.0
    B_ratio: float = 1.2
    # structural plasticity (Tab. 2G)
    p_form_ff: float = 0.16
    sigma_ff: float = 2.5
    p_form_lat: float = 1.0
    sigma_lat: float = 1.0
    p_elim_dep: float = 2.45e-2 * 50
    p_elim_pot: float = 1.36e-4 * 50
    n_att: int = 40
    rewire_every: int = 10

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def A_plus(self) -> float:
        return 0.1 * self.g_max

    @property
    def A_minus(self) -> float:
        return self.B_ratio * self.A_plus * self.tau_plus / self.tau_minus

    @property
    def g_theta(self) -> float:
        return 0.5 * self.g_max

    @property
    def n_ref(self) -> int:
        return int(round(self.tau_ref / self.dt))


def paper_setting(L: int = 16, **kw) -> TopoParams:
    """The model as Tab. 1-2 print it: time step h = 0.1 ms (so the 0.1 ms delay is one
    step), Gaussian input f_base 5 Hz + f_peak 152.8 Hz exp(-d^2 / (2 * 2^2)), stimulus
    interval 20 ms, rewiring every 1 ms with 10 attempts per 16 x 16 tile.  Conductances
    stay in units of g_leak (the one reading kept)."""
    dt = 0.1
    s = L // 16
    base = dict(L=L, dt=dt, f_base=5.0, f_in=152.8, sigma_stim=2.0, t_stim=int(round(20.0 / dt)),
                rewire_every=int(round(1.0 / dt)), n_att=10 * s * s, L_f=16 if s > 1 else None)
    base.update(kw)
    return TopoParams(**base)


def torus_d2(i: int, j: int, L: int) -> int:
    xi, yi, xj, yj = i % L, i // L, j % L, j // L
    dx = abs(xi - xj)
    dy = abs(yi - yj)
    dx = min(dx, L - dx)
    dy = min(dy, L - dy)
    return dx * dx + dy * dy


def form_thresholds(p_form: float, sigma: float, L: int) -> list[int]:
    """thr[d2] = threshold(p_form exp(-d2 / (2 sigma^2))) for every torus d2."""
    max_d2 = 2 * (L // 2) ** 2
    return [philox.threshold(p_form * math.exp(-d2 / (2.0 * sigma * sigma))) for d2 in range(max_d2 + 1)]


# ------------------------------------------------------------------------------ input

def focus(seed: int, period_idx: int, L_f: int) -> tuple[int, int]:
    u0 = philox.draw(seed, philox.TOPO_FOCUS, np.uint64(period_idx), 0, 0, 0, word=0)
    u1 = philox.draw(seed, philox.TOPO_FOCUS, np.uint64(period_idx), 0, 0, 0, word=1)
    return int(philox.mulhi(u0, L_f)), int(philox.mulhi(u1, L_f))


def input_spikes(seed: int, t: int, p: TopoParams) -> np.ndarray:
    L = p.L
    L_f = p.L_f or L
    fx, fy = focus(seed, t // p.t_stim, L_f)
    c = np.arange(L * L)
    dx = np.abs((c % L) % L_f - fx)
    dy = np.abs((c // L) % L_f - fy)
    dx = np.minimum(dx, L_f - dx)
    dy = np.minimum(dy, L_f - dy)
    d2 = dx * dx + dy * dy
    if p.sigma_stim > 0.0:
        # Tab. 1 "Input": rate f_base + f_peak exp(-d^2 / (2 sigma_stim^2)), f_in = f_peak
        thr = np.array([philox.threshold((p.f_base + p.f_in * math.exp(-int(q) / (2.0 * p.sigma_stim
                                                                                  * p.sigma_stim))) * p.dt * 1e-3)
                        for q in d2], dtype=np.uint64)
    else:
        inside = d2 <= p.radius * p.radius
        thr_in = np.uint64(philox.threshold(p.f_in * p.dt * 1e-3))
        thr_base = np.uint64(philox.threshold(p.f_base * p.dt * 1e-3))
        thr = np.where(inside, thr_in, thr_base).astype(np.uint64)
    cu = c.astype(np.uint64)
    u = philox.draw(seed, philox.TOPO_INPUT, np.uint64(t), cu // np.uint64(4), 0, 0,
                    word=(cu % np.uint64(4)).astype(np.int64))
    return u < thr


# ----------------------------------------------------------------------------- neuron

def neuron_step(V, gs, ref, I_in, p: TopoParams):
    """Returns (V, gs, ref, z) after one step of the conductance LIF."""
    V = V.copy()
    ref = ref.copy()
    gs = gs * math.exp(-p.dt / p.tau_s) + I_in
    z = np.zeros(len(V), dtype=bool)
    for i in range(len(V)):
        if ref[i] > 0:
            V[i] = p.V_reset
            ref[i] -= 1
            continue
        geff = gs[i] / p.g_leak
        Vinf = (p.V_rest + geff * p.E_exc) / (1.0 + geff)
        V[i] = Vinf + (V[i] - Vinf) * math.exp(-p.dt * (1.0 + geff) / p.tau_m)
        if V[i] >= p.V_theta:
            z[i] = True
            V[i] = p.V_reset
            ref[i] = p.n_ref
    return V, gs, ref, z


# ------------------------------------------------------------------------------- STDP

def stdp_step(projs, x_pre, y_post, pre_spikes, post_spikes, p: TopoParams):
    """All-to-all STDP for one step.  projs: list of (row_len, ind, g) arrays (modified
    in place), x_pre: list of pre-trace arrays (one per projection),
    pre_spikes: list of bool arrays, y_post/post_spikes: the shared target layer.
    Returns the new (x_pre list, y_post); traces are decayed inside."""
    dplus = math.exp(-p.dt / p.tau_plus)
    dminus = math.exp(-p.dt / p.tau_minus)
    y = y_post * dminus
    xs = [xp * dplus + sp for xp, sp in zip(x_pre, pre_spikes)]
    for (row_len, ind, g), sp in zip(projs, pre_spikes):
        for i in np.nonzero(sp)[0]:
            for s in range(int(row_len[i])):
                g[i, s] = max(0.0, g[i, s] - p.A_minus * y[ind[i, s]])
    post = np.asarray(post_spikes, dtype=bool)
    for (row_len, ind, g), x in zip(projs, xs):
        for i in range(len(row_len)):
            for s in range(int(row_len[i])):
                if post[ind[i, s]]:
                    g[i, s] = min(p.g_max, g[i, s] + p.A_plus * x[i])
    y = y + post
    return xs, y


# ----------------------------------------------------------------------------- rewire

@dataclass
class Draws:
    """Random decisions of one rewiring call; defaults come from Philox, tests may
    script them (Fig. 3)."""
    attempts: np.ndarray | None = None            # int [P] attempts per row
    candidates: dict = field(default_factory=dict)  # row -> list of targets
    R: dict = field(default_factory=dict)         # (row, target) -> uint64


def rewire(row_len, ind, g, C: int, Q: int, L: int, seed: int, rewire_idx: int, n_att: int,
           thr_dep: int, thr_pot: int, g_theta: float, thr_form: list[int], g_new: float,
           draws: Draws | None = None):
    """One parallel rewiring update (Sec. 2.1.3).  Returns a dict with the new
    (row_len, ind, g) and counts (removed, formed, overflow, attempts[P])."""
    P = len(row_len)
    row_len, ind, g = row_len.copy(), ind.copy(), g.copy()
    draws = draws or Draws()
    if draws.attempts is not None:
        att = np.asarray(draws.attempts, dtype=np.int64)
    else:
        k = np.arange(n_att, dtype=np.uint64)
        u = philox.draw(seed, philox.TOPO_ATT, np.uint64(rewire_idx), k // np.uint64(4), 0, 0,
                        word=(k % np.uint64(4)).astype(np.int64))
        att = np.bincount(philox.mulhi(u, P).astype(np.int64), minlength=P)
    att = np.minimum(att, Q)
    removed = formed = overflow = 0
    removed_d2, formed_d2 = [], []

    def R(i, j):
        if (i, j) in draws.R:
            return int(draws.R[(i, j)])
        return int(philox.draw(seed, philox.TOPO_DRAW, np.uint64(rewire_idx), np.uint64(i), np.uint64(j), 0, word=0))

    for i in range(P):
        a = int(att[i])
        if a == 0:
            continue
        cand = np.zeros(Q, dtype=bool)
        if i in draws.candidates:
            for j in draws.candidates[i]:
                cand[j] = True
        else:
            for kk in range(a):
                u = philox.draw(seed, philox.TOPO_CAND, np.uint64(rewire_idx), np.uint64(i), np.uint64(kk), 0, word=0)
                mth = int(philox.mulhi(u, Q - kk))
                free = np.nonzero(~cand)[0]
                cand[free[mth]] = True
        keep = []
        for s in range(int(row_len[i])):
            j = int(ind[i, s])
            if cand[j]:
                cand[j] = False
                thr = thr_dep if g[i, s] < g_theta else thr_pot
                if R(i, j) < thr:
                    removed += 1
                    removed_d2.append(torus_d2(i, j, L))
                    continue
            keep.append(s)
        k2 = len(keep)
        ind[i, :k2] = ind[i, keep]
        g[i, :k2] = g[i, keep]
        row_len[i] = k2
        for j in np.nonzero(cand)[0]:
            d2 = torus_d2(i, int(j), L)
            if R(i, int(j)) < thr_form[d2]:
                if row_len[i] < C:
                    s = int(row_len[i])
                    ind[i, s] = j
                    g[i, s] = g_new
                    row_len[i] = s + 1
                    formed += 1
                    formed_d2.append(d2)
                else:
                    overflow += 1
            cand[j] = False
    return {"row_len": row_len, "ind": ind, "g": g, "removed": removed, "formed": formed,
            "overflow": overflow, "attempts": att, "removed_d2": removed_d2, "formed_d2": formed_d2}


# ---------------------------------------------------------------------------- analysis
#
# Connectivity-evolution analysis of Sec. 3.2 (Figs. 8-9): eliminations and formations
# counted by the spatial separation of source and target (panels A-B), in- and
# out-degrees (panel C), connection probability and mean weight by displacement (panel D).

def d2_histogram(d2_list, L: int) -> np.ndarray:
    """Counts of squared torus distances, bins 0 .. 2 (L//2)^2."""
    h = np.zeros(2 * (L // 2) ** 2 + 1, dtype=np.int64)
    for d2 in d2_list:
        h[int(d2)] += 1
    return h


def unit_distance_bins(h_d2: np.ndarray) -> np.ndarray:
    """Regroup a squared-distance histogram into unit-width distance bins:
    bin b holds the d with b <= d < b + 1, i.e. the d^2 with floor(sqrt(d^2)) = b."""
    b = np.array([math.isqrt(d2) for d2 in range(len(h_d2))], dtype=np.int64)
    out = np.zeros(int(b[-1]) + 1, dtype=np.int64)
    np.add.at(out, b, np.asarray(h_d2, dtype=np.int64))
    return out


def connectivity_profile(row_len, ind, g, L: int):
    """For every synapse i -> j: displacement (dx, dy) = ((x_j - x_i) mod L,
    (y_j - y_i) mod L) with x = index mod L, y = index div L.  Returns
    count[dy*L + dx], wsum[dy*L + dx] (sum of the weights) and in_degree[j]; the
    out-degree of row i is row_len[i]."""
    N = L * L
    count = np.zeros(N, dtype=np.int64)
    wsum = np.zeros(N, dtype=np.float64)
    indeg = np.zeros(N, dtype=np.int64)
    for i in range(len(row_len)):
        for s in range(int(row_len[i])):
            j = int(ind[i, s])
            dx = (j % L - i % L) % L
            dy = (j // L - i // L) % L
            count[dy * L + dx] += 1
            wsum[dy * L + dx] += float(g[i, s])
            indeg[j] += 1
    return count, wsum, indeg


# ------------------------------------------------------------------------------- run

@dataclass
class TopoState:
    ff: list              # [row_len, ind, g]
    lat: list
    V: np.ndarray
    gs: np.ndarray
    ref: np.ndarray
    x_src: np.ndarray
    x_tgt: np.ndarray
    y: np.ndarray
    s_prev: np.ndarray    # source spikes of the previous step
    z_prev: np.ndarray    # target spikes of the previous step


def initial_state(ff, lat, p: TopoParams) -> TopoState:
    N = p.N
    return TopoState([a.copy() for a in ff], [a.copy() for a in lat], np.full(N, p.V_rest), np.zeros(N),
                     np.zeros(N, dtype=np.int64), np.zeros(N), np.zeros(N), np.zeros(N),
                     np.zeros(N, dtype=bool), np.zeros(N, dtype=bool))


def step(st: TopoState, t: int, p: TopoParams, seeds: dict, C: int, inputs=None) -> dict:
    """Advance the topographic network by one step (in place).  seeds: {"input",
    "ff", "lat"}.  inputs (tests): the source spikes of step t, instead of the Poisson
    draw.  Returns the step's spikes and rewiring stats."""
    N = p.N
    s = input_spikes(seeds["input"], t, p) if inputs is None else np.asarray(inputs, dtype=bool)
    I = propagate_rows(st.ff, st.s_prev, N)
    I += propagate_rows(st.lat, st.z_prev, N)
    st.V, st.gs, st.ref, z = neuron_step(st.V, st.gs, st.ref, I, p)
    projs = [tuple(st.ff), tuple(st.lat)]
    xs, st.y = stdp_step(projs, [st.x_src, st.x_tgt], st.y, [s, z], z, p)
    st.x_src, st.x_tgt = xs
    out = {"s": s, "z": z}
    if (t + 1) % p.rewire_every == 0:
        ridx = (t + 1) // p.rewire_every - 1
        for name, proj, pf, sg in (("ff", st.ff, p.p_form_ff, p.sigma_ff), ("lat", st.lat, p.p_form_lat, p.sigma_lat)):
            r = rewire(proj[0], proj[1], proj[2], C, N, p.L, seeds[name], ridx, p.n_att,
                       philox.threshold(p.p_elim_dep), philox.threshold(p.p_elim_pot), p.g_theta,
                       form_thresholds(pf, sg, p.L), p.g_max)
            proj[0], proj[1], proj[2] = r["row_len"], r["ind"], r["g"]
            out[name] = r
    st.s_prev, st.z_prev = s, z
    return out


def propagate_rows(proj, spikes, Q):
    row_len, ind, g = proj
    I = np.zeros(Q)
    for i in np.nonzero(spikes)[0]:
        for s in range(int(row_len[i])):
            I[ind[i, s]] += g[i, s]
    return I
