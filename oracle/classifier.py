"""Recurrent LIF/ALIF classifier with e-prop and Adam — FP64 oracle (test infrastructure).

Follows Sec. 2.2.1 of the paper (recurrent classifier) in its own indexing, with the
one-step synaptic delay of the voltage equation made explicit:

  I_j^t   = sum_{i: x_i^{t-1}} W^in_ji + sum_{i: z_i^{t-1}} W^rec_ji        (delay, Eq. for v)
  v_j^t   = alpha (v_j^{t-1} - z_j^{t-1} v_thr) + I_j^t                     (reset by subtraction)
  a_j^t   = rho a_j^{t-1} + z_j^{t-1}
  A_j^t   = v_thr + beta a_j^t ;  z_j^t = H(v_j^t - A_j^t), H(0) = 1
  psi_j^t = (0.3 / v_thr) max(0, 1 - |(v_j^t - A_j^t) / v_thr|)           (surrogate)
  y_k^t   = alpha y_k^{t-1} + sum_j W^out_kj z_j^{t-1} + b_k                (leaky readout)
  pi^t    = softmax(y^t) ;  d_k^t = pi_k^t - pi*_k ;  L_j^t = sum_k W^out_kj d_k^t  (B = W^out^T)

e-prop eligibility traces, forward in time, per synapse (i -> j), with zbar the
alpha-filtered presynaptic spike train (input spikes x for W^in):

  eps^t = psi_j^{t-1} zbar_i^{t-2} + (rho - psi_j^{t-1} beta) eps^{t-1}     (Eq. eprop_elig_1)
  e^t   = psi_j^t (zbar_i^{t-1} - beta eps^t)                               (Eq. eprop_elig_2, read as
                                                                             Bellec et al. 2020 write it)
  ebar^t = alpha ebar^{t-1} + e^t
  G_ji  += L_j^{t} ebar_ji^{t-1}      (learning signal paired one step after the trace,
                                       because z^{t-1} first reaches y at step t)
  G^out_kj += d_k^t zbar_j^{t-1} ;  G^b_k += d_k^t                          (delta rule)

LIF neurons are the case beta = 0, rho = 0, where e^t = psi_j^t zbar_i^{t-1}
(Eq. eprop_elig_lif).  Loss is the cross-entropy summed over every step; the
prediction is argmax_k sum_t y_k^t.  Gradients are summed over the trials of a batch,
L1 on the DEEP R sign bitfield is added, and Adam (Kingma & Ba; beta1 0.9, beta2 0.999,
eps 1e-8, bias correction by running products of beta) updates ragged and dense
weights (Sec. 2.1.2 "L1 regularisation", Sec. 3.1 "Adam optimizer with default
parameters").

Pins (tests/test_oracle_classifier.py): LIF closed form under constant drive and first
spike time; adaptation closed form; ragged propagation = dense masked product; e-prop
gradients = exact surrogate-gradient BPTT (torch.autograd, float64) when W^rec = 0;
Adam = torch.optim.Adam (float64); softmax/CE via the same BPTT check; L1 by hand.
The readout-bias rule (Delta b = sum_t d^t) is the paper's delta rule and is pinned by
hand sums, not by BPTT (it is not the exact gradient through a leaky readout).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import philox


@dataclass
class NeuronParams:
    tau_m: float = 20.0
    v_thr: float = 0.6
    beta: float = 0.0174
    tau_a: float | None = 2000.0     # None -> LIF (rho = 0, beta must be 0)
    dt: float = 1.0

    @property
    def alpha(self) -> float:
        return math.exp(-self.dt / self.tau_m)

    @property
    def rho(self) -> float:
        return 0.0 if self.tau_a is None else math.exp(-self.dt / self.tau_a)


def lif_params(v_thr: float = 1.0, tau_m: float = 20.0, dt: float = 1.0) -> NeuronParams:
    return NeuronParams(tau_m=tau_m, v_thr=v_thr, beta=0.0, tau_a=None, dt=dt)


# ------------------------------------------------------------------------------ input

def poisson_input(thr: np.ndarray, label: int, bin_len: int, trial_id: int, t: int, seed: int) -> np.ndarray:
    """Input spikes x^t of one trial: channel ch fires iff its 32-bit Philox draw is below
    the 32-bit threshold of its class template at the current (time-warped) bin.  One
    Philox block serves 8 channels: channel ch takes half ch % 2 (0 low, 1 high) of word
    (ch % 8) // 2 of counter (trial_id, t, ch // 8, 0)."""
    n_bins, n_in = thr.shape[1], thr.shape[2]
    b = min(n_bins - 1, t // int(bin_len))
    ch = np.arange(n_in, dtype=np.uint64)
    u = philox.draw(seed, philox.INPUT, np.uint64(trial_id), np.uint64(t), ch // np.uint64(8), 0,
                    word=((ch % np.uint64(8)) // np.uint64(2)).astype(np.int64))
    half = (u >> (np.uint64(32) * (ch % np.uint64(2)))) & np.uint64(0xFFFFFFFF)
    return half < thr[int(label), b, :].astype(np.uint64)


# ------------------------------------------------------------------------- propagation

def propagate(row_len: np.ndarray, ind: np.ndarray, w: np.ndarray, pre_spikes: np.ndarray, Q: int,
              out: np.ndarray | None = None) -> np.ndarray:
    """Ragged spike propagation (Fig. 1): for every spiking row i (ascending) and slot
    s < row_len[i], add w[i, s] to target ind[i, s]."""
    I = np.zeros(Q) if out is None else out
    for i in np.nonzero(pre_spikes)[0]:
        n = int(row_len[i])
        for s in range(n):
            I[ind[i, s]] += w[i, s]
    return I


# ----------------------------------------------------------------------------- neurons

def neuron_step(v, a, z_prev, I, p: NeuronParams):
    """One LIF/ALIF update; returns (v, a, z, psi, A)."""
    v = p.alpha * (v - z_prev * p.v_thr) + I
    a = p.rho * a + z_prev
    A = p.v_thr + p.beta * a
    z = (v >= A).astype(np.float64)
    psi = (0.3 / p.v_thr) * np.maximum(0.0, 1.0 - np.abs((v - A) / p.v_thr))
    return v, a, z, psi, A


def softmax(y: np.ndarray) -> np.ndarray:
    e = np.exp(y - np.max(y))
    return e / np.sum(e)


# ---------------------------------------------------------------------------- networks

@dataclass
class ClassifierNet:
    """Weights of one classifier (shared by every trial of a batch)."""
    n_in: int
    N: int
    K: int
    in_len: np.ndarray
    in_ind: np.ndarray
    w_in: np.ndarray
    rec_len: np.ndarray
    rec_ind: np.ndarray
    w_rec: np.ndarray
    W_out: np.ndarray      # [K, N]
    b_out: np.ndarray      # [K]
    neuron: NeuronParams


def forward_trial(net: ClassifierNet, thr: np.ndarray, label: int, bin_len: int, trial_id: int,
                  seed: int, T: int, state: dict | None = None, t0: int = 0) -> dict:
    """Simulate steps t0 .. t0+T-1 of one trial from `state` (v, a, z, x, y of step
    t0-1; zeros by default); return per-step records.

    records: x [T, n_in] (0/1), z [T, N], v, a, psi [T, N], y, pi, d [T, K],
    ysum [K] and the prediction argmax_k sum_t y_k^t.
    """
    p = net.neuron
    st = state or {}
    v = st.get("v", np.zeros(net.N)).copy()
    a = st.get("a", np.zeros(net.N)).copy()
    z = st.get("z", np.zeros(net.N)).copy()
    x_prev = st.get("x", np.zeros(net.n_in)).copy()
    y = st.get("y", np.zeros(net.K)).copy()
    onehot = np.zeros(net.K)
    onehot[int(label)] = 1.0
    rec = {k: [] for k in ("x", "z", "v", "a", "psi", "y", "pi", "d")}
    for t in range(t0, t0 + T):
        x = poisson_input(thr, label, bin_len, trial_id, t, seed).astype(np.float64)
        I = propagate(net.in_len, net.in_ind, net.w_in, x_prev, net.N)
        propagate(net.rec_len, net.rec_ind, net.w_rec, z, net.N, out=I)
        y = p.alpha * y + net.W_out @ z + net.b_out
        v, a, z, psi, _ = neuron_step(v, a, z, I, p)
        pi = softmax(y)
        for k, val in (("x", x), ("z", z), ("v", v), ("a", a), ("psi", psi), ("y", y), ("pi", pi),
                       ("d", pi - onehot)):
            rec[k].append(val.copy())
        x_prev = x
    out = {k: np.array(val) for k, val in rec.items()}
    out["ysum"] = out["y"].sum(axis=0)
    out["pred"] = int(np.argmax(out["ysum"]))
    out["final"] = {"v": v, "a": a, "z": z, "x": x_prev, "y": y}
    return out


def _slot_mask(row_len: np.ndarray, C: int) -> np.ndarray:
    return np.arange(C)[None, :] < row_len[:, None]


def eprop_gradients(net: ClassifierNet, x: np.ndarray, z: np.ndarray, psi: np.ndarray, d: np.ndarray):
    """e-prop gradients of one trial from its records, in the paper's forward-trace form.

    Returns (G_in [P_in, C_in], G_rec [N, C_rec], G_out [K, N], G_b [K]).
    """
    p = net.neuron
    alpha, rho, beta = p.alpha, p.rho, p.beta
    T = x.shape[0]
    projs = []
    for row_len, ind, pre in ((net.in_len, net.in_ind, x), (net.rec_len, net.rec_ind, z)):
        mask = _slot_mask(row_len, ind.shape[1])
        tgt = np.where(mask, ind, 0)
        projs.append({
            "mask": mask, "tgt": tgt, "pre": pre,
            "zb1": np.zeros(ind.shape[0]),       # zbar^{t-1}
            "zb2": np.zeros(ind.shape[0]),       # zbar^{t-2}
            "eps": np.zeros(ind.shape), "ebar": np.zeros(ind.shape), "G": np.zeros(ind.shape),
        })
    G_out = np.zeros((net.K, net.N))
    G_b = np.zeros(net.K)
    zbar_hid_prev = np.zeros(net.N)              # zbar_j^{t-1} for the readout rule
    psi_prev = np.zeros(net.N)
    for t in range(T):
        L = net.W_out.T @ d[t]
        for pr in projs:
            m = pr["mask"]
            pr["G"] += np.where(m, L[pr["tgt"]] * pr["ebar"], 0.0)
            psi_p = psi_prev[pr["tgt"]]
            pr["eps"] = np.where(m, psi_p * pr["zb2"][:, None] + (rho - psi_p * beta) * pr["eps"], 0.0)
            e = psi[t][pr["tgt"]] * (pr["zb1"][:, None] - beta * pr["eps"])
            pr["ebar"] = np.where(m, alpha * pr["ebar"] + e, 0.0)
            pr["zb2"] = pr["zb1"].copy()
            pr["zb1"] = alpha * pr["zb1"] + pr["pre"][t]
        G_out += np.outer(d[t], zbar_hid_prev)
        G_b += d[t]
        zbar_hid_prev = alpha * zbar_hid_prev + z[t]
        psi_prev = psi[t]
    return projs[0]["G"], projs[1]["G"], G_out, G_b


def eprop_synapse(pre: np.ndarray, psi_post: np.ndarray, L_post: np.ndarray, p: NeuronParams) -> float:
    """e-prop gradient of ONE synapse i -> j summed over trials, with the same trace
    recursion as eprop_gradients but vectorised over trials instead of synapses.
    pre: [B, T] presynaptic spikes, psi_post / L_post: [B, T] of the target neuron."""
    alpha, rho, beta = p.alpha, p.rho, p.beta
    B, T = pre.shape
    zb1 = np.zeros(B)
    zb2 = np.zeros(B)
    eps = np.zeros(B)
    ebar = np.zeros(B)
    G = np.zeros(B)
    psi_prev = np.zeros(B)
    for t in range(T):
        G += L_post[:, t] * ebar
        eps = psi_prev * zb2 + (rho - psi_prev * beta) * eps
        e = psi_post[:, t] * (zb1 - beta * eps)
        ebar = alpha * ebar + e
        zb2 = zb1
        zb1 = alpha * zb1 + pre[:, t]
        psi_prev = psi_post[:, t]
    return float(G.sum())


# ------------------------------------------------------------------------- optimiser

def l1_on_sign(G: np.ndarray, row_len: np.ndarray, ind: np.ndarray, sign_bits: np.ndarray, lam: float) -> np.ndarray:
    """DEEP R L1 custom update: add +lam to the gradient of slots whose potential
    connection is positive (sign bit set), -lam otherwise (Sec. 2.1.2)."""
    out = G.copy()
    for i in range(len(row_len)):
        for s in range(int(row_len[i])):
            j = int(ind[i, s])
            bit = (int(sign_bits[i, j >> 5]) >> (j & 31)) & 1
            out[i, s] += lam if bit else -lam
    return out


def adam_bias(beta: float, t: int) -> float:
    """beta^t as a running product (beta^0 = 1, then one multiplication per step): the
    form the bias correction 1 - beta^t of Adam takes when it is tracked step by step."""
    b = 1.0
    for _ in range(t):
        b *= beta
    return b


def adam(w, m, v, g, lr: float, b1t: float, b2t: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1); b1t, b2t are beta1^t, beta2^t."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - b1t)
    v_hat = v / (1.0 - b2t)
    w = w - lr * m_hat / (np.sqrt(v_hat) + eps)
    return w, m, v


def adam_ragged(w, m, v, g, row_len, lr, b1t, b2t, temperature: float = 0.0, nu=None, **kw):
    """Adam on the active slots (s < row_len) of a ragged matrix; padding untouched.
    temperature > 0: DEEP R's noise term, w += sqrt(2 lr T) nu after the Adam step
    (nu: standard normals per slot, from oracle.deepr.langevin_normals)."""
    mask = _slot_mask(row_len, w.shape[1])
    w2, m2, v2 = adam(w, m, v, g, lr, b1t, b2t, **kw)
    if temperature > 0.0:
        w2 = w2 + math.sqrt(2.0 * lr * temperature) * nu
    return np.where(mask, w2, w), np.where(mask, m2, m), np.where(mask, v2, v)
