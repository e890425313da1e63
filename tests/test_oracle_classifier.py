"""Pins of the classifier oracle: closed forms, brute force, BPTT and torch's Adam."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import classifier as oc

ALWAYS = np.uint64(2 ** 64 - 1)


def _net(n_in, N, K, in_rag, rec_rag, W_out, b, neuron):
    return oc.ClassifierNet(n_in, N, K, in_rag.row_len, in_rag.ind, in_rag.w, rec_rag.row_len, rec_rag.ind,
                            rec_rag.w, W_out, b, neuron)


def _one_to_one(I0):
    in_rag = synth.Ragged(1, 1, 1, np.array([1], np.int32), np.array([[0]], np.int32), np.array([[I0]]))
    rec_rag = synth.Ragged(1, 1, 1, np.array([0], np.int32), np.array([[-1]], np.int32), np.zeros((1, 1)))
    return in_rag, rec_rag


def test_lif_constant_drive_closed_form():
    I0 = 0.37
    p = oc.lif_params(v_thr=1e9)
    in_rag, rec_rag = _one_to_one(I0)
    net = _net(1, 1, 2, in_rag, rec_rag, np.zeros((2, 1)), np.zeros(2), p)
    thr = np.full((2, 1, 1), ALWAYS, dtype=np.uint64)
    r = oc.forward_trial(net, thr, 0, 100, 0, 1, 100)
    t = np.arange(100)
    a = p.alpha
    np.testing.assert_allclose(r["v"][:, 0], I0 * (1 - a ** t) / (1 - a), rtol=1e-12, atol=1e-15)
    assert r["z"].sum() == 0


def test_lif_spike_train_closed_form():
    """Between spikes the subtraction-reset LIF obeys v^{t1+k} = a^k (v^{t1} - v_thr)
    + I0 (1 - a^k)/(1 - a); predict the whole spike train interval by interval."""
    I0, v_thr, T = 0.3, 1.0, 300
    p = oc.lif_params(v_thr=v_thr)
    in_rag, rec_rag = _one_to_one(I0)
    net = _net(1, 1, 2, in_rag, rec_rag, np.zeros((2, 1)), np.zeros(2), p)
    thr = np.full((2, 1, 1), ALWAYS, dtype=np.uint64)
    r = oc.forward_trial(net, thr, 0, T, 0, 1, T)
    a = p.alpha
    spikes = []
    t = 0
    while t < T and I0 * (1 - a ** t) / (1 - a) < v_thr:      # before the first spike
        t += 1
    if t < T:
        tn, Vn = t, I0 * (1 - a ** t) / (1 - a)
        spikes.append(tn)
        while True:
            k = 1
            while tn + k < T:
                vk = a ** k * (Vn - v_thr) + I0 * (1 - a ** k) / (1 - a)
                if vk >= v_thr:
                    break
                k += 1
            if tn + k >= T:
                break
            tn, Vn = tn + k, vk
            spikes.append(tn)
    assert list(np.nonzero(r["z"][:, 0])[0]) == spikes
    assert len(spikes) > 10


def test_alif_adaptation_closed_form():
    rng = np.random.default_rng(3)
    n_in, N, K, T = 12, 8, 3, 150
    p = oc.NeuronParams(tau_m=20.0, v_thr=0.6, beta=0.2, tau_a=200.0)
    in_rag = synth.random_ragged(1, n_in, N, 0.5, w_std=0.5)
    in_rag.w = np.where(in_rag.ind >= 0, np.abs(in_rag.w) + 0.2, 0.0)
    rec_rag = synth.random_ragged(2, N, N, 0.3, no_autapse=True, w_std=0.3)
    net = _net(n_in, N, K, in_rag, rec_rag, rng.normal(0, 0.3, (K, N)), np.zeros(K), p)
    thr = synth.rates_to_thresholds(np.full((1, 1, n_in), 150.0), 1.0)
    r = oc.forward_trial(net, thr, 0, T, 5, 9, T)
    z = r["z"]
    assert 20 < z.sum() < T * N - 20
    for t in range(T):
        a_cf = sum(p.rho ** (t - 1 - s) * z[s] for s in range(t)) if t else np.zeros(N)
        np.testing.assert_allclose(r["a"][t], a_cf, rtol=1e-12, atol=1e-14)
        A = p.v_thr + p.beta * r["a"][t]
        np.testing.assert_array_equal(z[t], (r["v"][t] >= A).astype(float))


def test_propagate_equals_dense_masked_product():
    rag = synth.random_ragged(11, 30, 20, 0.3)
    W = np.zeros((20, 30))
    for i in range(30):
        for s in range(rag.row_len[i]):
            W[rag.ind[i, s], i] += rag.w[i, s]
    rng = np.random.default_rng(0)
    for _ in range(5):
        sp = rng.random(30) < 0.4
        np.testing.assert_allclose(oc.propagate(rag.row_len, rag.ind, rag.w, sp, 20), W @ sp, rtol=1e-13, atol=1e-14)


class _Spike(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v_thr):
        ctx.save_for_backward(u)
        ctx.v_thr = v_thr
        return (u >= 0).to(u.dtype)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        return g * (0.3 / ctx.v_thr) * torch.clamp(1 - torch.abs(u / ctx.v_thr), min=0), None


def _dense(rag, Q):
    W = np.zeros((Q, rag.P))
    M = np.zeros((Q, rag.P))
    for i in range(rag.P):
        for s in range(rag.row_len[i]):
            W[rag.ind[i, s], i] = rag.w[i, s]
            M[rag.ind[i, s], i] = 1
    return W, M


@pytest.mark.parametrize("kind", ["lif", "alif"])
def test_eprop_equals_bptt_without_recurrence(kind):
    """With W^rec = 0 e-prop is exact BPTT with the surrogate derivative and the
    reset path detached: compare W^in, W^rec (at 0) and W^out gradients."""
    n_in, N, K, T = 10, 7, 3, 80
    if kind == "lif":
        p = oc.lif_params(v_thr=1.0)
    else:
        p = oc.NeuronParams(tau_m=20.0, v_thr=0.6, beta=0.3, tau_a=100.0)
    in_rag = synth.random_ragged(4, n_in, N, 0.6, w_std=0.4)
    in_rag.w = np.where(in_rag.ind >= 0, in_rag.w + 0.15, 0.0)
    rec_rag = synth.random_ragged(5, N, N, 0.4, no_autapse=True)
    rec_rag.w[:] = 0.0
    rng = np.random.default_rng(8)
    W_out = rng.normal(0, 0.5, (K, N))
    b = rng.normal(0, 0.1, K)
    net = _net(n_in, N, K, in_rag, rec_rag, W_out, b, p)
    thr = synth.rates_to_thresholds(rng.uniform(50, 250, (K, 1, n_in)), 1.0)
    label = 1
    r = oc.forward_trial(net, thr, label, T, 3, 77, T)
    assert r["z"].sum() > 10 and (r["psi"] > 0).sum() > 50
    G_in, G_rec, G_out, G_b = oc.eprop_gradients(net, r["x"], r["z"], r["psi"], r["d"])

    Win_np, Min = _dense(in_rag, N)
    Wrec_np, Mrec = _dense(rec_rag, N)
    Win = torch.tensor(Win_np, requires_grad=True)
    Wrec = torch.tensor(Wrec_np, requires_grad=True)
    Wout = torch.tensor(W_out, requires_grad=True)
    bt = torch.tensor(b)
    X = torch.tensor(r["x"])
    v = torch.zeros(N, dtype=torch.float64)
    a = torch.zeros(N, dtype=torch.float64)
    z = torch.zeros(N, dtype=torch.float64)
    y = torch.zeros(K, dtype=torch.float64)
    xp = torch.zeros(n_in, dtype=torch.float64)
    loss = 0.0
    zs = []
    for t in range(T):
        I = Win @ xp + Wrec @ z
        y = p.alpha * y + Wout @ z + bt
        v = p.alpha * (v - z.detach() * p.v_thr) + I
        a = p.rho * a + z
        A = p.v_thr + p.beta * a
        z = _Spike.apply(v - A, p.v_thr)
        zs.append(z.detach().numpy())
        loss = loss - torch.log_softmax(y, 0)[label]
        xp = X[t]
    np.testing.assert_array_equal(np.array(zs), r["z"])
    loss.backward()

    def ragged_to_dense(G, rag):
        D = np.zeros((N, rag.P))
        for i in range(rag.P):
            for s in range(rag.row_len[i]):
                D[rag.ind[i, s], i] = G[i, s]
        return D

    for G, rag, Wt, M in ((G_in, in_rag, Win, Min), (G_rec, rec_rag, Wrec, Mrec)):
        ref = Wt.grad.numpy() * M
        got = ragged_to_dense(G, rag)
        assert np.abs(ref).max() > 1e-3
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(G_out, Wout.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_readout_bias_rule_closed_form():
    """No hidden spikes: y^t = b (1 - alpha^{t+1}) / (1 - alpha); the paper's bias rule
    is the sum over steps of softmax(y^t) - onehot."""
    n_in, N, K, T = 3, 4, 5, 40
    p = oc.lif_params()
    in_rag = synth.random_ragged(1, n_in, N, 0.5)
    in_rag.w[:] = 0.0
    rec_rag = synth.random_ragged(2, N, N, 0.5, no_autapse=True)
    b = np.array([0.3, -0.2, 0.1, 0.0, 0.5])
    net = _net(n_in, N, K, in_rag, rec_rag, np.ones((K, N)), b, p)
    thr = np.zeros((K, 1, n_in), dtype=np.uint64)
    r = oc.forward_trial(net, thr, 2, T, 0, 0, T)
    a = p.alpha
    Gb = np.zeros(K)
    for t in range(T):
        yt = b * (1 - a ** (t + 1)) / (1 - a)
        np.testing.assert_allclose(r["y"][t], yt, rtol=1e-12)
        e = np.exp(yt - yt.max())
        Gb += e / e.sum() - np.eye(K)[2]
    _, _, G_out, G_b = oc.eprop_gradients(net, r["x"], r["z"], r["psi"], r["d"])
    np.testing.assert_allclose(G_b, Gb, rtol=1e-12, atol=1e-14)
    assert np.all(G_out == 0)


def test_adam_equals_torch():
    rng = np.random.default_rng(2)
    w0 = rng.normal(size=50)
    w = torch.tensor(w0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-3)
    ow, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    b1t = b2t = 1.0
    for step in range(6):
        g = rng.normal(size=50) * (10.0 ** rng.uniform(-4, 1))
        w.grad = torch.tensor(g)
        opt.step()
        b1t *= 0.9
        b2t *= 0.999
        ow, m, v = oc.adam(ow, m, v, g, 1e-3, b1t, b2t)
    np.testing.assert_allclose(ow, w.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_adam_ragged_leaves_padding_untouched():
    """Only the synapses s < row_len take the Adam step (the padding slots are room for
    growth, Fig. 1): padding w, m, v come back bit for bit, live slots equal the dense
    Adam step (torch.optim.Adam is pinned separately)."""
    rng = np.random.default_rng(4)
    P, C = 6, 5
    row_len = np.array([0, 1, 5, 3, 2, 4], np.int32)
    w, m, v = rng.normal(size=(P, C)), rng.normal(size=(P, C)), rng.random((P, C))
    g = rng.normal(size=(P, C))
    w2, m2, v2 = oc.adam_ragged(w, m, v, g, row_len, 1e-3, 0.9 ** 3, 0.999 ** 3)
    wd, md, vd = oc.adam(w, m, v, g, 1e-3, 0.9 ** 3, 0.999 ** 3)
    live = np.arange(C)[None] < row_len[:, None]
    for got, dense, before in ((w2, wd, w), (m2, md, m), (v2, vd, v)):
        np.testing.assert_array_equal(got[~live], before[~live])
        np.testing.assert_array_equal(got[live], dense[live])
        assert not np.array_equal(dense[~live], before[~live])   # the dense step would have moved them


def test_l1_on_sign_by_hand():
    G = np.array([[1.0, 2.0, 9.0], [0.5, 7.0, 7.0]])
    row_len = np.array([2, 1])
    ind = np.array([[3, 0, -1], [33, -1, -1]])
    sign = np.zeros((2, 2), dtype=np.uint32)
    sign[0, 0] = 1 << 3
    sign[1, 1] = 1 << 1
    out = oc.l1_on_sign(G, row_len, ind, sign, 0.25)
    np.testing.assert_array_equal(out, [[1.25, 1.75, 9.0], [0.75, 7.0, 7.0]])


def test_poisson_input_counts_binomial():
    thr = synth.rates_to_thresholds(np.array([[[20.0, 100.0, 0.0]]]), 1.0)
    T = 20000
    counts = np.zeros(3)
    for t in range(T):
        counts += oc.poisson_input(thr, 0, T, 12, t, 99)
    for c, p in zip(counts, (0.02, 0.1, 0.0)):
        sd = math.sqrt(T * p * (1 - p))
        assert abs(c - T * p) <= 5 * sd + 1e-9


def test_poisson_time_warp_bins():
    rates = np.zeros((1, 4, 2))
    rates[0, 2, :] = 1000.0           # p = 1 in bin 2 only
    thr = synth.rates_to_thresholds(rates, 1.0)
    fired = [oc.poisson_input(thr, 0, 7, 0, t, 1).all() for t in range(40)]
    assert fired == [14 <= t < 21 for t in range(40)]


def test_eprop_synapse_vectorised_over_trials_equals_trace_form():
    """The per-synapse trace recursion vectorised over trials (used for full-size sampled
    parity) gives the same sums as eprop_gradients slot by slot."""
    n_in, N, K, T, B = 12, 9, 3, 60, 4
    p = oc.NeuronParams(tau_m=20.0, v_thr=0.6, beta=0.3, tau_a=100.0)
    in_rag = synth.random_ragged(4, n_in, N, 0.5, w_std=0.4)
    in_rag.w = np.where(in_rag.ind >= 0, in_rag.w + 0.15, 0.0)
    rec_rag = synth.random_ragged(5, N, N, 0.4, no_autapse=True, w_std=0.3)
    rng = np.random.default_rng(8)
    net = _net(n_in, N, K, in_rag, rec_rag, rng.normal(0, 0.5, (K, N)), np.zeros(K), p)
    thr = synth.rates_to_thresholds(rng.uniform(50, 250, (K, 1, n_in)), 1.0)
    recs = [oc.forward_trial(net, thr, b % K, T, b, 77, T) for b in range(B)]
    G_in = sum(oc.eprop_gradients(net, r["x"], r["z"], r["psi"], r["d"])[0] for r in recs)
    G_rec = sum(oc.eprop_gradients(net, r["x"], r["z"], r["psi"], r["d"])[1] for r in recs)
    for G, rag, key in ((G_in, in_rag, "x"), (G_rec, rec_rag, "z")):
        for i in range(rag.P):
            for s in range(rag.row_len[i]):
                j = rag.ind[i, s]
                pre = np.array([r[key][:, i] for r in recs])
                psi = np.array([r["psi"][:, j] for r in recs])
                L = np.array([r["d"] @ net.W_out[:, j] for r in recs])
                np.testing.assert_allclose(oc.eprop_synapse(pre, psi, L, p), G[i, s], rtol=1e-12, atol=1e-13)


def test_neuron_constants_match_paper():
    """NeuronParams' defaults are the printed constants; alpha, rho and psi's peak follow
    from them by the printed formulas (psi peaks at gain / v_thr where v = A, and is
    zero once |v - A| >= v_thr)."""
    import os
    tab = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "classifier_parameters.txt")
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            name, value = line.split(";", 1)[0].split()[:2]
            tab[name] = float(value)
    p = oc.NeuronParams()
    assert (p.tau_m, p.v_thr, p.tau_a, p.beta, p.dt) == (tab["tau_mem"], tab["v_thr"], tab["tau_adapt"],
                                                        tab["beta"], tab["dt"])
    assert p.alpha == pytest.approx(math.exp(-1.0 / 20.0), rel=1e-15)
    assert p.rho == pytest.approx(math.exp(-1.0 / 2000.0), rel=1e-15)
    # z_prev = 0, v_prev = 0: v = I; a_prev = 2 / rho: a = 2, A = v_thr + 2 beta
    A = p.v_thr + 2.0 * p.beta
    I = np.array([A, A + 0.5 * p.v_thr, A - p.v_thr, A + 2 * p.v_thr, A - 1e-9])
    v, a, z, psi, A_out = oc.neuron_step(np.zeros(5), np.full(5, 2.0 / p.rho), np.zeros(5), I, p)
    np.testing.assert_allclose(a, 2.0, rtol=1e-15)
    np.testing.assert_allclose(A_out, 0.6 + 2 * 0.0174, rtol=1e-15)
    # peak gain / v_thr = 0.3 / 0.6 at v = A, half of it halfway out, zero at the edges
    np.testing.assert_allclose(psi[:4], [0.5, 0.25, 0.0, 0.0], atol=1e-12)
    assert tab["psi_gain"] / tab["v_thr"] == pytest.approx(0.5)
    np.testing.assert_array_equal(z, [1, 1, 0, 1, 0])
