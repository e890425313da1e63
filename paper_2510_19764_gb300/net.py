"""Device-memory plumbing around the C ABI: torch tensors hold every array the library
reads or writes, and these classes fill the descriptor structs.  No arithmetic of the
method happens here; every step runs in libsnnsp.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import abi

_DT = {abi.SNN_F32: torch.float32, abi.SNN_F64: torch.float64}


def _tdtype(dtype: int) -> torch.dtype:
    return _DT[dtype]


def words(n: int) -> int:
    return (n + 31) // 32


def _u64_tensor(a: np.ndarray, device) -> torch.Tensor:
    """uint64 host array -> int64 device tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def _u32_tensor(a: np.ndarray, device) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)


def u32_to_numpy(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def u64_to_numpy(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


class DeviceRagged:
    """A ragged matrix in device memory plus its library handle."""

    def __init__(self, row_len, ind, w, Q: int, dtype: int = abi.SNN_F32, no_autapse: bool = False,
                 adam: bool = False, grad: bool = False, deepr: bool = False, seed: int = 0, device="cuda",
                 stream=None, m=None, v=None, sign_bits=None):
        P, C = np.shape(ind)
        self.P, self.Q, self.C, self.dtype = P, Q, C, dtype
        td = _tdtype(dtype)
        self.row_len = torch.as_tensor(np.asarray(row_len, np.int32), device=device).contiguous()
        self.ind = torch.as_tensor(np.where(np.asarray(ind) >= 0, ind, 0).astype(np.int32), device=device).contiguous()
        self.w = torch.as_tensor(np.asarray(w, np.float64), dtype=td, device=device).contiguous()
        self.m = self.v = self.grad = self.sign_bits = self.conn_bits = None
        if adam:
            self.m = torch.zeros((P, C), dtype=td, device=device) if m is None else \
                torch.as_tensor(np.asarray(m), dtype=td, device=device).contiguous()
            self.v = torch.zeros((P, C), dtype=td, device=device) if v is None else \
                torch.as_tensor(np.asarray(v), dtype=td, device=device).contiguous()
        if grad:
            self.grad = torch.zeros((P, C), dtype=td, device=device)
        if deepr:
            self.sign_bits = torch.zeros((P, words(Q)), dtype=torch.int32, device=device)
            self.conn_bits = torch.zeros((P, words(Q)), dtype=torch.int32, device=device)
        d = abi.RaggedDesc()
        d.P, d.Q, d.C, d.dtype, d.no_autapse, d.reserved = P, Q, C, dtype, int(no_autapse), 0
        d.row_len, d.ind, d.w = abi.ptr(self.row_len), abi.ptr(self.ind), abi.ptr(self.w)
        d.m, d.v, d.grad = abi.ptr(self.m), abi.ptr(self.v), abi.ptr(self.grad)
        d.sign_bits, d.conn_bits = abi.ptr(self.sign_bits), abi.ptr(self.conn_bits)
        d.seed = seed
        self.desc = d
        self.handle = abi.snn_create_ragged(d, deepr, stream)
        if sign_bits is not None:
            # scripted sign bits (tests): replace the drawn ones after the library's init
            self.sign_bits.copy_(_u32_tensor(sign_bits, device))

    def host(self) -> dict:
        out = {"row_len": self.row_len.cpu().numpy(), "ind": self.ind.cpu().numpy(),
               "w": self.w.double().cpu().numpy()}
        for k in ("m", "v", "grad"):
            t = getattr(self, k)
            if t is not None:
                out[k] = t.double().cpu().numpy()
        if self.sign_bits is not None:
            out["sign_bits"] = u32_to_numpy(self.sign_bits)
            out["conn_bits"] = u32_to_numpy(self.conn_bits)
        return out

    def status(self, stream=None) -> int:
        return abi.snn_ragged_status(self.handle, stream)

    def close(self):
        if self.handle:
            abi.snn_destroy_ragged(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class NeuronCfg:
    tau_m: float = 20.0
    v_thr: float = 0.6
    beta: float = 0.0174
    tau_a: float = 2000.0     # <= 0: LIF
    dt: float = 1.0


class DeviceClassifier:
    """Readout weights, Adam moments, gradients and the classifier handle."""

    def __init__(self, n_in: int, N: int, K: int, w_in: DeviceRagged, w_rec: DeviceRagged, W_out, b_out,
                 in_thr: np.ndarray, in_seed: int, neuron: NeuronCfg, max_B: int, max_T: int,
                 dtype: int = abi.SNN_F32, device="cuda"):
        td = _tdtype(dtype)
        self.n_in, self.N, self.K, self.dtype = n_in, N, K, dtype
        self.w_in, self.w_rec = w_in, w_rec
        self.W_out = torch.as_tensor(np.asarray(W_out, np.float64), dtype=td, device=device).contiguous()
        self.b_out = torch.as_tensor(np.asarray(b_out, np.float64), dtype=td, device=device).contiguous()
        self.W_out_m = torch.zeros_like(self.W_out)
        self.W_out_v = torch.zeros_like(self.W_out)
        self.b_m = torch.zeros_like(self.b_out)
        self.b_v = torch.zeros_like(self.b_out)
        self.G_out = torch.zeros_like(self.W_out)
        self.G_b = torch.zeros_like(self.b_out)
        self.in_thr = _u32_tensor(in_thr, device)
        n_classes, n_bins, _ = in_thr.shape
        d = abi.ClassifierDesc()
        d.n_in, d.N, d.K, d.dtype = n_in, N, K, dtype
        d.tau_m, d.v_thr, d.beta, d.tau_a, d.dt = neuron.tau_m, neuron.v_thr, neuron.beta, neuron.tau_a, neuron.dt
        d.n_classes, d.n_bins = n_classes, n_bins
        d.in_thr, d.in_seed = abi.ptr(self.in_thr), in_seed
        d.w_in, d.w_rec = w_in.handle, w_rec.handle
        d.W_out, d.b_out = abi.ptr(self.W_out), abi.ptr(self.b_out)
        d.W_out_m, d.W_out_v, d.b_m, d.b_v = (abi.ptr(self.W_out_m), abi.ptr(self.W_out_v), abi.ptr(self.b_m),
                                              abi.ptr(self.b_v))
        d.G_out, d.G_b = abi.ptr(self.G_out), abi.ptr(self.G_b)
        d.max_B, d.max_T = max_B, max_T
        self.desc = d
        self.handle = abi.snn_create_classifier(d)

    def close(self):
        if self.handle:
            abi.snn_destroy_classifier(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceBatch:
    """State, records and workspace of one batch of trials."""

    def __init__(self, cls: DeviceClassifier, labels, bin_len, trial_ids, T: int, record_state: bool = False,
                 device="cuda", workspace: bool = True, records: bool = True, trial_T=None):
        B = len(labels)
        N, K, n_in = cls.N, cls.K, cls.n_in
        td = _tdtype(cls.dtype)
        Kp = (K + 3) // 4 * 4
        self.B, self.T = B, T
        self.labels = torch.as_tensor(np.asarray(labels, np.int32), device=device)
        self.bin_len = torch.as_tensor(np.asarray(bin_len, np.int32), device=device)
        self.trial_ids = torch.as_tensor(np.asarray(trial_ids, np.int64), device=device)
        z = lambda *s, dt=td: torch.zeros(s, dtype=dt, device=device)  # noqa: E731
        self.v, self.a, self.y, self.ysum = z(B, N), z(B, N), z(B, K), z(B, K)
        self.x_bits = z(B, words(n_in), dt=torch.int32)
        self.z_bits = z(B, words(N), dt=torch.int32)
        self.x_rec = z(B, T, words(n_in), dt=torch.int32)
        self.z_rec = z(B, T, words(N), dt=torch.int32)
        self.psi_rec = torch.empty((B, T, N), dtype=td, device=device) if records else None
        self.d_rec = torch.empty((B, T, K), dtype=td, device=device) if records else None
        self.trial_T = None if trial_T is None else torch.as_tensor(np.asarray(trial_T, np.int32), device=device)
        self.v_rec = self.a_rec = self.y_rec = None
        if record_state:
            self.v_rec = torch.empty((B, T, N), dtype=td, device=device)
            self.a_rec = torch.empty((B, T, N), dtype=td, device=device)
            self.y_rec = torch.empty((B, T, K), dtype=td, device=device)
        self.delta = torch.empty((B, T, N), dtype=td, device=device) if workspace else None
        self.Dout = torch.empty((B, T, Kp), dtype=td, device=device) if workspace else None
        b = abi.Batch()
        b.B, b.T = B, T
        for name in ("labels", "bin_len", "trial_ids", "v", "a", "y", "x_bits", "z_bits", "x_rec", "z_rec",
                     "psi_rec", "d_rec", "ysum", "v_rec", "a_rec", "y_rec", "delta", "Dout", "trial_T"):
            setattr(b, name, abi.ptr(getattr(self, name)))
        self.desc = b

    def reset_state(self):
        for t in (self.v, self.a, self.y, self.ysum, self.x_bits, self.z_bits):
            t.zero_()

    def set_trials(self, labels, bin_len, trial_ids):
        """Refill the per-trial inputs in place (same B) and zero the state."""
        self.labels.copy_(torch.as_tensor(np.asarray(labels, np.int32)))
        self.bin_len.copy_(torch.as_tensor(np.asarray(bin_len, np.int32)))
        self.trial_ids.copy_(torch.as_tensor(np.asarray(trial_ids, np.int64)))
        self.reset_state()


def spikes_from_bits(bits: np.ndarray, n: int) -> np.ndarray:
    """[..., W] uint32 words -> [..., n] 0/1 array (bit j of word j >> 5)."""
    b = np.asarray(bits).view(np.uint32)
    out = ((b[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return out.reshape(*b.shape[:-1], -1)[..., :n]


def adam_params(lr: float, step: int, l1: float = 0.0, beta1: float = 0.9, beta2: float = 0.999,
                eps: float = 1e-8, step_dev=None, temperature: float = 0.0, noise_idx: int | None = None,
                noise_idx_dev=None) -> abi.Adam:
    """Adam hyper-parameters for the step-th update (the library forms the bias
    corrections); step_dev (device int64 holding the step count) makes the kernels read
    it from device memory.  temperature > 0 turns on the DEEP R noise term with Philox
    counter noise_idx (default: step - 1) or, if given, the device int64 noise_idx_dev."""
    a = abi.Adam()
    a.lr, a.beta1, a.beta2, a.eps, a.l1 = lr, beta1, beta2, eps, l1
    a.step = step
    a.step_dev = abi.ptr(step_dev)
    a.temperature = temperature
    a.noise_idx = step - 1 if noise_idx is None else noise_idx
    a.noise_idx_dev = abi.ptr(noise_idx_dev)
    return a


def train_batch(cls: DeviceClassifier, batch: DeviceBatch, adam: abi.Adam, rewire_idx: int,
                stats_in=None, stats_rec=None, stream=None, deepr: bool = True) -> None:
    """One e-prop + DEEP R training batch: all T steps of every trial in one launch,
    the gradient, L1 + Adam, then DEEP R on both sparse projections."""
    abi.snn_step_neurons(cls.handle, batch.desc, 0, batch.T, stream)
    abi.snn_eprop_update(cls.handle, batch.desc, abi.SNN_EPROP_GRAD, None, stream)
    abi.snn_eprop_update(cls.handle, batch.desc, abi.SNN_EPROP_APPLY, adam, stream)
    if deepr:
        abi.snn_rewire_deepr(cls.w_in.handle, rewire_idx, stats_in, stream)
        abi.snn_rewire_deepr(cls.w_rec.handle, rewire_idx, stats_rec, stream)


# ------------------------------------------------------------------ topographic map

def topo_params(L: int = 32, L_f: int | None = None, radius: int = 3, t_stim: int = 20, dt: float = 1.0,
                tau_m=20.0, V_rest=-70.0, E_exc=0.0, V_theta=-54.0, V_reset=-70.0, tau_ref=5.0, tau_s=5.0,
                g_leak=1.0, f_base=20.0, f_in=100.0, g_max=0.2, tau_plus=20.0, tau_minus=64.0,
                B_ratio=1.2, A_plus_rel=0.1, sigma_stim: float = 0.0) -> abi.TopoParams:
    """Topographic-map parameters (Tab. 1-2).  t_stim is in steps; sigma_stim > 0 selects
    the Gaussian input profile (f_in then is the peak rate), 0 the disc of `radius`."""
    p = abi.TopoParams()
    p.L, p.L_f, p.radius2, p.t_stim = L, L_f or L, radius * radius, t_stim
    p.dt, p.tau_m, p.V_rest, p.E_exc, p.V_theta, p.V_reset = dt, tau_m, V_rest, E_exc, V_theta, V_reset
    p.tau_s, p.g_leak, p.tau_ref, p.f_base, p.f_in, p.g_max = tau_s, g_leak, tau_ref, f_base, f_in, g_max
    p.tau_plus, p.tau_minus, p.A_plus_rel, p.B = tau_plus, tau_minus, A_plus_rel, B_ratio
    p.sigma_stim = sigma_stim
    return p


def topo_rewire(L: int, p_form: float, sigma: float, n_att: int, g_max: float = 0.2,
                p_elim_dep: float = 2.45e-2 * 50, p_elim_pot: float = 1.36e-4 * 50) -> abi.TopoRewire:
    r = abi.TopoRewire()
    r.p_form, r.sigma, r.p_elim_dep, r.p_elim_pot = p_form, sigma, p_elim_dep, p_elim_pot
    r.g_max, r.L, r.n_att = g_max, L, n_att
    return r


def attach_event_histograms(rw: abi.TopoRewire, L: int, device="cuda"):
    """Zeroed elimination / formation histograms (int64, bins = squared torus distance
    0 .. 2 (L/2)^2) that the rewiring with parameters `rw` adds to; the caller keeps
    the returned tensors alive while `rw` is in use."""
    n = 2 * (L // 2) ** 2 + 1
    elim = torch.zeros(n, dtype=torch.int64, device=device)
    form = torch.zeros(n, dtype=torch.int64, device=device)
    rw.elim_d2, rw.form_d2 = abi.ptr(elim), abi.ptr(form)
    return elim, form


def topo_connectivity(r: "DeviceRagged", L: int, stream=None):
    """(count [L*L] int64, wsum [L*L] float64, in_degree [L*L] int32) by torus
    displacement dy*L + dx of a topographic projection, on the device."""
    dev = r.row_len.device
    count = torch.empty(L * L, dtype=torch.int64, device=dev)
    wsum = torch.empty(L * L, dtype=torch.float64, device=dev)
    indeg = torch.empty(L * L, dtype=torch.int32, device=dev)
    abi.snn_topo_connectivity(r.handle, L, count, wsum, indeg, stream)
    return count, wsum, indeg


class DeviceTopoState:
    def __init__(self, N: int, V_rest: float, device="cuda"):
        f = lambda: torch.zeros(N, dtype=torch.float32, device=device)  # noqa: E731
        self.V = torch.full((N,), V_rest, dtype=torch.float32, device=device)
        self.gs, self.x_src, self.x_tgt, self.y, self.ydec = f(), f(), f(), f(), f()
        self.ref = torch.zeros(N, dtype=torch.int32, device=device)
        self.src_bits = torch.zeros((2, words(N)), dtype=torch.int32, device=device)
        self.tgt_bits = torch.zeros((2, words(N)), dtype=torch.int32, device=device)
        self.acc = torch.zeros(N, dtype=torch.int64, device=device)
        s = abi.TopoState()
        for name in ("V", "gs", "ref", "x_src", "x_tgt", "y", "ydec", "src_bits", "tgt_bits", "acc"):
            setattr(s, name, abi.ptr(getattr(self, name)))
        self.desc = s
