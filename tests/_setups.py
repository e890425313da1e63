"""Matched oracle / CUDA setups for the parity tests (seeded synthetic inputs)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import synth
from oracle import classifier as oc
from oracle import deepr as od


@dataclass
class ClsSetup:
    task: synth.ClassifierTask
    onet: oc.ClassifierNet
    dev: object            # net.DeviceClassifier
    in_rag: synth.Ragged
    rec_rag: synth.Ragged
    in_seed: int
    dtype: int


def as_dtype(x, dtype):
    """Round to the device dtype and back, so both sides start from identical values."""
    from paper_2510_19764_gb300 import abi
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64) if dtype == abi.SNN_F32 \
        else np.asarray(x, np.float64)


def classifier(seed=0, n_in=32, N=64, K=4, p_in=0.1, p_rec=0.1, lif=True, v_thr=1.0, T=200, n_classes=4,
               n_bins=1, dtype=None, max_B=8, rate_hz=40.0, w_scale=1.0, deepr_seed=None, C_in=None, C_rec=None,
               spoken=False):
    from paper_2510_19764_gb300 import abi, net
    dtype = abi.SNN_F32 if dtype is None else dtype
    if spoken:
        task = synth.spoken_digit_task(seed, n_in=n_in, n_classes=n_classes, T=T, n_bins=n_bins)
    else:
        task = synth.tiny_task(seed, n_in=n_in, n_classes=n_classes, T=T, max_rate_hz=rate_hz)
    in_rag = synth.random_ragged(seed + 1, n_in, N, p_in, C=C_in)
    rec_rag = synth.random_ragged(seed + 2, N, N, p_rec, no_autapse=True, C=C_rec)
    in_rag.w = as_dtype(in_rag.w * w_scale, dtype)
    rec_rag.w = as_dtype(rec_rag.w * w_scale, dtype)
    W_out, b = synth.dense_readout(seed + 3, K, N)
    W_out = as_dtype(W_out, dtype)
    b = as_dtype(b, dtype)
    if lif:
        npar = oc.lif_params(v_thr=v_thr)
        ncfg = net.NeuronCfg(tau_m=20.0, v_thr=v_thr, beta=0.0, tau_a=-1.0)
    else:
        npar = oc.NeuronParams(tau_m=20.0, v_thr=v_thr, beta=0.0174, tau_a=2000.0)
        ncfg = net.NeuronCfg(tau_m=20.0, v_thr=v_thr, beta=0.0174, tau_a=2000.0)
    onet = oc.ClassifierNet(n_in, N, K, in_rag.row_len, in_rag.ind, in_rag.w, rec_rag.row_len, rec_rag.ind,
                            rec_rag.w, W_out, b, npar)
    ds = seed + 100 if deepr_seed is None else deepr_seed
    d_in = net.DeviceRagged(in_rag.row_len, in_rag.ind, in_rag.w, N, dtype=dtype, adam=True, grad=True, deepr=True,
                            seed=ds)
    d_rec = net.DeviceRagged(rec_rag.row_len, rec_rag.ind, rec_rag.w, N, dtype=dtype, no_autapse=True, adam=True,
                             grad=True, deepr=True, seed=ds + 1)
    in_seed = seed + 7
    dev = net.DeviceClassifier(n_in, N, K, d_in, d_rec, W_out, b, task.thr, in_seed, ncfg, max_B=max_B, max_T=T,
                               dtype=dtype)
    return ClsSetup(task, onet, dev, in_rag, rec_rag, in_seed, dtype)


def oracle_bitfields(rag: synth.Ragged, Q: int, seed: int):
    return od.init_bitfields(rag.row_len, rag.ind, rag.w, Q, seed)


_POOL = None


def oracle_pool(n: int = 8):
    """Process pool for oracle trials (spawned processes: they never touch the GPU)."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        import os
        _POOL = mp.get_context("spawn").Pool(max(1, min(n, (os.cpu_count() or 2) - 1)))
    return _POOL


def oracle_trial(args):
    """Pool worker: one trial's forward and e-prop gradients in the oracle.  args =
    (ClassifierNet constructor arrays, neuron params, thresholds, label, bin_len,
    trial id, input seed, T).  Returns (z raster uint8 [T, N], prediction, ysum,
    (G_in, G_rec, G_out, G_b))."""
    arrays, neuron, thr, label, bin_len, trial_id, seed, T = args
    net = oc.ClassifierNet(*arrays, neuron)
    r = oc.forward_trial(net, thr, label, bin_len, trial_id, seed, T)
    g = oc.eprop_gradients(net, r["x"], r["z"], r["psi"], r["d"])
    return r["z"].astype(np.uint8), r["pred"], r["ysum"], g


def oracle_grad_from_records(args):
    """Pool worker: the oracle's e-prop gradients (forward-trace form) of one trial from
    given records.  args = (ClassifierNet constructor arrays, neuron params, x [T, n_in],
    z [T, N], psi [T, N], d [T, K]).  Returns (G_in, G_rec, G_out, G_b)."""
    arrays, neuron, x, z, psi, d = args
    net = oc.ClassifierNet(*arrays, neuron)
    return oc.eprop_gradients(net, x, z, psi, d)
