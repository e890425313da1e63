"""Checkpoint / resume: the whole training state is plain arrays (ragged rows, weights,
Adam moments, DEEP R bitfields, readout and its moments) and every random number is a
counter-based Philox draw, so saving the arrays after k batches, rebuilding the handles
from them in a fresh classifier and training on gives bit-for-bit the run that never
stopped."""
import numpy as np
import pytest
import torch

import synth
from tests import _setups

pytestmark = pytest.mark.gpu

F32 = 0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _train(dev, task, first, last, B, T, lr=1e-3, l1=1e-5):
    from paper_2510_19764_gb300 import net
    tb = synth.trial_batch(task, 5, first, B)
    batch = net.DeviceBatch(dev, tb.labels, tb.bin_len, tb.trial_ids, T)
    for i in range(first, last):
        tb = synth.trial_batch(task, 5, i, B)
        batch.set_trials(tb.labels, tb.bin_len, tb.trial_ids)
        for t_ in (batch.v, batch.a, batch.y, batch.ysum, batch.x_bits, batch.z_bits):
            t_.zero_()
        net.train_batch(dev, batch, net.adam_params(lr, i + 1, l1=l1), i)
    torch.cuda.synchronize()


def _state(dev):
    out = {}
    for name, r in (("in", dev.w_in), ("rec", dev.w_rec)):
        for k, v in r.host().items():
            out[f"{name}.{k}"] = v
    for k in ("W_out", "b_out", "W_out_m", "W_out_v", "b_m", "b_v"):
        out[k] = getattr(dev, k).cpu().numpy().copy()
    return out


def test_save_reload_continue_equals_straight_run():
    from paper_2510_19764_gb300 import net
    T, B, n_in, N, K = 150, 4, 48, 96, 4
    kw = dict(seed=7, dtype=F32, lif=False, v_thr=0.6, T=T, max_B=B, n_in=n_in, N=N, K=K, n_classes=K, n_bins=3,
              spoken=True, p_in=0.2, p_rec=0.15, w_scale=1.5)
    straight = _setups.classifier(**kw)
    _train(straight.dev, straight.task, 0, 6, B, T)
    ref = _state(straight.dev)

    first = _setups.classifier(**kw)
    _train(first.dev, first.task, 0, 3, B, T)
    saved = _state(first.dev)
    del first

    # a fresh classifier built from the saved arrays only
    s = _setups.classifier(**kw)
    d = s.dev
    for name in ("in", "rec"):
        old = getattr(d, "w_in" if name == "in" else "w_rec")
        new = net.DeviceRagged(saved[f"{name}.row_len"], saved[f"{name}.ind"], saved[f"{name}.w"], old.Q,
                               dtype=old.dtype, no_autapse=name == "rec", adam=True, grad=True, deepr=True,
                               seed=old.desc.seed, m=saved[f"{name}.m"], v=saved[f"{name}.v"],
                               sign_bits=saved[f"{name}.sign_bits"])
        setattr(d, "w_in" if name == "in" else "w_rec", new)
    resumed = net.DeviceClassifier(n_in, N, K, d.w_in, d.w_rec, saved["W_out"], saved["b_out"], s.task.thr,
                                   s.in_seed, net.NeuronCfg(tau_m=20.0, v_thr=0.6, beta=0.0174, tau_a=2000.0),
                                   max_B=B, max_T=T, dtype=F32)
    for k in ("W_out_m", "W_out_v", "b_m", "b_v"):
        getattr(resumed, k).copy_(torch.from_numpy(saved[k]).cuda())
    _train(resumed, s.task, 3, 6, B, T)
    got = _state(resumed)
    assert set(got) == set(ref)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert ref["rec.row_len"].sum() > 0
