"""Batched scheduler: the CUDA-graph form over many uneven instances gives bit-identical
results to the plain one-instance-at-a-time form with per-step launches; the autotuner
fills its table with admissible schedules."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()


def _instances(specs, temperature=0.0):
    from paper_2510_19764_gb300 import sched
    task = synth.spoken_digit_task(3, n_in=sched.N_IN, n_classes=sched.N_CLASSES, T=1000, n_bins=sched.N_BINS)
    return [sched.Instance(s, task, temperature=temperature) for s in specs]


@pytest.mark.parametrize("temperature", [0.0, 1e-4])
def test_batched_graph_equals_plain_per_step(temperature):
    """Also with DEEP R's noise term, whose Philox counter the captured graph reads from
    the instance's device iteration counter."""
    from paper_2510_19764_gb300 import sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in
             enumerate([(64, 37, 0.2), (128, 80, 0.1), (256, 55, 0.05), (96, 64, 0.15), (300, 41, 0.1)])]
    plain = _instances(specs, temperature)
    pr = sched.PlainRunner(plain)
    for _ in range(3):
        pr.iterate()
    torch.cuda.synchronize()
    batched = _instances(specs, temperature)
    br = sched.BatchedRunner(batched, n_streams=3)
    br.capture()
    for _ in range(3):
        br.iterate()
    torch.cuda.synchronize()
    rewired = 0
    for a, b in zip(plain, batched):
        sa, sb = a.snapshot(), b.snapshot()
        for proj in ("in", "rec"):
            np.testing.assert_array_equal(sa[proj]["row_len"], sb[proj]["row_len"])
            mask = np.arange(sa[proj]["ind"].shape[1])[None] < sa[proj]["row_len"][:, None]
            np.testing.assert_array_equal(sa[proj]["ind"][mask], sb[proj]["ind"][mask])
            np.testing.assert_array_equal(sa[proj]["w"][mask], sb[proj]["w"][mask])
            np.testing.assert_array_equal(sa[proj]["conn_bits"], sb[proj]["conn_bits"])
        np.testing.assert_array_equal(sa["W_out"], sb["W_out"])
        np.testing.assert_array_equal(sa["ysum"], sb["ysum"])
        assert int(a.step.item()) == int(b.step.item()) == 3
        rewired += int(b.stats[:, 0].sum().item())
        assert a.d_in.status() == 0 and a.d_rec.status() == 0
    assert rewired > 0
    if temperature > 0:
        # the noise is there: a noiseless run of the first instance ends elsewhere
        quiet = _instances(specs[:1])
        qr = sched.PlainRunner(quiet)
        for _ in range(3):
            qr.iterate()
        torch.cuda.synchronize()
        assert not np.array_equal(quiet[0].snapshot()["in"]["w"], plain[0].snapshot()["in"]["w"])


def test_autotuner_picks_admissible_schedules():
    from paper_2510_19764_gb300 import sched
    specs = [sched.InstanceSpec(N, 60, 0.1, i) for i, N in enumerate([128, 512, 2048])]
    insts = _instances(specs)
    tuner = sched.Autotuner()
    table = tuner.tune(insts)
    assert len(table) >= 3
    for k, w in table.items():
        assert w in (4, 8, 16) and k[0] <= 8 * 32 * w
        assert all(t > 0 for t in tuner.timings[k].values())
