"""Batched forms over many uneven instances give bit-identical results to the plain
one-instance-at-a-time form: the CUDA graph of per-call launches, and the persistent
multi-instance kernel (one launch per iteration, also captured in a graph, also fed by a
host producer through its mailbox).  A bounded wait of the persistent kernel that nothing
satisfies gives up with SNN_ETIMEOUT and leaves the instances untouched.  The autotuner
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


def _instances(specs, temperature=0.0, modes=None):
    from paper_2510_19764_gb300 import abi, sched
    task = synth.spoken_digit_task(3, n_in=sched.N_IN, n_classes=sched.N_CLASSES, T=1000, n_bins=sched.N_BINS)
    out = [sched.Instance(s, task, temperature=temperature) for s in specs]
    for inst, mode in zip(out, modes or []):
        abi.snn_classifier_set_row_schedule(inst.cls.handle, mode)
    return out


def _assert_same(plain, other, iters):
    rewired = 0
    for a, b in zip(plain, other):
        sa, sb = a.snapshot(), b.snapshot()
        for proj in ("in", "rec"):
            np.testing.assert_array_equal(sa[proj]["row_len"], sb[proj]["row_len"])
            mask = np.arange(sa[proj]["ind"].shape[1])[None] < sa[proj]["row_len"][:, None]
            np.testing.assert_array_equal(sa[proj]["ind"][mask], sb[proj]["ind"][mask])
            np.testing.assert_array_equal(sa[proj]["w"][mask], sb[proj]["w"][mask])
            np.testing.assert_array_equal(sa[proj]["conn_bits"], sb[proj]["conn_bits"])
        np.testing.assert_array_equal(sa["W_out"], sb["W_out"])
        np.testing.assert_array_equal(sa["ysum"], sb["ysum"])
        assert int(a.step.item()) == int(b.step.item()) == iters
        assert torch.equal(a.stats, b.stats)
        rewired += int(b.stats[:, 0].sum().item())
        for inst in (a, b):
            assert inst.d_in.status() == 0 and inst.d_rec.status() == 0
    assert rewired > 0


SPECS = [(64, 37, 0.2), (128, 80, 0.1), (256, 55, 0.05), (96, 64, 0.15), (300, 41, 0.1)]


@pytest.mark.parametrize("temperature", [0.0, 1e-4])
def test_batched_graph_equals_plain_per_step(temperature):
    """Also with DEEP R's noise term, whose Philox counter the captured graph reads from
    the instance's device iteration counter."""
    from paper_2510_19764_gb300 import sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in enumerate(SPECS)]
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
    _assert_same(plain, batched, 3)
    if temperature > 0:
        # the noise is there: a noiseless run of the first instance ends elsewhere
        quiet = _instances(specs[:1])
        qr = sched.PlainRunner(quiet)
        for _ in range(3):
            qr.iterate()
        torch.cuda.synchronize()
        assert not np.array_equal(quiet[0].snapshot()["in"]["w"], plain[0].snapshot()["in"]["w"])


@pytest.mark.parametrize("temperature", [0.0, 1e-4])
def test_persistent_kernel_equals_plain_whole_trial(temperature):
    """Uneven instances (hidden 64 .. 2048, 37 .. 300 steps, 5-20 %, each of the three
    row schedules): three iterations of the persistent kernel (two of them replayed
    from one captured graph) equal three plain iterations bit for bit."""
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in
             enumerate(SPECS + [(2048, 300, 0.2), (512, 200, 0.1), (1024, 120, 0.05)])]
    modes = [i % 3 for i in range(len(specs))]
    plain = _instances(specs, temperature, modes)
    pr = sched.PlainRunner(plain, per_step=False)
    for _ in range(3):
        pr.iterate()
    torch.cuda.synchronize()
    multi = _instances(specs, temperature, modes)
    mr = sched.MultiRunner(multi)
    mr.iterate()
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_OK
    mr.capture(2)
    mr.replay()
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_OK
    _assert_same(plain, multi, 3)


def test_persistent_kernel_fed_by_a_host_producer():
    """With SNN_MULTI_HOST_POSTS the kernel trains the instances the host posts while it
    runs: all of them (equal to the self-seeded run), then a subset (only those advance)."""
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in enumerate(SPECS)]
    ref = _instances(specs)
    rr = sched.MultiRunner(ref)
    rr.iterate()
    torch.cuda.synchronize()
    fed = _instances(specs)
    fr = sched.MultiRunner(fed)
    s = torch.cuda.Stream()
    fr.iterate(stream=s, flags=abi.SNN_MULTI_HOST_POSTS)
    abi.snn_multi_post(fr.handle, [4, 2, 0, 1, 3])
    s.synchronize()
    assert fr.status(s) == abi.SNN_OK
    _assert_same(ref, fed, 1)
    before = [i.snapshot() for i in fed]
    fr.iterate(stream=s, flags=abi.SNN_MULTI_HOST_POSTS)
    abi.snn_multi_post(fr.handle, [3])
    s.synchronize()
    assert fr.status(s) == abi.SNN_OK
    assert [int(i.step.item()) for i in fed] == [1, 1, 1, 2, 1]
    for k, inst in enumerate(fed):
        if k != 3:
            np.testing.assert_array_equal(inst.snapshot()["in"]["w"], before[k]["in"]["w"])
    assert not np.array_equal(fed[3].snapshot()["in"]["w"], before[3]["in"]["w"])


def test_persistent_kernel_wait_gives_up_when_nothing_is_posted():
    """A host producer that never posts: the kernel's bounded mailbox wait gives up after
    its limit, every CTA leaves, snn_multi_status reports SNN_ETIMEOUT, no instance has
    moved, and the next (self-seeded) run of the same plan is correct."""
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in enumerate(SPECS[:3])]
    multi = _instances(specs)
    mr = sched.MultiRunner(multi, wait_limit_ns=50_000_000)
    before = [i.snapshot() for i in multi]
    mr.iterate(flags=abi.SNN_MULTI_HOST_POSTS)
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_ETIMEOUT
    for inst, b in zip(multi, before):
        assert int(inst.step.item()) == 0
        np.testing.assert_array_equal(inst.snapshot()["in"]["w"], b["in"]["w"])
    mr.iterate()
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_OK
    plain = _instances(specs)
    sched.PlainRunner(plain, per_step=False).iterate()
    torch.cuda.synchronize()
    _assert_same(plain, multi, 1)


def test_autotuner_for_the_persistent_kernel_and_wide_schedules():
    """The persistent kernel's autotuner times one-instance runs for every row schedule
    (wide ones included); whatever it picks, the results stay those of the plain path."""
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in enumerate([(2048, 60, 0.2), (256, 50, 0.05)])]
    tuned = _instances(specs)
    tuner = sched.Autotuner(target="multi")
    table = tuner.tune(tuned)
    assert all(len(v) == len(sched.Autotuner.MULTI_MODES) for v in tuner.timings.values())
    assert all(mode in sched.Autotuner.MULTI_MODES for _, mode in table.values())
    # each wide schedule on its own: persistent equals plain
    for mode in (abi.SNN_ROWS_WIDE, abi.SNN_ROWS_QUAD):
        plain = _instances(specs, modes=[mode, mode])
        pr = sched.PlainRunner(plain, per_step=False)
        pr.iterate()
        multi = _instances(specs, modes=[mode, mode])
        sched.MultiRunner(multi).iterate()
        torch.cuda.synchronize()
        _assert_same(plain, multi, 1)


def test_autotuner_picks_admissible_schedules():
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, 60, 0.1, i) for i, N in enumerate([128, 512, 2048])]
    insts = _instances(specs)
    tuner = sched.Autotuner()
    table = tuner.tune(insts)
    assert len(table) >= 3
    for k, (w, mode) in table.items():
        assert w in (4, 8, 16) and k[0] <= 8 * 32 * w
        assert mode in (abi.SNN_ROWS_PAIRS, abi.SNN_ROWS_PER_WARP, abi.SNN_ROWS_PER_BLOCK)
        assert all(t > 0 for t in tuner.timings[k].values())


def test_persistent_kernel_phase_trace():
    """Tracing: with a trace buffer set, a run stamps every instance's start and the end
    of each of its phases, in phase order; clearing it stops the stamping."""
    from paper_2510_19764_gb300 import abi, sched
    specs = [sched.InstanceSpec(N, T, p, i) for i, (N, T, p) in enumerate(SPECS[:4])]
    multi = _instances(specs)
    mr = sched.MultiRunner(multi)
    tr = mr.trace()
    mr.iterate()
    torch.cuda.synchronize()
    assert mr.status() == abi.SNN_OK
    t = tr.times.cpu().numpy()
    assert np.all(t > 0)
    assert np.all(np.diff(t, axis=1) >= 0)
    assert np.all(np.diff(t, axis=1)[:, 3] > 0)          # every instance's forward took time
    s = tr.summary(multi)
    assert s["iteration_ms"] > 0 and set(s["slowest_instance"]["phase_us"]) == set(sched.MultiRunner.PHASES)
    abi.snn_multi_set_trace(mr.handle, None)
    tr.times.zero_()
    mr.iterate()
    torch.cuda.synchronize()
    assert not tr.times.any()
