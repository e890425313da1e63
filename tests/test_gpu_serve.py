"""Serving loop: every request's result is identical served alone (one at a time) and
served in the mix (continuous batching across models, overlapping launches), including
fine-tuning jobs on private weight copies."""
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


def test_results_identical_alone_and_in_the_mix():
    from paper_2510_19764_gb300 import serve
    task = synth.spoken_digit_task(5, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX, n_bins=serve.N_BINS)
    models = [serve.Model(0, 64, task, max_batch=8), serve.Model(1, 160, task, max_batch=8),
              serve.Model(2, 96, task, max_batch=8)]
    reqs = serve.poisson_requests(48, 1000.0, len(models), seed=3, finetune_frac=0.15, t_range=(20, 120))
    assert any(r.finetune for r in reqs)
    eng = serve.Engine(models, max_batch=8, slots_per_model=2, n_streams=4)
    mixed = eng.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert eng.stats["max_batch_seen"] > 1 and eng.stats["max_in_flight"] > 1
    alone = serve.Engine(models, max_batch=8, slots_per_model=1, n_streams=1).run_plain(reqs, realtime=False)
    assert [r.rid for r in mixed] == [r.rid for r in alone] == list(range(len(reqs)))
    for a, b in zip(mixed, alone):
        np.testing.assert_array_equal(a.ysum, b.ysum)
        assert a.pred == b.pred
    assert all(np.abs(r.ysum).sum() > 0 for r in mixed)


def test_realtime_loop_reports_latency():
    from paper_2510_19764_gb300 import serve
    task = synth.spoken_digit_task(5, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX, n_bins=serve.N_BINS)
    models = [serve.Model(0, 128, task, max_batch=16)]
    reqs = serve.poisson_requests(60, 2000.0, 1, seed=4, finetune_frac=0.0, t_range=(50, 200))
    eng = serve.Engine(models, max_batch=16)
    t0 = torch.cuda.Event(enable_timing=True)
    res = eng.run(reqs, realtime=True)
    s = serve.latency_summary(res, max(r.latency for r in res) + reqs[-1].arrival)
    assert s["requests"] == 60 and 0 < s["p50_ms"] <= s["p99_ms"]


def test_admission_failure_is_reported_not_hung():
    """Host-side fault: a memory budget too small for any slot or fine-tuning copy.  The
    loop raises AdmissionError at once instead of waiting for memory nothing will free;
    a budget that fits one slot at a time still serves everything, one launch at a time."""
    from paper_2510_19764_gb300 import serve
    task = synth.spoken_digit_task(5, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX, n_bins=serve.N_BINS)
    models = [serve.Model(0, 64, task, max_batch=4)]
    reqs = serve.poisson_requests(6, 1000.0, 1, seed=4, finetune_frac=0.0, t_range=(20, 40))
    with pytest.raises(serve.AdmissionError):
        serve.Engine(models, max_batch=4, slots_per_model=1, n_streams=1, mem_budget=1024).run(reqs, realtime=False)
    eng = serve.Engine(models, max_batch=4, slots_per_model=2, n_streams=2, mem_budget=1024)
    one_slot = eng.slots[0][0].bytes
    eng.mem_budget = one_slot
    res = eng.run(reqs, realtime=False)
    assert [r.rid for r in res] == list(range(len(reqs)))
    assert eng.stats["max_in_flight"] == 1


def test_serving_loop_allocates_nothing_and_admits_finetunes_by_their_bytes():
    """Fine-tuning copies are created with the engine: run() makes no device allocation
    (torch's allocator counts none) and admits a fine-tuning job by the exact byte count
    of its model's copy; a budget below that count is refused at once."""
    from paper_2510_19764_gb300 import serve
    task = synth.spoken_digit_task(5, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX, n_bins=serve.N_BINS)
    models = [serve.Model(0, 128, task, max_batch=8), serve.Model(1, 64, task, max_batch=8)]
    reqs = serve.poisson_requests(40, 1000.0, len(models), seed=8, finetune_frac=0.3, t_range=(20, 100))
    assert sum(r.finetune for r in reqs) >= 5
    eng = serve.Engine(models, max_batch=8, slots_per_model=2, n_streams=4, ft_slots_per_model=2)
    eng.run(reqs[:4], realtime=False)                       # first calls outside the count
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats()["allocation.all.allocated"]
    res = eng.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == before
    assert len(res) == len(reqs)
    ft = eng.ft_slots[0][0]
    assert ft.bytes > eng.slots[0][0].bytes
    eng.mem_budget = ft.bytes - 1
    with pytest.raises(serve.AdmissionError) as e:
        eng.run([r for r in reqs if r.finetune and r.model == 0][:1], realtime=False)
    assert str(ft.bytes) in str(e.value)


def test_concurrent_forward_launches_on_one_model_read_only_scratch():
    """Several batches of one served model's requests launched on different streams at
    once, with the packed rows built beforehand (SNN_STEP_PACKED_READY): each batch's
    results equal the same batch run alone, and the handle reports no error."""
    from paper_2510_19764_gb300 import abi, net, serve
    task = synth.spoken_digit_task(5, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX, n_bins=serve.N_BINS)
    m = serve.Model(0, 512, task, max_batch=16)
    rng = np.random.default_rng(3)
    batches = []
    for k in range(6):
        lab = rng.integers(0, serve.N_CLASSES, 16)
        b = net.DeviceBatch(m.cls, lab, np.full(16, 30), np.arange(16) + 100 * k, 300, workspace=False, records=False)
        batches.append(b)
    alone = []
    for b in batches:
        abi.snn_step_neurons_ex(m.cls.handle, b.desc, 0, 300, abi.SNN_STEP_PACKED_READY)
        torch.cuda.synchronize()
        alone.append(b.ysum.clone())
        b.reset_state()
    streams = [torch.cuda.Stream() for _ in batches]
    torch.cuda.synchronize()
    for b, s in zip(batches, streams):
        abi.snn_step_neurons_ex(m.cls.handle, b.desc, 0, 300, abi.SNN_STEP_PACKED_READY, s)
    torch.cuda.synchronize()
    for b, y in zip(batches, alone):
        assert torch.equal(b.ysum, y)
    assert m.d_in.status() == abi.SNN_OK
    with pytest.raises(abi.SnnError):
        abi.snn_step_neurons_ex(m.cls.handle, batches[0].desc, 0, 300, 4)
