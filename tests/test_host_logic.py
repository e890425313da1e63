"""Host-side logic of the batched and served forms, no GPU: the request stream of the
serving loop (Poisson arrivals, request mix), its latency summary, and the instance mix
of the batched form."""
import numpy as np

from paper_2510_19764_gb300 import sched, serve


def test_poisson_requests_arrivals_and_mix():
    rate, n = 1000.0, 20000
    reqs = serve.poisson_requests(n, rate, n_models=4, seed=3, finetune_frac=0.1)
    assert [r.rid for r in reqs] == list(range(n))
    arr = np.array([r.arrival for r in reqs])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    # exponential gaps: mean 1/rate (standard error 0.7 % at n = 20000)
    assert abs(np.diff(arr).mean() * rate - 1.0) < 0.05
    # fine-tuning share 10 % (standard error 0.2 %)
    assert abs(np.mean([r.finetune for r in reqs]) - 0.1) < 0.01
    assert {r.model for r in reqs} == {0, 1, 2, 3}
    assert all(0 <= r.label < serve.N_CLASSES for r in reqs)
    assert all(100 <= r.T <= 1000 for r in reqs)
    # time-warped bins: round(w T / n_bins) with w in [0.8, 1.2], at least one step
    assert all(max(1, int(0.8 * r.T / serve.N_BINS) - 1) <= r.bin_len <= int(1.2 * r.T / serve.N_BINS) + 1
               for r in reqs)


def test_poisson_requests_are_reproducible_per_seed():
    a = serve.poisson_requests(50, 200.0, 3, seed=7)
    b = serve.poisson_requests(50, 200.0, 3, seed=7)
    c = serve.poisson_requests(50, 200.0, 3, seed=8)
    assert a == b
    assert a != c


def test_latency_summary_percentiles():
    lat = np.random.default_rng(0).uniform(0.001, 0.02, size=999)
    res = [serve.Result(i, np.zeros(2), 0, float(x), False) for i, x in enumerate(lat)]
    s = serve.latency_summary(res, wall=2.0)
    assert s["requests"] == 999
    assert s["throughput_req_s"] == 999 / 2.0
    assert np.isclose(s["p50_ms"], np.percentile(lat * 1e3, 50))
    assert np.isclose(s["p99_ms"], np.percentile(lat * 1e3, 99))
    assert np.isclose(s["mean_ms"], lat.mean() * 1e3)
    assert s["p50_ms"] <= s["p99_ms"]


def test_batched_instance_mix():
    specs = sched.batched_specs(64, seed=0)
    assert len(specs) == 64
    assert {s.N for s in specs} == {256, 512, 1024, 2048}
    assert all(200 <= s.T <= 1000 for s in specs)
    assert all(0.05 <= s.p <= 0.20 for s in specs)
    assert len({s.seed for s in specs}) == 64
    assert specs == sched.batched_specs(64, seed=0)
    assert specs != sched.batched_specs(64, seed=1)
