#!/usr/bin/env python
"""Benchmark: e-prop + DEEP R training of the sparse recurrent classifier on one GB300.

Workload (one "step" = one training batch through the whole hot path):
  700 Poisson input channels -> 1024 ALIF (tau_m 20 ms, tau_a 2000 ms, v_thr 0.6,
  beta 0.0174) -> 20 leaky readouts; 10 % ragged input->hidden and hidden->hidden
  connectivity (row capacity 288 = roundup32(2 x max initial row length)); 20 classes of
  log-normal rate templates (0-50 Hz, 10 time bins) with per-trial time warp; 1000 steps
  of 1 ms; batch 512; e-prop gradient, L1 (1e-5) + Adam (lr 1e-3) and one DEEP R
  rewiring of both sparse projections per batch.  Synthetic data of the spoken-digit
  benchmark's shape (the dataset itself is not used).

Per step the GPU runs: every trial's 1000 steps in one launch (input spikes,
propagation, neurons, readout), the adjoint e-prop gradient, L1 + Adam, DEEP R.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# library kernels per training batch: forward call 5 (k_input, k_colsum, k_pack_narrow,
# k_forward, k_softmax_d), gradient 9 (k_readout_scan, k_backward_bulk, k_reduce_gb,
# k_sort_rows x2, k_gather, k_reduce_ragged x2, k_reduce_out), Adam 4 (k_adam_ragged x2,
# k_adam_dense x2), DEEP R 10 (eliminate, round0, accept0, distribute, form per
# projection; plus one 16-byte memset each)
LAUNCHES_PER_BATCH = 28
# DRAM bytes (read + write) of one k_forward launch at 512 trials from one ncu capture of
# the current kernel build (None until it has been captured; see profiles/)
FORWARD_TRAFFIC = 4 * 506.57e6
FORWARD_TRAFFIC_SOURCE = ("k_forward DRAM read+write per launch from one ncu capture of the current build at 128 "
                          "trials (14.4 MB read + 492.2 MB written = 506.6 MB), scaled by 4 (the psi record grows "
                          "with the trials)")
METRIC = "e-prop+DEEP R training samples/s"
UNIT = "samples/s"
WORKLOAD = {"n_in": 700, "N": 1024, "K": 20, "T": 1000, "B": 512, "p": 0.1, "n_bins": 10, "n_classes": 20}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sample-steps", type=int, default=100,
                    help="--impl reference: steps of the one trial each timed step simulates")
    ap.add_argument("--batch", type=int, default=512, help="trials per batch (512 = the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the batched and served rows of the default line (profiling runs)")
    ap.add_argument("--workload", default="classifier",
                    choices=["classifier", "batched", "serve", "topo", "topo-evolution", "kernels"],
                    help="classifier (default, the benchmark line); batched: 64 uneven instances, plain vs "
                         "graph-batched; serve: request loop latency; topo: topographic map steps/s; "
                         "topo-evolution: connectivity evolution of the map over a long run")
    ap.add_argument("--scale", type=int, default=2, help="topo: grid side 16*scale")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 4, 8, 16],
                    help="forward row schedule (warps per trial); 0 = the library default")
    ap.add_argument("--topo-steps", type=int, default=10000)
    ap.add_argument("--evolution-steps", type=int, default=100000,
                    help="topo-evolution: steps (time bins of 200 ms)")
    ap.add_argument("--topo-setting", default="disc", choices=["disc", "paper"],
                    help="topo / topo-evolution: disc = 1 ms steps with the disc input; paper = the printed "
                         "setting, h = 0.1 ms, Gaussian input, 20 ms stimulus interval, rewiring every 1 ms")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


# ------------------------------------------------------------------------ workload

def classifier_config(in_C: int, rec_C: int, world: int) -> dict:
    """The `config` of the classifier bench line (both arms)."""
    W = WORKLOAD
    return {"workload": "spoken-digit-shaped sparse ALIF classifier, e-prop + DEEP R training batch",
            "n_in": W["n_in"], "hidden": W["N"], "readouts": W["K"], "steps_per_trial": W["T"],
            "global_batch": W["B"] * world, "connectivity": W["p"], "row_capacity": [in_C, rec_C],
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (per-batch records and adjoint > 4 GB rewritten every step)"}


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value of x over all ranks (the bench's per-rank times)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(seed: int, device="cuda"):
    import numpy as np
    import synth
    from paper_2510_19764_gb300 import abi, net
    W = WORKLOAD
    task = synth.spoken_digit_task(seed, n_in=W["n_in"], n_classes=W["n_classes"], T=W["T"], n_bins=W["n_bins"])
    in_rag = synth.random_ragged(seed + 1, W["n_in"], W["N"], W["p"])
    rec_rag = synth.random_ragged(seed + 2, W["N"], W["N"], W["p"], no_autapse=True)
    W_out, b = synth.dense_readout(seed + 3, W["K"], W["N"])
    F32 = abi.SNN_F32
    d_in = net.DeviceRagged(in_rag.row_len, in_rag.ind, in_rag.w, W["N"], dtype=F32, adam=True, grad=True,
                            deepr=True, seed=seed + 100, device=device)
    d_rec = net.DeviceRagged(rec_rag.row_len, rec_rag.ind, rec_rag.w, W["N"], dtype=F32, no_autapse=True, adam=True,
                             grad=True, deepr=True, seed=seed + 101, device=device)
    cls = net.DeviceClassifier(W["n_in"], W["N"], W["K"], d_in, d_rec, W_out, b, task.thr, seed + 7,
                               net.NeuronCfg(tau_m=20.0, v_thr=0.6, beta=0.0174, tau_a=2000.0),
                               max_B=W["B"], max_T=W["T"], dtype=F32, device=device)
    return task, in_rag, rec_rag, cls


def count_events(batch, cls, device="cuda"):
    """Synaptic events of one batch: presynaptic spikes x row lengths (measurement only)."""
    import torch
    shifts = torch.arange(32, device=device, dtype=torch.int32)

    def per_neuron(rec, n):
        bits = (rec.unsqueeze(-1) >> shifts) & 1
        return bits.reshape(rec.shape[0], rec.shape[1], -1)[..., :n].sum(dim=(0, 1)).double()

    xin = per_neuron(batch.x_rec, cls.n_in)
    zh = per_neuron(batch.z_rec, cls.N)
    ev = float((xin * cls.w_in.row_len.double()).sum() + (zh * cls.w_rec.row_len.double()).sum())
    return ev, float(xin.sum() + zh.sum())


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, build, net
    if rank == 0 or world > 1:
        build.build()
    abi.load()
    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    W = WORKLOAD
    B, T = W["B"], W["T"]
    task, in_rag, rec_rag, cls = make_workload(args.seed + 1000 * rank, dev)
    n_total = args.warmup + args.steps
    batches = [synth.trial_batch(task, args.seed + rank, i, B) for i in range(2 * n_total + 4)]
    # device copies of every batch's trial descriptors (the device-resident leg)
    d_desc = [(torch.as_tensor(tb.labels, device=dev), torch.as_tensor(tb.bin_len, device=dev),
               torch.as_tensor(tb.trial_ids, device=dev)) for tb in batches]
    # pinned host copies (the end-to-end leg)
    h_desc = [(torch.as_tensor(tb.labels).pin_memory(), torch.as_tensor(tb.bin_len).pin_memory(),
               torch.as_tensor(tb.trial_ids).pin_memory()) for tb in batches]
    # NB batch buffers: the input spikes of the batches after the current one are drawn
    # on a side stream (they depend only on trial, step and channel), DEPTH steps ahead
    DEPTH = 2
    NB = DEPTH + 1
    bufs = [net.DeviceBatch(cls, batches[0].labels, batches[0].bin_len, batches[0].trial_ids, T, device=dev)
            for _ in range(NB)]
    if args.schedule:
        abi.snn_classifier_set_schedule(cls.handle, args.schedule)
    # the training steps run on a high-priority stream, the input draws on a low-priority
    # one: the block scheduler then fills only the slots the training kernels leave free
    stream = torch.cuda.Stream(device=dev, priority=-5)    # mapped to the highest priority
    side = torch.cuda.Stream(device=dev, priority=0)       # the default, lowest priority
    torch.cuda.set_stream(stream)
    ev_free = [torch.cuda.Event() for _ in range(NB)]     # buffer's last training step done
    ev_drawn = [torch.cuda.Event() for _ in range(NB)]    # buffer's inputs drawn
    for e in ev_free:
        e.record(stream)
    stats = torch.zeros((n_total, 2, 4), dtype=torch.int64, device=dev)   # DEEP R counts per batch
    lr, l1 = 1e-3, 1e-5
    calls = ["snn_step_neurons", "snn_eprop_update(GRAD)", "snn_eprop_update(APPLY)", "snn_rewire_deepr"]
    ev_pairs = []

    def draw(i, desc):
        X = bufs[i % NB]
        lab, bl, tid = desc
        side.wait_event(ev_free[i % NB])
        with torch.cuda.stream(side):
            X.labels.copy_(lab, non_blocking=True)
            X.bin_len.copy_(bl, non_blocking=True)
            X.trial_ids.copy_(tid, non_blocking=True)
            abi.snn_draw_inputs(cls.handle, X.desc, 0, T, side)
        ev_drawn[i % NB].record(side)

    def train(i, timed):
        X = bufs[i % NB]
        stream.wait_event(ev_drawn[i % NB])
        for t_ in (X.v, X.a, X.y, X.ysum, X.x_bits, X.z_bits):
            t_.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if timed else None
        if ev:
            ev[0].record(stream)
        abi.snn_step_neurons_ex(cls.handle, X.desc, 0, T, abi.SNN_STEP_INPUTS_READY, stream)
        if ev:
            ev[1].record(stream)
        abi.snn_eprop_update(cls.handle, X.desc, abi.SNN_EPROP_GRAD, None, stream)
        if ev:
            ev[2].record(stream)
        abi.snn_eprop_update(cls.handle, X.desc, abi.SNN_EPROP_APPLY, net.adam_params(lr, i + 1, l1=l1), stream)
        if ev:
            ev[3].record(stream)
        abi.snn_rewire_deepr(cls.w_in.handle, i, stats[i, 0], stream)
        abi.snn_rewire_deepr(cls.w_rec.handle, i, stats[i, 1], stream)
        if ev:
            ev[4].record(stream)
            ev_pairs.append(ev)
        ev_free[i % NB].record(stream)

    def run(lo, hi, desc, timed, after=None, fill=None):
        # steps lo .. hi-1; the inputs of steps lo .. lo+DEPTH-1 were drawn before, those
        # of hi .. hi+DEPTH-1 are drawn (or uploaded, fill) here: the same number per step
        fill = fill or draw
        for i in range(lo, hi):
            train(i, timed)
            fill(i + DEPTH, desc[i + DEPTH])
            if after:
                after(i)
        stream.wait_stream(side)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for i in range(DEPTH):
        draw(i, d_desc[i])
    run(0, args.warmup, d_desc, False)
    barrier()
    # the trainable state at the start of the timed region; the end-to-end leg restores
    # it and replays the same batches, so both legs time the same work
    state = [cls.W_out, cls.b_out, cls.W_out_m, cls.W_out_v, cls.b_m, cls.b_v]
    for r_ in (cls.w_in, cls.w_rec):
        state += [r_.row_len, r_.ind, r_.w, r_.m, r_.v, r_.sign_bits, r_.conn_bits]
    saved = [t_.clone() for t_ in state]
    # ---- device-resident timed region
    stats.zero_()
    with ClockSampler(local) as clk:
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        start.record(stream)
        run(args.warmup, n_total, d_desc, True)
        end.record(stream)
        barrier()
    ms = start.elapsed_time(end)
    ms_max = max_over_ranks(ms, world, dev)
    per_call = [0.0] * 4
    for ev in ev_pairs:
        for c in range(4):
            per_call[c] += ev[c].elapsed_time(ev[c + 1])
    per_call = [x / len(ev_pairs) for x in per_call]
    # the roofline pairs the last timed batch's work with that batch's own call times
    # (spike counts, hence work, drift as training proceeds)
    last_call = [ev_pairs[-1][c].elapsed_time(ev_pairs[-1][c + 1]) for c in range(4)]
    batch = bufs[(n_total - 1) % NB]
    events, spikes = count_events(batch, cls, dev)
    timed_stats = stats[args.warmup:n_total].cpu()
    rewired = int(timed_stats[:, :, :2].sum())                              # removed + formed, timed batches
    active = int(cls.w_in.row_len.sum().item() + cls.w_rec.row_len.sum().item())
    # fraction of the sparse synapses DEEP R replaced in each timed batch (Fig. 6's curve)
    rewired_fraction = [round(float(x) / active, 6) for x in timed_stats[:, :, 0].sum(1).tolist()]
    # ---- end-to-end leg through the public calls, host buffers each step: the same
    # batches from the same state as the timed region, their input spike rasters coming
    # from pinned host memory as a dataset's would (bit-packed, 700 channels x 1000 steps
    # per trial: 45 MB per batch), uploaded on the side stream while the previous batch
    # trains, then snn_step_neurons_ex(SNN_STEP_INPUTS_READY)
    ref_ysum = bufs[(n_total - 1) % NB].ysum.clone()      # the timed region's last predictions
    scratch = net.DeviceBatch(cls, batches[0].labels, batches[0].bin_len, batches[0].trial_ids, T, device=dev,
                              workspace=False, records=False)
    h_x = {}
    for i in range(args.warmup, n_total + DEPTH):
        lab, bl, tid = d_desc[i]
        scratch.labels.copy_(lab)
        scratch.bin_len.copy_(bl)
        scratch.trial_ids.copy_(tid)
        abi.snn_draw_inputs(cls.handle, scratch.desc, 0, T, stream)
        h_x[i] = torch.empty(scratch.x_rec.shape, dtype=scratch.x_rec.dtype).pin_memory()
        h_x[i].copy_(scratch.x_rec)
    del scratch
    out_host = torch.empty((B, W["K"]), dtype=torch.float32).pin_memory()
    stats_host = torch.empty((2, 4), dtype=torch.int64).pin_memory()
    for t_, v_ in zip(state, saved):
        t_.copy_(v_)

    def upload(i, desc):
        X = bufs[i % NB]
        lab, bl, tid = desc
        side.wait_event(ev_free[i % NB])
        with torch.cuda.stream(side):
            X.labels.copy_(lab, non_blocking=True)
            X.bin_len.copy_(bl, non_blocking=True)
            X.trial_ids.copy_(tid, non_blocking=True)
            X.x_rec.copy_(h_x[i], non_blocking=True)
        ev_drawn[i % NB].record(side)

    for i in range(args.warmup, args.warmup + DEPTH):
        upload(i, h_desc[i])
    barrier()

    def read_back(i):
        out_host.copy_(bufs[i % NB].ysum, non_blocking=True)
        stats_host.copy_(stats[i], non_blocking=True)
        stream.synchronize()

    e2e_start, e2e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_start.record(stream)
    t_host0 = time.perf_counter()
    run(args.warmup, n_total, h_desc, False, after=read_back, fill=upload)
    e2e_end.record(stream)
    barrier()
    e2e_ms = max(e2e_start.elapsed_time(e2e_end), (time.perf_counter() - t_host0) * 1e3)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_match = bool(torch.equal(out_host, ref_ysum.cpu()))
    h2d = sum(x.numel() * x.element_size() for x in h_desc[0]) + h_x[args.warmup].numel() * 4
    d2h = out_host.numel() * out_host.element_size() + stats_host.numel() * stats_host.element_size()
    ok = cls.w_in.status(stream) == abi.SNN_OK and cls.w_rec.status(stream) == abi.SNN_OK
    if rank != 0:
        return None
    value = B * args.steps * world / (ms_max / 1e3)
    pk = peaks()
    # dominant call and its algorithmic bytes
    dom = max(range(4), key=lambda c: per_call[c])
    N, n_in, K = W["N"], W["n_in"], W["K"]
    algs = {
        # forward: 8 B per synaptic event (ind + w) + 4 B per spike-bit list entry + 32 B per
        # ALIF neuron-step (v, a read/write; psi record)
        0: events * 8 + spikes * 4 + B * T * N * 32.0,
        # gradient: psi read + delta write/read + synaptic events gathered (4 B delta + 4 B ind)
        1: B * T * N * 4.0 * 3 + events * 8,
        # Adam: 28 B per active slot; DEEP R: 8 B read per active slot (+ moves, formations)
        2: 28.0 * active,
        3: 8.0 * active,
    }
    alg = algs[dom]
    traffic = FORWARD_TRAFFIC * B / 512 if dom == 0 and FORWARD_TRAFFIC else None
    achieved = alg / (last_call[dom] / 1e3) / 1e9
    by_call = {calls[c]: {"achieved_gbs": round(algs[c] / (last_call[c] / 1e3) / 1e9, 1),
                          "frac": round(algs[c] / (last_call[c] / 1e3) / 1e9 / pk["hbm_gbs"], 4)}
               for c in range(4) if last_call[c] > 0}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": classifier_config(in_rag.C, rec_rag.C, world),
        # synaptic events of the last timed batch over its own step time
        "synaptic_events_per_s": round(events * world / (sum(last_call) / 1e3), 1),
        # e-prop as computed here (adjoint form): per batch the reverse-time scan visits
        # every (trial, step, hidden neuron) once and the gather reads one adjoint value per
        # synaptic event; both over the gradient call's own time
        "eprop_adjoint": {"neuron_steps_scanned_per_s": round(B * T * N * world / (last_call[1] / 1e3), 1),
                          "gathered_events_per_s": round(events * world / (last_call[1] / 1e3), 1)},
        # NOT work done: the update count of the per-synapse trace form (every active
        # synapse of every trial at every step) that the adjoint form replaces, per second
        # of the whole training step; a nominal equivalent for comparison with trace-form
        # implementations only
        "trace_form_equivalent_synapse_updates_per_s": round(active * B * T * world / (ms_max / 1e3 / args.steps), 1),
        # DEEP R: (removed + formed) over the rewiring calls' own time
        "rewired_synapses_per_s": round(rewired / (per_call[3] * args.steps / 1e3), 1) if per_call[3] > 0 else None,
        "deepr_rewired_fraction": {"per_batch": rewired_fraction,
                                   "mean": round(sum(rewired_fraction) / len(rewired_fraction), 6)},
        "per_call_ms": {c: round(x, 4) for c, x in zip(calls, per_call)},
        "roofline": {"kernel": calls[dom], "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                     "achieved_is": "algorithmic bytes (events x 8 B + spike entries x 4 B + neuron-steps x 32 B) "
                                    "per launch / CUDA-event time; most of them are served from L2 and shared "
                                     "memory, see achieved_dram_gbs",
                     "traffic": traffic,
                     "achieved_dram_gbs": round(traffic / (last_call[dom] / 1e3) / 1e9, 1) if traffic else None,
                     "dram_frac": round(traffic / (last_call[dom] / 1e3) / 1e9 / pk["hbm_gbs"], 4) if traffic
                     else None,
                     "traffic_source": FORWARD_TRAFFIC_SOURCE if traffic else
                     "null: no ncu capture of the current k_forward build",
                     "peak_source": pk["source"]},
        "roofline_by_call": by_call,
        "e2e": {"value": round(B * args.steps * world / (e2e_ms / 1e3), 2), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "inputs": "each batch's input spike rasters (bit-packed, 512 x 1000 x 700) and trial descriptors "
                          "copied from pinned host memory every step; predictions and rewiring counts read back",
                "same_results_as_device_leg": e2e_match},
        "gpu_launches": LAUNCHES_PER_BATCH * args.steps,
        "clocks": clocks,
        "status_ok": bool(ok),
    }
    return line


def cpu_info() -> dict:
    """Host CPU model and the threads the oracle uses (one)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def oracle_batch_sample(seed: int, sample_steps: int, n_trials: int):
    """The FP64 oracle on one core for one training batch step of the bench workload,
    on a bounded sample: n_trials trials of sample_steps steps each (forward, e-prop
    traces and gradients), then the whole per-batch update on the full matrices (L1 +
    Adam on both projections and the readout, DEEP R on both projections).  The batch
    time is B x (per-trial time scaled to 1000 steps) + the update time.  Returns
    (samples/s, description)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import synth
    from oracle import classifier as oc
    from oracle import deepr as od
    W = WORKLOAD
    task = synth.spoken_digit_task(seed, n_in=W["n_in"], n_classes=W["n_classes"], T=W["T"], n_bins=W["n_bins"])
    in_rag = synth.random_ragged(seed + 1, W["n_in"], W["N"], W["p"])
    rec_rag = synth.random_ragged(seed + 2, W["N"], W["N"], W["p"], no_autapse=True)
    W_out, b = synth.dense_readout(seed + 3, W["K"], W["N"])
    onet = oc.ClassifierNet(W["n_in"], W["N"], W["K"], in_rag.row_len, in_rag.ind, in_rag.w, rec_rag.row_len,
                            rec_rag.ind, rec_rag.w, W_out, b, oc.NeuronParams())
    tb = synth.trial_batch(task, seed, 0, n_trials)
    t0 = time.perf_counter()
    G = None
    for k in range(n_trials):
        r = oc.forward_trial(onet, task.thr, tb.labels[k], tb.bin_len[k], tb.trial_ids[k], seed + 7, sample_steps)
        g = oc.eprop_gradients(onet, r["x"], r["z"], r["psi"], r["d"])
        G = list(g) if G is None else [a + c for a, c in zip(G, g)]
    t_trials = time.perf_counter() - t0
    t1 = time.perf_counter()
    b1t, b2t = oc.adam_bias(0.9, 1), oc.adam_bias(0.999, 1)
    counts = 0
    for (rag, Gm, sd, no_aut) in ((in_rag, G[0], seed + 100, False), (rec_rag, G[1], seed + 101, True)):
        sign, conn = od.init_bitfields(rag.row_len, rag.ind, rag.w, W["N"], sd)
        Gl = oc.l1_on_sign(Gm, rag.row_len, rag.ind, sign, 1e-5)
        w, m, v = oc.adam_ragged(rag.w, 0 * rag.w, 0 * rag.w, Gl, rag.row_len, 1e-3, b1t, b2t)
        out = od.rewire(rag.row_len, rag.ind, w, m, v, sign, conn, rag.C, W["N"], no_aut, sd, 0)
        counts += out["removed"] + out["formed"]
    oc.adam(W_out, 0 * W_out, 0 * W_out, G[2], 1e-3, b1t, b2t)
    oc.adam(b, 0 * b, 0 * b, G[3], 1e-3, b1t, b2t)
    t_update = time.perf_counter() - t1
    per_trial = t_trials / n_trials * W["T"] / sample_steps
    batch_s = W["B"] * per_trial + t_update
    desc = (f"{n_trials} trial(s) x {sample_steps} of {W['T']} steps (forward + e-prop traces, {t_trials:.1f} s) "
            f"scaled to {W['B']} full trials, + one L1/Adam/DEEP R update of both full projections "
            f"({t_update:.2f} s, {counts} synapses rewired); FP64 numpy, 1 thread")
    return W["B"] / batch_s, desc, (in_rag.C, rec_rag.C), batch_s


# ------------------------------------------------------------------ other workloads

def run_batched(args, timed: int | None = None):
    """64 independent classifier instances of uneven size and trial length (hidden
    256..2048, 200..1000 steps, 5..20 %), one training trial + DEEP R each per
    iteration, in four forms of the same computation: the persistent multi-instance
    kernel (one launch per iteration, row schedules autotuned), a CUDA graph of the
    per-call launches over 16 streams, and the plain one-instance-at-a-time forms with
    one forward launch per trial and with one per step.  samples/s = instances /
    iteration time (CUDA events for the device-timed forms, the host clock around a
    synchronised iteration for the plain ones)."""
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, build, sched
    build.build()
    abi.load()
    timed = timed or max(3, args.steps)
    specs = sched.batched_specs(64, args.seed)
    task = synth.spoken_digit_task(args.seed, n_in=sched.N_IN, n_classes=sched.N_CLASSES, T=1000,
                                   n_bins=sched.N_BINS)
    insts = [sched.Instance(s, task) for s in specs]
    tuner = sched.Autotuner(target="multi")
    table = tuner.tune(insts)

    def dev_time(fn, n):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / n

    def host_time(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    mr = sched.MultiRunner(insts)
    for _ in range(3):
        mr.iterate()
    t_multi = dev_time(mr.iterate, timed)
    ok_multi = mr.status() == abi.SNN_OK
    trace = mr.trace()                 # one more run with phase timing (not in the timed region)
    mr.iterate()
    torch.cuda.synchronize()
    phases = trace.summary(insts)
    abi.snn_multi_set_trace(mr.handle, None)
    mr.capture(4)
    mr.replay()
    t_multi_graph = dev_time(mr.replay, max(1, timed // 4)) / 4
    br = sched.BatchedRunner(insts, n_streams=16)
    for inst in insts:          # first calls outside capture
        inst.enqueue(torch.cuda.current_stream())
    br.capture()
    br.iterate()
    t_graph = dev_time(br.iterate, timed)
    whole = sched.PlainRunner(insts, per_step=False)
    whole.iterate()
    t_whole = host_time(whole.iterate)
    per_step = sched.PlainRunner(insts, per_step=True)
    t_step = host_time(per_step.iterate)
    ok = ok_multi and all(i.d_in.status() == abi.SNN_OK and i.d_rec.status() == abi.SNN_OK for i in insts)
    n = len(insts)
    mr.close()
    return {"workload": "batched", "metric": "training samples/s (64 uneven instances, one trial each)",
            "instances": n, "steps_total": int(sum(s.T for s in specs)),
            "persistent_samples_per_s": round(n / t_multi, 2),
            "persistent_graph_samples_per_s": round(n / t_multi_graph, 2),
            "graph_of_calls_samples_per_s": round(n / t_graph, 2),
            "plain_whole_trial_samples_per_s": round(n / t_whole, 2),
            "plain_per_step_samples_per_s": round(n / t_step, 2),
            "speedup_vs_plain_whole_trial": round(t_whole / t_multi, 2),
            "speedup_vs_plain_per_step": round(t_step / t_multi, 2),
            "ms_per_iteration": {"persistent": round(t_multi * 1e3, 3), "persistent_graph": round(t_multi_graph * 1e3, 3),
                                 "graph_of_calls": round(t_graph * 1e3, 3), "plain_whole_trial": round(t_whole * 1e3, 2),
                                 "plain_per_step": round(t_step * 1e3, 1)},
            "status_ok": bool(ok),
            "persistent_phase_trace": phases,
            "row_schedule_table": {str(k): list(v) for k, v in table.items()},
            "row_schedule_ms": {str(k): {str(m[1]): round(t, 3) for m, t in v.items()} for k, v in tuner.timings.items()}}


def run_serve(args, quick: bool = False):
    """Request loop over 4 resident classifiers (hidden 256..2048, 10 %), requests of
    100-1000 steps, 10 % fine-tuning jobs, Poisson arrivals at 200 / 1000 / 5000 req/s:
    continuous batching vs one request at a time (latency = arrival to result on the
    host)."""
    import numpy as np
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, build, serve
    build.build()
    abi.load()
    task = synth.spoken_digit_task(args.seed, n_in=serve.N_IN, n_classes=serve.N_CLASSES, T=serve.T_MAX,
                                   n_bins=serve.N_BINS)
    models = [serve.Model(i, N, task, max_batch=64) for i, N in enumerate((256, 512, 1024, 2048))]
    eng = serve.Engine(models, max_batch=64, slots_per_model=3, n_streams=16)
    warm = serve.poisson_requests(64, 1e6, len(models), seed=99)
    eng.run(warm, realtime=False)
    eng.run_plain(warm[:8], realtime=False)
    out = {"workload": "serve", "metric": "served requests/s with p50/p99 latency (ms)", "rates": {}}
    for rate in (200.0, 1000.0, 5000.0):
        n = int(min(1500 if quick else 4000, rate * (1.0 if quick else 2.0)))
        reqs = serve.poisson_requests(n, rate, len(models), seed=int(rate))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = eng.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        s_b = serve.latency_summary(res, wall)
        t0 = time.perf_counter()
        res_p = eng.run_plain(reqs, realtime=True)
        wall_p = time.perf_counter() - t0
        s_p = serve.latency_summary(res_p, wall_p)
        same = all(np.array_equal(x.ysum, y.ysum) for x, y in zip(res, res_p))
        out["rates"][str(int(rate))] = {"requests": n, "continuous": s_b, "plain": s_p,
                                        "results_identical": bool(same)}
    out["engine_stats"] = eng.stats
    return out


def systems_rows(args) -> dict:
    """The systems rows of the metric on the default line: the batched form against
    both plain forms, and served p50/p99 against plain serving (shorter runs than the
    --workload batched / serve lines)."""
    import gc
    import torch
    gc.collect()
    torch.cuda.empty_cache()
    out = {"batched": run_batched(args, timed=5)}
    gc.collect()
    torch.cuda.empty_cache()
    out["served"] = run_serve(args, quick=True)
    return out


def topo_setup(args):
    """The topographic map of the topo workloads: two L x L sheets (L = 16 * scale),
    capacity 64, pairwise-Bernoulli initial connectivity, 10 s^2 attempts per projection
    per rewiring.  Returns (L, N, dt_ms, device projections, params, rewiring params,
    state)."""
    import synth
    from paper_2510_19764_gb300 import net
    L = 16 * args.scale
    N = L * L
    C = 64
    ff = synth.topo_initial(args.seed + 1, L, 0.16, 2.5, C, 0.2)
    lat = synth.topo_initial(args.seed + 2, L, 1.0, 1.0, C, 0.2)
    dff = net.DeviceRagged(ff.row_len, ff.ind, ff.w, N, seed=11)
    dlat = net.DeviceRagged(lat.row_len, lat.ind, lat.w, N, seed=12)
    L_f = 16 if args.scale > 2 else L
    if args.topo_setting == "paper":
        dt = 0.1
        tp = net.topo_params(L=L, L_f=L_f, dt=dt, t_stim=200, f_base=5.0, f_in=152.8, sigma_stim=2.0)
    else:
        dt = 1.0
        tp = net.topo_params(L=L, L_f=L_f)
    n_att = 10 * args.scale * args.scale
    rw = {"ff": net.topo_rewire(L, 0.16, 2.5, n_att), "lat": net.topo_rewire(L, 1.0, 1.0, n_att)}
    st = net.DeviceTopoState(N, -70.0)
    return L, N, dt, {"ff": dff, "lat": dlat}, tp, rw, st


def run_topo(args):
    """Topographic map (two L x L sheets, L = 16 * scale): steps/s of the full step
    sequence (input, propagation, conductance LIF, STDP on both projections, rewiring
    every 10 steps with 10 s^2 attempts per projection)."""
    import torch
    from paper_2510_19764_gb300 import abi, build
    build.build()
    abi.load()
    L, N, dt, dev, tp, rw, st = topo_setup(args)
    s_ff = torch.zeros(4, dtype=torch.int64, device="cuda")
    s_lat = torch.zeros(4, dtype=torch.int64, device="cuda")
    abi.snn_topo_run(tp, st.desc, dev["ff"].handle, dev["lat"].handle, rw["ff"], rw["lat"], 5, 10, 0, 200, s_ff,
                     s_lat)
    torch.cuda.synchronize()
    n = args.topo_steps
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    abi.snn_topo_run(tp, st.desc, dev["ff"].handle, dev["lat"].handle, rw["ff"], rw["lat"], 5, 10, 200, n, s_ff,
                     s_lat)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    stats_ff, stats_lat = s_ff.cpu().tolist(), s_lat.cpu().tolist()
    cpu = topo_cpu_baseline(args, L)
    return {"workload": "topo", "metric": f"simulated steps/s ({dt:g} ms steps)", "setting": args.topo_setting,
            "cpu_baseline": cpu,
            "L": L, "neurons_per_sheet": N, "steps": n, "steps_per_s": round(n / (ms / 1e3), 1),
            "realtime_factor": round(n * dt / ms, 2), "ms_per_1000_steps": round(ms / n * 1000, 3),
            "path": "one thread-block-cluster launch per 1000 steps (up to 4 neurons per thread)",
            "rewire_ff": dict(zip(["removed", "formed", "overflow", "attempts"], stats_ff)),
            "rewire_lat": dict(zip(["removed", "formed", "overflow", "attempts"], stats_lat))}


def topo_cpu_baseline(args, L, budget_s=3.0, max_steps=1000):
    """The FP64 oracle on one core for the same map, setting and seeds: steps from t = 0
    until about budget_s seconds have passed (at most max_steps), rewiring included."""
    import synth
    from oracle import topo as ot
    p = ot.paper_setting(L) if args.topo_setting == "paper" else \
        ot.TopoParams(L=L, n_att=10 * args.scale * args.scale, L_f=16 if args.scale > 2 else None)
    ff = synth.topo_initial(args.seed + 1, L, 0.16, 2.5, 64, 0.2)
    lat = synth.topo_initial(args.seed + 2, L, 1.0, 1.0, 64, 0.2)
    st = ot.initial_state([ff.row_len, ff.ind, ff.w], [lat.row_len, lat.ind, lat.w], p)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps and (n < 20 or time.perf_counter() - t0 < budget_s):
        ot.step(st, n, p, {"input": 5, "ff": 11, "lat": 12}, 64)
        n += 1
    dt_s = time.perf_counter() - t0
    return {"value": round(n / dt_s, 2), "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} steps from t = 0 of the same map ({dt_s:.1f} s)"}


def run_topo_evolution(args):
    """Connectivity evolution of the topographic map over a long run (the analysis of
    Sec. 3.2, Figs. 8-9): the map of run_topo simulated in time bins of 200 steps; per
    bin the rewiring's elimination and formation histograms (by squared distance) and
    the in-/out-degrees of both projections; at the start and the end the connection
    probability and mean weight by displacement.  All recording is done by the
    library's kernels on the device; the host reads the records once at the end."""
    import math
    import torch
    from paper_2510_19764_gb300 import abi, build, net
    build.build()
    abi.load()
    L, N, dt, dev, tp, rw, st = topo_setup(args)
    BIN = int(round(200.0 / dt))                  # 200 ms time bins
    n_bins = max(1, args.evolution_steps // BIN)
    projs = ("ff", "lat")
    hist = {k: net.attach_event_histograms(rw[k], L) for k in projs}
    nb = hist["ff"][0].numel()
    # device records: [bin][elim, form][d2] and [bin][in, out][neuron]
    rec_ev = {k: torch.zeros((n_bins, 2, nb), dtype=torch.int64, device="cuda") for k in projs}
    rec_deg = {k: torch.zeros((n_bins + 1, 2, N), dtype=torch.int32, device="cuda") for k in projs}
    prof = {}

    def snapshot(b):
        for k in projs:
            count, wsum, indeg = net.topo_connectivity(dev[k], L)
            rec_deg[k][b, 0].copy_(indeg)
            rec_deg[k][b, 1].copy_(dev[k].row_len)
            if b in (0, n_bins):
                prof[(k, b)] = (count, wsum)

    snapshot(0)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for b in range(n_bins):
        abi.snn_topo_run(tp, st.desc, dev["ff"].handle, dev["lat"].handle, rw["ff"], rw["lat"], 5, 10, b * BIN, BIN)
        for k in projs:
            rec_ev[k][b, 0].copy_(hist[k][0])
            rec_ev[k][b, 1].copy_(hist[k][1])
            hist[k][0].zero_()
            hist[k][1].zero_()
        snapshot(b + 1)
    e.record()
    e.synchronize()
    ms = a.elapsed_time(e)
    unit_bin = [math.isqrt(d2) for d2 in range(nb)]
    n_unit = unit_bin[-1] + 1

    def unit(h):                       # squared-distance bins -> unit-distance bins
        out = [0] * n_unit
        for d2, c in enumerate(h):
            out[unit_bin[d2]] += int(c)
        return out

    fifths = [(n_bins * q // 5, max(n_bins * (q + 1) // 5, n_bins * q // 5 + 1)) for q in range(5)]
    out = {"workload": "topo-evolution", "setting": args.topo_setting, "L": L, "neurons_per_sheet": N,
           "dt_ms": dt, "steps": n_bins * BIN, "bin_steps": BIN, "model_s": round(n_bins * BIN * dt / 1e3, 1),
           "steps_per_s_with_analysis": round(n_bins * BIN / (ms / 1e3), 1),
           "initial_degree_theory": round(2 * math.pi * 0.16 * 2.5 ** 2, 3),
           "rates": "events per 200 ms bin, averaged over each fifth of the run"}
    for k in projs:
        ev = rec_ev[k].cpu().numpy()
        deg = rec_deg[k].cpu().numpy().astype(float)
        head, tail = max(1, n_bins // 10), max(1, n_bins // 10)
        cnt0, w0 = (x.cpu().numpy() for x in prof[(k, 0)])
        cnt1, w1 = (x.cpu().numpy() for x in prof[(k, n_bins)])
        dy = list(range(L // 2 + 1))
        out[k] = {
            "elim_rate": [round(float(ev[lo:hi, 0].sum(1).mean()), 2) for lo, hi in fifths],
            "form_rate": [round(float(ev[lo:hi, 1].sum(1).mean()), 2) for lo, hi in fifths],
            "elim_by_distance_first_tenth": unit(ev[:head, 0].sum(0)),
            "elim_by_distance_last_tenth": unit(ev[-tail:, 0].sum(0)),
            "form_by_distance_first_tenth": unit(ev[:head, 1].sum(0)),
            "form_by_distance_last_tenth": unit(ev[-tail:, 1].sum(0)),
            "in_degree_mean": [round(float(deg[b, 0].mean()), 3) for b in (0, *[hi for _, hi in fifths])],
            "in_degree_std": [round(float(deg[b, 0].std()), 3) for b in (0, *[hi for _, hi in fifths])],
            "out_degree_mean": [round(float(deg[b, 1].mean()), 3) for b in (0, *[hi for _, hi in fifths])],
            "out_degree_std": [round(float(deg[b, 1].std()), 3) for b in (0, *[hi for _, hi in fifths])],
            "p_conn_dx0_start": [round(float(cnt0[d * L] / N), 4) for d in dy],
            "p_conn_dx0_end": [round(float(cnt1[d * L] / N), 4) for d in dy],
            "w_mean_dx0_end": [round(float(w1[d * L] / cnt1[d * L]), 4) if cnt1[d * L] else None for d in dy],
        }
    return out


def run_kernels(args):
    """DEEP R rewiring and standalone ragged propagation on a 65536 x 65536 projection
    (~287 synapses per row, 18.8 M synapses; arrays and bitfields ~1.4 GB, far larger
    than L2): mean CUDA-event time per call after warm-up, and the algorithmic bytes of
    each call (bytes the method must move per unit of work) per second against the measured HBM
    copy bandwidth."""
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, build, net
    build.build()
    abi.load()
    dev = "cuda"
    P = Q = 65536
    k, C = 288, 320
    rag = synth.large_ragged(args.seed, P, Q, k, C)
    r = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, adam=True, deepr=True, seed=args.seed + 3)
    pk = peaks()
    gen = torch.Generator(device=dev)
    gen.manual_seed(args.seed)
    slot = torch.arange(C, device=dev)[None, :]
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    rw = []
    for rep in range(8):
        # a fixed fraction of live synapses turns against its sign bit, as after an
        # optimiser step; DEEP R removes exactly those and regrows as many elsewhere
        live = slot < r.row_len[:, None].long()
        flip = live & (torch.rand((P, C), generator=gen, device=dev) < 0.02) & (r.w != 0)
        r.w[flip] = -r.w[flip]
        first = torch.where(flip.any(1), flip.int().argmax(1), torch.full((P,), C, device=dev))
        moved = int((live & ~flip & (slot > first[:, None])).sum())
        active, removed = int(live.sum()), int(flip.sum())
        len_after_elim = r.row_len.long() - flip.sum(1)
        stats.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        abi.snn_rewire_deepr(r.handle, rep, stats)
        b.record()
        b.synchronize()
        formed = int(stats[1])
        act_rows = int((r.row_len.long() > len_after_elim).sum())
        # elimination: 8 B per active slot + 16 B per moved slot + one bitfield word per
        # removal; formation: 16 B per new synapse + Q/8 B bitfield row per row with activations
        by = 8 * active + 16 * moved + 4 * removed + 16 * formed + (Q // 8) * act_rows
        if rep >= 3:
            rw.append((a.elapsed_time(b), by, removed + formed))
    ms = sum(x[0] for x in rw) / len(rw)
    by = sum(x[1] for x in rw) / len(rw)
    nrw = sum(x[2] for x in rw) / len(rw)
    out = {"workload": "kernels", "matrix": {"P": P, "Q": Q, "C": C, "synapses": int(r.row_len.sum())},
           "snn_rewire_deepr": {"ms": round(ms, 4), "rewired_synapses_per_s": round(nrw / (ms / 1e3), 1),
                                "algorithmic_bytes": int(by),
                                "roofline": {"bound": "hbm", "achieved": round(by / (ms / 1e3) / 1e9, 1),
                                             "peak": pk["hbm_gbs"], "unit": "GB/s",
                                             "frac": round(by / (ms / 1e3) / 1e9 / pk["hbm_gbs"], 4),
                                             "peak_source": pk["source"]}}}
    # standalone propagation of B spike vectors (10 % of rows spiking) with shared weights
    B = 16
    spk = torch.rand((B, P), generator=gen, device=dev) < 0.1
    shifts = torch.arange(32, device=dev, dtype=torch.int64)
    words = (spk.view(B, P // 32, 32).long() << shifts).sum(-1)
    pre = torch.where(words >= 2 ** 31, words - 2 ** 32, words).int().contiguous()
    acc = torch.zeros((B, Q), dtype=torch.int64, device=dev)
    events = int((spk.long() * r.row_len.long()[None, :]).sum())
    spikes = int(spk.sum())
    times = []
    for rep in range(8):
        acc.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        abi.snn_propagate(r.handle, pre, B, acc)
        b.record()
        b.synchronize()
        if rep >= 3:
            times.append(a.elapsed_time(b))
    ms = sum(times) / len(times)
    by = 8 * events + 4 * spikes
    out["snn_propagate"] = {"ms": round(ms, 4), "instances": B, "synaptic_events": events,
                            "synaptic_events_per_s": round(events / (ms / 1e3), 1), "algorithmic_bytes": by,
                            "roofline": {"bound": "hbm", "achieved": round(by / (ms / 1e3) / 1e9, 1),
                                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                                         "frac": round(by / (ms / 1e3) / 1e9 / pk["hbm_gbs"], 4),
                                         "peak_source": pk["source"]}}
    # the same propagation from a target-tiled plan: each tile's synapses read once for all
    # 16 instances, sums in shared memory; its algorithmic bytes count that reuse: the
    # shared weights once per row that spiked in any instance
    plan = abi.snn_create_prop_plan(r.handle, B)
    try:
        pack_t, times = [], []
        for rep in range(8):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.snn_prop_plan_pack(plan)
            b.record()
            b.synchronize()
            if rep >= 3:
                pack_t.append(a.elapsed_time(b))
        ref = acc.clone()
        for rep in range(8):
            acc.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.snn_propagate_tiled(plan, pre, B, acc)
            b.record()
            b.synchronize()
            if rep >= 3:
                times.append(a.elapsed_time(b))
        assert torch.equal(acc, ref), "tiled propagation differs from the row-major one"
    finally:
        abi.snn_destroy_prop_plan(plan)
    ms_t = sum(times) / len(times)
    union_slots = int((spk.any(0).long() * r.row_len.long()).sum())
    by_t = 8 * union_slots + 4 * spikes
    nsyn = int(r.row_len.sum())
    out["snn_propagate_tiled"] = {
        "ms": round(ms_t, 4), "instances": B, "synaptic_events": events,
        "synaptic_events_per_s": round(events / (ms_t / 1e3), 1), "same_sums_as_snn_propagate": True,
        "algorithmic_bytes": by_t,
        "algorithmic_bytes_is": "8 B per slot of every row that spiked in at least one instance (read once for "
                                "all instances) + 4 B per spike",
        "roofline": {"bound": "hbm", "achieved": round(by_t / (ms_t / 1e3) / 1e9, 1), "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": round(by_t / (ms_t / 1e3) / 1e9 / pk["hbm_gbs"], 4),
                     "peak_source": pk["source"]},
        "per_instance_event_bytes_per_s": round(by / (ms_t / 1e3) / 1e9, 1),
        "pack_ms": round(sum(pack_t) / len(pack_t), 4),
        "pack_bytes_per_s": round(20 * nsyn / (sum(pack_t) / len(pack_t) / 1e3) / 1e9, 1)}
    out["deepr_guided_vs_uniform"] = deepr_guided_timing(args, dev)
    out["snn_rewire_topo"] = topo_rewire_timing(args, dev, pk)
    return out


def topo_rewire_timing(args, dev, pk):
    """Topographic rewiring (Sec. 2.2's elimination and distance-dependent formation) of
    the lateral projection alone: a 112 x 112 sheet with 490 attempts per rewiring (one
    CTA) and a 256 x 256 sheet with 65536 attempts (rows spread over the grid).  Mean
    CUDA-event time per call after warm-up; algorithmic bytes = per row with attempts its
    length word and 8 B per synapse read, per changed row its length and 8 B per synapse
    written back.  The candidate bitfields live in shared memory and move no HBM bytes."""
    import numpy as np
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, net
    res = {}
    for L, C, n_att in ((112, 32, 490), (256, 32, 65536)):
        N = L * L
        rag = synth.topo_initial(args.seed + 7, L, 1.0, 1.0, C, 0.2)
        g = np.where(rag.ind >= 0, np.random.default_rng(args.seed).uniform(0, 0.2, rag.w.shape), 0.0)
        r = net.DeviceRagged(rag.row_len, rag.ind, g.astype(np.float32), N, dtype=0, seed=args.seed + 8)
        rw = net.topo_rewire(L, 1.0, 1.0, n_att, g_max=0.2)
        stats = torch.zeros(4, dtype=torch.int64, device=dev)
        times, bys, nrw = [], [], []
        for rep in range(8):
            before_len = r.row_len.long().clone()
            before_ind = r.ind.clone()
            stats.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.snn_rewire_topo(r.handle, rw, rep, stats)
            b.record()
            b.synchronize()
            st = stats.cpu().tolist()
            changed = (r.row_len.long() != before_len) | (r.ind != before_ind).any(1)
            # rows with attempts: the expected number of distinct rows among n_att uniform draws
            touched = N * (1.0 - (1.0 - 1.0 / N) ** n_att)
            by = touched * (4 + 8 * float(before_len.float().mean())) + \
                int((4 + 8 * r.row_len.long()[changed]).sum())
            if rep >= 3:
                times.append(a.elapsed_time(b))
                bys.append(by)
                nrw.append(st[0] + st[1])
        assert r.status() == abi.SNN_OK
        ms = sum(times) / len(times)
        by = sum(bys) / len(bys)
        res[f"{L}x{L}"] = {"attempts": n_att, "ms": round(ms, 4), "form": "one CTA" if n_att <= 4096 else "grid",
                           "rewired_synapses_per_call": round(sum(nrw) / len(nrw), 1),
                           "attempts_per_s": round(n_att / (ms / 1e3), 1), "algorithmic_bytes": int(by),
                           "roofline": {"bound": "hbm", "achieved": round(by / (ms / 1e3) / 1e9, 2),
                                        "peak": pk["hbm_gbs"], "unit": "GB/s",
                                        "frac": round(by / (ms / 1e3) / 1e9 / pk["hbm_gbs"], 5),
                                        "peak_source": pk["source"]}}
    return res


def deepr_guided_timing(args, dev):
    """DEEP R on the classifier's recurrent projection shape (1024 x 1024, 10 %, no
    autapses; 2 % of the synapses turned against their sign per rewiring) with uniform
    and with distance-guided formation (neurons on a 32 x 32 torus, sigma 2): mean
    CUDA-event time per rewiring."""
    import torch
    import synth
    from paper_2510_19764_gb300 import abi, net
    N, L = 1024, 32
    res = {}
    for mode in ("uniform", "guided"):
        rag = synth.random_ragged(args.seed + 5, N, N, 0.1, no_autapse=True)
        r = net.DeviceRagged(rag.row_len, rag.ind, rag.w, N, no_autapse=True, adam=True, deepr=True, seed=5)
        keep = None
        if mode == "guided":
            g = abi.DeeprGuide()
            g.L, g.reserved, g.sigma = L, 0, 2.0
            keep = torch.arange(N, dtype=torch.int32, device=dev)
            g.pre_site = g.post_site = abi.ptr(keep)
            abi.snn_ragged_set_deepr_guide(r.handle, g)
        gen = torch.Generator(device=dev)
        gen.manual_seed(args.seed)
        slot = torch.arange(r.C, device=dev)[None, :]
        stats = torch.zeros(4, dtype=torch.int64, device=dev)
        times, formed = [], 0
        for rep in range(8):
            live = slot < r.row_len[:, None].long()
            flip = live & (torch.rand(r.w.shape, generator=gen, device=dev) < 0.02) & (r.w != 0)
            r.w[flip] = -r.w[flip]
            stats.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.snn_rewire_deepr(r.handle, rep, stats)
            b.record()
            b.synchronize()
            if rep >= 3:
                times.append(a.elapsed_time(b))
                formed += int(stats[1])
        assert r.status() == abi.SNN_OK
        res[mode] = {"ms": round(sum(times) / len(times), 4), "formed_per_rewire": formed // len(times)}
        del keep
    return res


def main():
    args = parse()
    if args.workload != "classifier":
        fn = {"batched": run_batched, "serve": run_serve, "topo": run_topo, "topo-evolution": run_topo_evolution,
              "kernels": run_kernels}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return 0
    WORKLOAD["B"] = args.batch
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        if rank != 0:
            return 0
        # each timed step is one bounded sample: one trial of --sample-steps steps plus
        # the per-batch update (the oracle needs no warm-up)
        vals, last = [], None
        for _ in range(max(1, args.steps)):
            last = oracle_batch_sample(args.seed, args.sample_steps, 1)
            vals.append(last[0])
        v = sum(vals) / len(vals)
        cpu = cpu_info()
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(WORKLOAD["B"] / v * 1e3, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": classifier_config(last[2][0], last[2][1], world),
                "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": last[1], **cpu},
                "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    line = run_ours(args, world, rank, local)
    if rank == 0 and world == 1 and not args.no_systems:
        line["systems"] = systems_rows(args)
    if rank == 0 and args.no_cpu_baseline:
        print(json.dumps(line), flush=True)
    elif rank == 0:
        cv, desc, _, _ = oracle_batch_sample(args.seed, 1000, 1)
        line["cpu_baseline"] = {"value": round(cv, 5), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                **cpu_info()}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
