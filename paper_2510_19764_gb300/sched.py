"""Batched execution of many independent e-prop + DEEP R classifier instances.

Each instance is its own sparse ALIF classifier (700 inputs -> N hidden -> 20 readouts,
its own ragged matrices, connectivity and Philox seeds) training with one trial per
iteration and DEEP R after every trial.  Instances differ in hidden size and trial
length.  Three execution forms run the same device code:

* plain:   one instance after another on one stream, no graph: either one
           `snn_step_neurons` launch per simulated step (`per_step=True`) or one
           launch for the whole trial, then the gradient, Adam and DEEP R calls.
* graph:   the whole iteration of every instance (per-call launches) captured once in
           a CUDA graph over several streams and replayed.
* multi:   ONE persistent kernel launch per iteration (`snn_multi_run`): a device work
           queue of (instance, phase, item) entries that all CTAs of the GPU drain; an
           instance's phases (inputs, forward, readout scan, adjoint, gather, Adam, DEEP
           R) follow one another while the instances interleave.  Iterations can be
           captured in a CUDA graph as well.

Everything that changes between iterations (trial id, label, time warp, Adam's step,
the DEEP R rewiring index) is derived on the device from the instance's iteration
counter, so all forms give bit-identical results (tests/test_gpu_sched.py).

The row schedule of the forward (how a trial's warps share the spiking rows of a step)
is picked per (hidden size, mean row length, spike rate) class by `Autotuner`, which
times the candidate schedules on a sample trial of a representative instance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import abi, net

N_IN, K_OUT, N_CLASSES, N_BINS = 700, 20, 20, 10


@dataclass
class InstanceSpec:
    N: int
    T: int
    p: float
    seed: int


def batched_specs(n: int = 64, seed: int = 0) -> list[InstanceSpec]:
    """Hidden sizes uniform over {256, 512, 1024, 2048}, trial lengths uniform in
    [200, 1000], connectivity uniform in [5 %, 20 %]."""
    rng = np.random.default_rng([seed, 0x5C4E])
    out = []
    for i in range(n):
        out.append(InstanceSpec(int(rng.choice([256, 512, 1024, 2048])), int(rng.integers(200, 1001)),
                                float(rng.uniform(0.05, 0.20)), seed * 1000 + i))
    return out


class Instance:
    """One classifier with its training state and device-resident iteration counters."""

    def __init__(self, spec: InstanceSpec, task, device="cuda", lr: float = 1e-3, l1: float = 1e-5,
                 temperature: float = 0.0):
        import synth
        self.spec = spec
        N, T, p, sd = spec.N, spec.T, spec.p, spec.seed
        in_rag = synth.random_ragged(sd * 7 + 1, N_IN, N, p)
        rec_rag = synth.random_ragged(sd * 7 + 2, N, N, p, no_autapse=True)
        W_out, b = synth.dense_readout(sd * 7 + 3, K_OUT, N)
        F32 = abi.SNN_F32
        self.d_in = net.DeviceRagged(in_rag.row_len, in_rag.ind, in_rag.w, N, dtype=F32, adam=True, grad=True,
                                     deepr=True, seed=sd * 7 + 4, device=device)
        self.d_rec = net.DeviceRagged(rec_rag.row_len, rec_rag.ind, rec_rag.w, N, dtype=F32, no_autapse=True,
                                      adam=True, grad=True, deepr=True, seed=sd * 7 + 5, device=device)
        self.cls = net.DeviceClassifier(N_IN, N, K_OUT, self.d_in, self.d_rec, W_out, b, task.thr, sd * 7 + 6,
                                        net.NeuronCfg(), max_B=1, max_T=T, dtype=F32, device=device)
        rng = np.random.default_rng([sd, 0xB1])
        self.bin_table = torch.as_tensor(
            np.maximum(1, np.rint(rng.uniform(0.8, 1.2, 64) * T / N_BINS)).astype(np.int32), device=device)
        self.batch = net.DeviceBatch(self.cls, [0], [int(self.bin_table[0])], [0], T, device=device)
        self.label_table = torch.arange(N_CLASSES, dtype=torch.int32, device=device)
        self.step = torch.zeros(1, dtype=torch.int64, device=device)          # iterations done
        self.adam_t = torch.zeros(1, dtype=torch.int64, device=device)        # Adam step count of this iteration
        self.stats = torch.zeros((2, 4), dtype=torch.int64, device=device)
        # DEEP R noise (temperature > 0) draws with the iteration counter as Philox field
        self.adam = net.adam_params(lr, 1, l1=l1, step_dev=self.adam_t, temperature=temperature,
                                    noise_idx_dev=self.step)
        self.lr, self.l1 = lr, l1
        self.events = 0

    def _prologue(self):
        """Device-side bookkeeping of one iteration: trial id = iteration index, label and
        time warp from it, Adam step count advanced, state reset."""
        bt = self.batch
        bt.trial_ids.copy_(self.step)
        bt.labels.copy_(self.label_table.index_select(0, self.step % self.label_table.numel()))
        bt.bin_len.copy_(self.bin_table.index_select(0, self.step % self.bin_table.numel()))
        self.adam_t.copy_(self.step + 1)
        for t in (bt.v, bt.a, bt.y, bt.ysum, bt.x_bits, bt.z_bits):
            t.zero_()

    def enqueue(self, stream, per_step: bool = False):
        """Launch one training iteration on `stream` (torch stream)."""
        with torch.cuda.stream(stream):
            self._prologue()
        h, bt = self.cls.handle, self.batch.desc
        if per_step:
            for t in range(self.spec.T):
                abi.snn_step_neurons(h, bt, t, 1, stream)
        else:
            abi.snn_step_neurons(h, bt, 0, self.spec.T, stream)
        abi.snn_eprop_update(h, bt, abi.SNN_EPROP_GRAD, None, stream)
        abi.snn_eprop_update(h, bt, abi.SNN_EPROP_APPLY, self.adam, stream)
        abi.snn_rewire_deepr_dev(self.d_in.handle, self.step, self.stats[0], stream)
        abi.snn_rewire_deepr_dev(self.d_rec.handle, self.step, self.stats[1], stream)
        with torch.cuda.stream(stream):
            self.step.add_(1)

    def multi_instance(self) -> abi.MultiInstance:
        """This instance's entry of a persistent multi-instance plan (same iteration
        semantics as enqueue)."""
        m = abi.MultiInstance()
        m.cls = self.cls.handle
        m.batch = self.batch.desc
        m.label_table, m.n_label = abi.ptr(self.label_table), self.label_table.numel()
        m.bin_table, m.n_bin = abi.ptr(self.bin_table), self.bin_table.numel()
        m.iter = abi.ptr(self.step)
        m.lr, m.beta1, m.beta2, m.eps = self.adam.lr, self.adam.beta1, self.adam.beta2, self.adam.eps
        m.l1, m.temperature = self.adam.l1, self.adam.temperature
        m.stats = abi.ptr(self.stats)
        return m

    def snapshot(self) -> dict:
        out = {}
        for name, d in (("in", self.d_in), ("rec", self.d_rec)):
            h = d.host()
            out[name] = {k: h[k] for k in ("row_len", "ind", "w", "conn_bits")}
        out["W_out"] = self.cls.W_out.cpu().numpy()
        out["ysum"] = self.batch.ysum.cpu().numpy()
        return out


class PlainRunner:
    """One instance at a time on one stream, no graph: per-step forward launches
    (per_step=True) or one forward launch per trial."""

    def __init__(self, instances, stream=None, per_step: bool = True):
        self.instances = instances
        self.stream = stream or torch.cuda.current_stream()
        self.per_step = per_step

    def iterate(self):
        for inst in self.instances:
            inst.enqueue(self.stream, per_step=self.per_step)


class BatchedRunner:
    """All instances' iterations captured in one CUDA graph over `n_streams` streams."""

    def __init__(self, instances, n_streams: int = 16):
        self.instances = instances
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.graph = None

    def capture(self):
        main = torch.cuda.Stream()
        # warm-up outside capture: first calls set kernel attributes and build tables
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=main):
            for s in self.streams:
                s.wait_stream(main)
            for i, inst in enumerate(self.instances):
                inst.enqueue(self.streams[i % len(self.streams)])
            for s in self.streams:
                main.wait_stream(s)
        self.graph = g

    def iterate(self):
        self.graph.replay()


class MultiRunner:
    """All instances' iterations in one persistent kernel launch each (snn_multi_run);
    capture() puts `n_iter` such launches into one CUDA graph."""

    def __init__(self, instances, wait_limit_ns: int = 2_000_000_000):
        self.instances = instances
        self.handle = abi.snn_multi_create([inst.multi_instance() for inst in instances])
        self.wait_limit_ns = wait_limit_ns
        self.graph = None
        self.graph_iters = 0

    PHASES = ("prep", "inputs+sums", "pack", "forward+sort", "readout_scan", "adjoint", "gather", "adam",
              "deepr_elim", "deepr_dist", "deepr_form")

    def iterate(self, stream=None, flags: int = 0):
        abi.snn_multi_run(self.handle, flags, self.wait_limit_ns, stream or torch.cuda.current_stream())

    def trace(self) -> "PhaseTrace":
        """Record the phase completion times of the following runs (PhaseTrace.summary()
        reads them after a run)."""
        t = PhaseTrace(len(self.instances))
        abi.snn_multi_set_trace(self.handle, t.times)
        return t

    def capture(self, n_iter: int = 1):
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(n_iter):
                abi.snn_multi_run(self.handle, 0, self.wait_limit_ns, s)
        self.graph, self.graph_iters = g, n_iter

    def replay(self):
        self.graph.replay()

    def status(self, stream=None) -> int:
        return abi.snn_multi_status(self.handle, stream)

    def close(self):
        if self.handle:
            abi.snn_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PhaseTrace:
    """Global-timer stamps of one persistent run: per instance its start and the end of
    each phase (device int64 [n][12])."""

    def __init__(self, n: int):
        self.times = torch.zeros((n, len(MultiRunner.PHASES) + 1), dtype=torch.int64, device="cuda")

    def summary(self, instances) -> dict:
        t = self.times.cpu().numpy().astype(np.float64)
        t0 = t[:, 0].min()
        end = t[:, -1] - t0
        slow = int(np.argmax(end))
        step = np.diff(t[slow]) / 1e3
        return {"iteration_ms": round(float(end.max()) / 1e6, 3),
                "slowest_instance": {"N": instances[slow].spec.N, "T": instances[slow].spec.T,
                                     "p": round(instances[slow].spec.p, 3),
                                     "phase_us": {k: round(float(v), 1) for k, v in zip(MultiRunner.PHASES, step)}},
                "median_instance_ms": round(float(np.median(end)) / 1e6, 3)}


class Autotuner:
    """Row-schedule table keyed on (hidden size, mean row length, spike rate): for each
    class, time a representative instance with every admissible schedule and keep the
    fastest.  target="plain": the per-call forward of one trial for every (warps per
    trial, row schedule) pair; target="multi": one-instance runs of the persistent
    kernel (8 warps per trial) for every row schedule, the wide ones included."""

    MODES = (abi.SNN_ROWS_PAIRS, abi.SNN_ROWS_PER_WARP, abi.SNN_ROWS_PER_BLOCK)
    MULTI_MODES = MODES + (abi.SNN_ROWS_WIDE, abi.SNN_ROWS_QUAD)

    def __init__(self, warps=(4, 8, 16), target: str = "plain"):
        assert target in ("plain", "multi")
        self.warps = tuple(warps) if target == "plain" else (8,)
        self.target = target
        self.table: dict[tuple, tuple] = {}
        self.timings: dict[tuple, dict] = {}

    @staticmethod
    def key(inst: Instance, spike_rate: float) -> tuple:
        mean_len = float(inst.d_in.row_len.float().mean() + inst.d_rec.row_len.float().mean()) / 2
        return (inst.spec.N, int(round(math.log2(max(mean_len, 1.0)))), int(round(math.log2(max(spike_rate, 1e-4)))))

    @staticmethod
    def spike_rate(inst: Instance) -> float:
        z = net.spikes_from_bits(inst.batch.z_rec[0].cpu().numpy().view(np.uint32), inst.spec.N)
        return float(z.mean())

    @staticmethod
    def _apply(inst: Instance, choice: tuple):
        abi.snn_classifier_set_schedule(inst.cls.handle, choice[0])
        abi.snn_classifier_set_row_schedule(inst.cls.handle, choice[1])

    def _time(self, inst: Instance, choice: tuple, reps: int = 3) -> float:
        self._apply(inst, choice)
        s = torch.cuda.current_stream()
        best = float("inf")
        if self.target == "multi":
            mr = MultiRunner([inst])             # the plan reads the schedule when created
            mr.iterate(s)
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                mr.iterate(s)
                b.record(s)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            mr.close()
            return best
        for _ in range(reps):
            for t in (inst.batch.v, inst.batch.a, inst.batch.y, inst.batch.ysum, inst.batch.x_bits,
                      inst.batch.z_bits):
                t.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            abi.snn_step_neurons(inst.cls.handle, inst.batch.desc, 0, inst.spec.T, s)
            b.record(s)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    def tune(self, instances) -> dict:
        modes = self.MULTI_MODES if self.target == "multi" else self.MODES
        for inst in instances:
            # a sample trial at the default schedule gives the spike rate of the class
            self._time(inst, (8, abi.SNN_ROWS_PAIRS), reps=1)
            k = self.key(inst, self.spike_rate(inst))
            if k not in self.table:
                times = {(w, mode): self._time(inst, (w, mode)) for w in self.warps for mode in modes
                         if inst.spec.N <= 8 * 32 * w}
                self.table[k] = min(times, key=times.get)
                self.timings[k] = times
            self._apply(inst, self.table[k])
        return self.table
