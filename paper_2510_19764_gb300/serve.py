"""Continuous-batching request loop for sparse spiking classifiers on one GPU.

Models (700 inputs -> N hidden ALIF -> 20 readouts, 10 % ragged connectivity, N in
256..2048) stay resident in device memory.  A request is a synthetic 700-channel spike
sequence (a class template, a time warp and a trial id for the Philox input stream) of
100-1000 steps; a fraction of requests are fine-tuning jobs that run one e-prop + L1 +
Adam + DEEP R step on a private copy of their model's weights.

Engine.run() is the serving loop.  Each pass it
  * admits requests that have arrived, while batch slots and the memory budget allow
    (each in-flight launch reserves the bytes of its buffers; a fine-tuning job takes a
    pre-allocated fine-tuning slot of its model, whose byte count is known before it
    starts),
  * groups admitted inference requests by model into one multi-trial forward launch
    (one CTA per trial, each trial stopping at its own length) on a free stream, so
    launches for different models — and new launches for a busy model — overlap on the
    device,
  * starts admitted fine-tuning jobs on their own stream: the slot's trainable copy is
    refreshed from the model's weights by device-to-device copies (no allocation, no
    handle creation and no synchronisation inside the loop), then trained,
  * polls completion events and records each request's latency (arrival to result on
    the host).
Results depend only on the request (integer spike accumulation, per-trial CTAs), so a
request's output is identical alone and in any mix (tests/test_gpu_serve.py).

The plain form serves one request at a time: launch, wait, next.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import abi, net

N_IN, K_OUT, N_CLASSES, N_BINS, T_MAX = 700, 20, 20, 10, 1000


class AdmissionError(RuntimeError):
    """A request can never be admitted (its slot or fine-tuning copy exceeds the budget)."""


@dataclass
class Request:
    rid: int
    model: int
    label: int
    T: int
    bin_len: int
    finetune: bool
    arrival: float = 0.0          # seconds on the serving clock


@dataclass
class Result:
    rid: int
    ysum: np.ndarray
    pred: int
    latency: float
    finetune: bool


def poisson_requests(n: int, rate_hz: float, n_models: int, seed: int = 0, finetune_frac: float = 0.1,
                     t_range=(100, 1000)) -> list[Request]:
    rng = np.random.default_rng([seed, 0x5E])
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    arrival = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        w = rng.uniform(0.8, 1.2)
        out.append(Request(i, int(rng.integers(0, n_models)), int(rng.integers(0, N_CLASSES)), T,
                           max(1, int(round(w * T / N_BINS))), bool(rng.random() < finetune_frac), float(arrival[i])))
    return out


class Model:
    """Resident weights of one served classifier."""

    def __init__(self, mid: int, N: int, task, device="cuda", p: float = 0.1, max_batch: int = 32):
        import synth
        self.mid, self.N, self.task, self.device = mid, N, task, device
        self.in_seed = 9003 + 7 * mid
        self.host_in = synth.random_ragged(9000 + 7 * mid, N_IN, N, p)
        self.host_rec = synth.random_ragged(9001 + 7 * mid, N, N, p, no_autapse=True)
        self.W_out, self.b = synth.dense_readout(9002 + 7 * mid, K_OUT, N)
        self.d_in = net.DeviceRagged(self.host_in.row_len, self.host_in.ind, self.host_in.w, N, device=device)
        self.d_rec = net.DeviceRagged(self.host_rec.row_len, self.host_rec.ind, self.host_rec.w, N,
                                      no_autapse=True, device=device)
        self.cls = net.DeviceClassifier(N_IN, N, K_OUT, self.d_in, self.d_rec, self.W_out, self.b, task.thr,
                                        9003 + 7 * mid, net.NeuronCfg(), max_B=max_batch, max_T=T_MAX, device=device)
        # the served weights do not change: pack the forward rows once, so that concurrent
        # launches of this model only read the handle's scratch
        abi.snn_classifier_pack(self.cls.handle, None)
        torch.cuda.synchronize()

    def private_copy(self):
        """Trainable copy (own ragged matrices, Adam state, DEEP R bitfields) for a
        fine-tuning job."""
        d_in = net.DeviceRagged(self.host_in.row_len, self.host_in.ind, self.host_in.w, self.N, adam=True, grad=True,
                                deepr=True, seed=9004 + 7 * self.mid, device=self.device)
        d_rec = net.DeviceRagged(self.host_rec.row_len, self.host_rec.ind, self.host_rec.w, self.N, no_autapse=True,
                                 adam=True, grad=True, deepr=True, seed=9005 + 7 * self.mid, device=self.device)
        cls = net.DeviceClassifier(N_IN, self.N, K_OUT, d_in, d_rec, self.W_out, self.b, self.task.thr,
                                   9003 + 7 * self.mid, net.NeuronCfg(), max_B=1, max_T=T_MAX, device=self.device)
        return cls


class _FineTuneSlot:
    """A model's pre-allocated fine-tuning copy: trainable ragged matrices with Adam
    moments and DEEP R bitfields, a classifier handle and one-trial buffers of T_MAX
    steps, plus the copy's initial contents (the model's weights with freshly initialised
    bitfields), which refresh() restores before each job."""

    def __init__(self, model: Model, device):
        self.model = model
        self.cls = model.private_copy()
        self.batch = net.DeviceBatch(self.cls, [0], [1], [0], T_MAX, device=device)
        self.h_ysum = torch.zeros((1, K_OUT), dtype=torch.float32).pin_memory()
        self.h_lab = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.h_bin = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.h_tid = torch.zeros(1, dtype=torch.int64).pin_memory()
        live = []
        for r in (self.cls.w_in, self.cls.w_rec):
            live += [r.row_len, r.ind, r.w, r.sign_bits, r.conn_bits]
        live += [self.cls.W_out, self.cls.b_out]
        self.live = live
        self.init = [t.clone() for t in live]
        self.zero = [t for r in (self.cls.w_in, self.cls.w_rec) for t in (r.m, r.v)] + \
            [self.cls.W_out_m, self.cls.W_out_v, self.cls.b_m, self.cls.b_v]
        tensors = live + self.init + self.zero + [getattr(self.batch, k) for k in (
            "v", "a", "y", "ysum", "x_bits", "z_bits", "x_rec", "z_rec", "psi_rec", "d_rec", "delta", "Dout")]
        tensors += [r.grad for r in (self.cls.w_in, self.cls.w_rec)] + [self.cls.G_out, self.cls.G_b]
        self.bytes = sum(t.numel() * t.element_size() for t in tensors)
        self.busy = False

    def refresh(self, stream):
        with torch.cuda.stream(stream):
            for dst, src in zip(self.live, self.init):
                dst.copy_(src, non_blocking=True)
            for t in self.zero:
                t.zero_()


class _BatchView:
    """A DeviceBatch descriptor with its own step count (what train_batch reads)."""

    def __init__(self, desc, T: int):
        self.desc, self.T = desc, T


class _Slot:
    """Reusable inference buffers for up to max_batch trials of one model."""

    def __init__(self, model: Model, max_batch: int, device):
        B = max_batch
        self.model = model
        self.batch = net.DeviceBatch(model.cls, np.zeros(B, np.int32), np.ones(B, np.int32), np.zeros(B, np.int64),
                                     T_MAX, device=device, workspace=False, records=False,
                                     trial_T=np.full(B, T_MAX, np.int32))
        self.h_lab = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.h_bin = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.h_tid = torch.zeros(B, dtype=torch.int64).pin_memory()
        self.h_T = torch.zeros(B, dtype=torch.int32).pin_memory()
        self.h_ysum = torch.zeros((B, K_OUT), dtype=torch.float32).pin_memory()
        self.bytes = sum(t.numel() * t.element_size() for t in (self.batch.x_rec, self.batch.z_rec, self.batch.v,
                                                                self.batch.a))
        self.busy = False


@dataclass
class _Flight:
    kind: str
    reqs: list
    event: torch.cuda.Event
    stream: torch.cuda.Stream
    slot: object = None
    cls: object = None
    batch: object = None
    h_ysum: object = None
    bytes: int = 0


class Engine:
    def __init__(self, models: list[Model], max_batch: int = 32, slots_per_model: int = 2, n_streams: int = 8,
                 mem_budget: int = 8 << 30, max_finetune: int = 4, device="cuda", ft_slots_per_model: int = 2):
        self.models = models
        self.max_batch = max_batch
        self.slots = {m.mid: [_Slot(m, max_batch, device) for _ in range(slots_per_model)] for m in models}
        # fine-tuning copies are created here, once: run() allocates nothing
        self.ft_slots = {m.mid: [_FineTuneSlot(m, device) for _ in range(ft_slots_per_model)] for m in models}
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.mem_budget = mem_budget
        self.max_finetune = max_finetune
        self.device = device
        self.stats = {"launches": 0, "max_in_flight": 0, "max_batch_seen": 0}

    # --- launches -----------------------------------------------------------
    def _launch_infer(self, slot: _Slot, reqs: list[Request], stream) -> _Flight:
        n = len(reqs)
        for k, r in enumerate(reqs):
            slot.h_lab[k], slot.h_bin[k], slot.h_tid[k], slot.h_T[k] = r.label, r.bin_len, r.rid, r.T
        bt = slot.batch
        Tmax = max(r.T for r in reqs)
        with torch.cuda.stream(stream):
            bt.labels[:n].copy_(slot.h_lab[:n], non_blocking=True)
            bt.bin_len[:n].copy_(slot.h_bin[:n], non_blocking=True)
            bt.trial_ids[:n].copy_(slot.h_tid[:n], non_blocking=True)
            bt.trial_T[:n].copy_(slot.h_T[:n], non_blocking=True)
            for t in (bt.v, bt.a, bt.y, bt.ysum, bt.x_bits, bt.z_bits):
                t[:n].zero_()
        desc = abi.Batch.from_buffer_copy(bt.desc)
        desc.B = n
        abi.snn_step_neurons_ex(slot.model.cls.handle, desc, 0, Tmax, abi.SNN_STEP_PACKED_READY, stream)
        with torch.cuda.stream(stream):
            slot.h_ysum[:n].copy_(bt.ysum[:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        slot.busy = True
        return _Flight("infer", reqs, ev, stream, slot=slot, h_ysum=slot.h_ysum, bytes=slot.bytes)

    def _launch_finetune(self, slot: _FineTuneSlot, r: Request, stream) -> _Flight:
        slot.refresh(stream)
        slot.h_lab[0], slot.h_bin[0], slot.h_tid[0] = r.label, r.bin_len, r.rid
        bt = slot.batch
        with torch.cuda.stream(stream):
            bt.labels.copy_(slot.h_lab, non_blocking=True)
            bt.bin_len.copy_(slot.h_bin, non_blocking=True)
            bt.trial_ids.copy_(slot.h_tid, non_blocking=True)
            for t in (bt.v, bt.a, bt.y, bt.ysum, bt.x_bits, bt.z_bits):
                t.zero_()
        desc = abi.Batch.from_buffer_copy(bt.desc)
        desc.T = r.T                       # one trial: its records are the first T rows of the buffers
        view = _BatchView(desc, r.T)
        net.train_batch(slot.cls, view, net.adam_params(1e-3, 1, l1=1e-5), r.rid, stream=stream)
        with torch.cuda.stream(stream):
            slot.h_ysum.copy_(bt.ysum, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        slot.busy = True
        return _Flight("finetune", [r], ev, stream, slot=slot, h_ysum=slot.h_ysum, bytes=slot.bytes)

    # --- serving loops ------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests` (arrival times in seconds from the start) with continuous
        batching.  realtime=False admits everything at once (for equality tests)."""
        pending: list[Request] = []
        queue = sorted(requests, key=lambda r: r.arrival)
        qi = 0
        flights: list[_Flight] = []
        results: list[Result] = []
        used = 0
        si = 0
        t_start = time.perf_counter()
        while qi < len(queue) or pending or flights:
            now = time.perf_counter() - t_start
            while qi < len(queue) and (not realtime or queue[qi].arrival <= now):
                pending.append(queue[qi])
                qi += 1
            # completions
            still = []
            for f in flights:
                if f.event.query():
                    done = time.perf_counter() - t_start
                    ys = f.h_ysum.numpy()
                    for k, r in enumerate(f.reqs):
                        y = ys[k].copy()
                        results.append(Result(r.rid, y, int(np.argmax(y)), done - (r.arrival if realtime else 0.0),
                                              r.finetune))
                    if f.slot is not None:
                        f.slot.busy = False
                    used -= f.bytes
                else:
                    still.append(f)
            flights = still
            # admissions
            if pending:
                rest = []
                n_ft = sum(1 for f in flights if f.kind == "finetune")
                by_model: dict[int, list[Request]] = {}
                for r in pending:
                    if r.finetune:
                        slot = next((x for x in self.ft_slots[r.model] if not x.busy), None)
                        if slot is not None and n_ft < self.max_finetune and used + slot.bytes <= self.mem_budget:
                            f = self._launch_finetune(slot, r, self.streams[si % len(self.streams)])
                            si += 1
                            n_ft += 1
                            used += f.bytes
                            flights.append(f)
                            self.stats["launches"] += 1
                        else:
                            rest.append(r)
                    else:
                        by_model.setdefault(r.model, []).append(r)
                for mid, reqs in by_model.items():
                    while reqs:
                        slot = next((s for s in self.slots[mid] if not s.busy), None)
                        if slot is None or used + slot.bytes > self.mem_budget:
                            rest.extend(reqs)
                            break
                        take, reqs = reqs[:self.max_batch], reqs[self.max_batch:]
                        f = self._launch_infer(slot, take, self.streams[si % len(self.streams)])
                        si += 1
                        used += f.bytes
                        flights.append(f)
                        self.stats["launches"] += 1
                        self.stats["max_batch_seen"] = max(self.stats["max_batch_seen"], len(take))
                pending = rest
                if pending and not flights:
                    # nothing in flight will free a slot or memory: these requests can never start
                    need = max(self.ft_slots[r.model][0].bytes if r.finetune else self.slots[r.model][0].bytes
                               for r in pending)
                    raise AdmissionError(f"{len(pending)} request(s) cannot be admitted: one needs {need} bytes "
                                         f"of device memory, the budget is {self.mem_budget} bytes")
            self.stats["max_in_flight"] = max(self.stats["max_in_flight"], len(flights))
            if not flights and qi < len(queue) and not pending and realtime:
                wait = queue[qi].arrival - (time.perf_counter() - t_start)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        return sorted(results, key=lambda x: x.rid)

    def run_plain(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """One request at a time, in arrival order: launch, wait for its result, next."""
        stream = self.streams[0]
        results = []
        t_start = time.perf_counter()
        for r in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                wait = r.arrival - (time.perf_counter() - t_start)
                if wait > 0:
                    time.sleep(wait)
            if r.finetune:
                f = self._launch_finetune(self.ft_slots[r.model][0], r, stream)
            else:
                slot = self.slots[r.model][0]
                f = self._launch_infer(slot, [r], stream)
            f.event.synchronize()
            if f.slot is not None:
                f.slot.busy = False
            done = time.perf_counter() - t_start
            y = f.h_ysum.numpy()[0].copy()
            results.append(Result(r.rid, y, int(np.argmax(y)), done - (r.arrival if realtime else 0.0), r.finetune))
        return sorted(results, key=lambda x: x.rid)


def latency_summary(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    return {"requests": len(results), "throughput_req_s": len(results) / wall if wall > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
