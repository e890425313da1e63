"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no arithmetic of the structural-plasticity method itself: it only
draws the *inputs* a user would bring (rate templates, trial labels and time warps,
initial ragged connectivity and weights, initial topographic connectivity) from
numpy's seeded generator. Everything the method computes from these inputs (Poisson
spike decisions, neuron dynamics, e-prop, Adam, DEEP R, STDP, rewiring) lives in
`oracle/` (FP64 reference) and in the CUDA library, independently.

Shapes follow the paper's workloads:
* classifier inputs: per-class, per-channel rate templates (Sec. 2.2.1 trains on
  N-MNIST / DVS gesture; spoken-digit-like 700-channel inputs stand in for them),
* sparse ragged matrices at a fixed connection probability (Sec. 2.2.1, "fixed
  probability of connection between each pair"), rows padded to a capacity
  (Sec. 2.1, Fig. 1),
* topographic sheets on a periodic square grid initialised by the pairwise-Bernoulli
  rule with the Gaussian formation probability (Sec. 2.2.2, Tab. 1-2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO32 = float(2 ** 32)


def rate_threshold(p: float) -> int:
    """Encode a per-step spike probability p as a 32-bit threshold.

    A 32-bit Philox draw h fires iff h < thr.  thr = floor(p * 2^32) for p < 1,
    saturated at 2^32 - 1 for p >= 1 and 0 for p <= 0.  p * 2^32 is an exact
    power-of-two scaling of the double p, so the conversion is exact.
    """
    if p <= 0.0:
        return 0
    if p >= 1.0:
        return (1 << 32) - 1
    return int(p * TWO32)


def rates_to_thresholds(rates_hz: np.ndarray, dt_ms: float) -> np.ndarray:
    """uint32 thresholds of per-step spike probabilities rate * dt."""
    flat = [rate_threshold(float(r) * dt_ms * 1e-3) for r in np.asarray(rates_hz, dtype=np.float64).ravel()]
    return np.array(flat, dtype=np.uint32).reshape(np.shape(rates_hz))


# --------------------------------------------------------------------------------------
# Classifier inputs
# --------------------------------------------------------------------------------------

@dataclass
class ClassifierTask:
    """Rate templates [n_classes][n_bins][n_in] (Hz) and their spike thresholds."""
    rates_hz: np.ndarray
    thr: np.ndarray          # uint32 Bernoulli thresholds, same shape
    n_classes: int
    n_bins: int
    n_in: int
    T: int
    dt_ms: float


def tiny_task(seed: int = 0, n_in: int = 32, n_classes: int = 4, T: int = 200,
              max_rate_hz: float = 40.0, dt_ms: float = 1.0) -> ClassifierTask:
    """Tiny 4-class task: each class has a fixed per-channel rate drawn U[0, 40) Hz
    (20 Hz mean), constant over the trial (one time bin)."""
    rng = np.random.default_rng([seed, 0xC0])
    rates = rng.uniform(0.0, max_rate_hz, size=(n_classes, 1, n_in))
    return ClassifierTask(rates, rates_to_thresholds(rates, dt_ms), n_classes, 1, n_in, T, dt_ms)


def spoken_digit_task(seed: int = 0, n_in: int = 700, n_classes: int = 20, T: int = 1000,
                      n_bins: int = 10, max_rate_hz: float = 50.0, dt_ms: float = 1.0) -> ClassifierTask:
    """Spoken-digit-shaped task: 20 classes x 10 time bins x 700 channels of
    log-normal rates (median 8 Hz) clipped to [0, 50] Hz."""
    rng = np.random.default_rng([seed, 0xC1])
    rates = np.minimum(max_rate_hz, np.exp(rng.normal(math.log(8.0), 1.0, size=(n_classes, n_bins, n_in))))
    return ClassifierTask(rates, rates_to_thresholds(rates, dt_ms), n_classes, n_bins, n_in, T, dt_ms)


@dataclass
class TrialBatch:
    labels: np.ndarray      # int32 [B]
    bin_len: np.ndarray     # int32 [B] steps per template bin (time warp)
    trial_ids: np.ndarray   # int64 [B] global trial index (Philox counter field)


def trial_batch(task: ClassifierTask, seed: int, batch_idx: int, B: int,
                warp: tuple[float, float] = (0.8, 1.2)) -> TrialBatch:
    """Labels uniform over classes; each trial draws a time warp w ~ U[warp] and
    its template bins last round(w * T / n_bins) steps (>= 1)."""
    rng = np.random.default_rng([seed, 0xB0, batch_idx])
    labels = rng.integers(0, task.n_classes, size=B).astype(np.int32)
    if task.n_bins == 1:
        bin_len = np.full(B, task.T, dtype=np.int32)
    else:
        w = rng.uniform(warp[0], warp[1], size=B)
        bin_len = np.maximum(1, np.rint(w * task.T / task.n_bins)).astype(np.int32)
    trial_ids = (np.int64(batch_idx) * B + np.arange(B, dtype=np.int64)).astype(np.int64)
    return TrialBatch(labels, bin_len, trial_ids)


def round_up(x: int, m: int) -> int:
    return ((x + m - 1) // m) * m


@dataclass
class Ragged:
    """Host copy of a ragged matrix: row = presynaptic neuron, slot s < row_len."""
    P: int
    Q: int
    C: int
    row_len: np.ndarray   # int32 [P]
    ind: np.ndarray       # int32 [P, C] (padding slots hold -1)
    w: np.ndarray         # float64 [P, C] (padding slots hold 0)


def random_ragged(seed: int, P: int, Q: int, p: float, C: int | None = None,
                  no_autapse: bool = False, w_std: float | None = None,
                  capacity_factor: float = 2.0, align: int = 32) -> Ragged:
    """Each (i, j) pair connected independently with probability p; targets kept in a
    shuffled (unsorted) order; weights N(0, w_std) with w_std = 1/sqrt(p * fan-in pool)
    by default.  Capacity defaults to roundup(capacity_factor * max initial row length)."""
    rng = np.random.default_rng([seed, 0xAA, P, Q])
    mask = rng.random((P, Q)) < p
    if no_autapse:
        k = min(P, Q)
        mask[np.arange(k), np.arange(k)] = False
    rows = [rng.permutation(np.nonzero(mask[i])[0]) for i in range(P)]
    maxlen = max((len(r) for r in rows), default=0)
    if C is None:
        C = max(align, round_up(int(math.ceil(capacity_factor * max(maxlen, 1))), align))
    if w_std is None:
        pool = (P - 1) if no_autapse else P
        w_std = 1.0 / math.sqrt(max(p * pool, 1e-12))
    row_len = np.zeros(P, dtype=np.int32)
    ind = np.full((P, C), -1, dtype=np.int32)
    w = np.zeros((P, C), dtype=np.float64)
    for i, r in enumerate(rows):
        r = r[:C]
        row_len[i] = len(r)
        ind[i, :len(r)] = r
        w[i, :len(r)] = rng.normal(0.0, w_std, size=len(r))
    return Ragged(P, Q, C, row_len, ind, w)


def large_ragged(seed: int, P: int, Q: int, k: int, C: int, w_std: float = 1.0) -> Ragged:
    """Large random ragged matrix for bandwidth measurements: each row draws k targets
    uniformly with replacement and keeps the distinct ones (about k - k^2/(2Q)), in
    ascending order; weights N(0, w_std) in float32-representable values."""
    rng = np.random.default_rng([seed, 0x1A, P, Q, k])
    t = np.sort(rng.integers(0, Q, size=(P, k), dtype=np.int64), axis=1)
    keep = np.ones_like(t, dtype=bool)
    keep[:, 1:] = t[:, 1:] != t[:, :-1]
    row_len = keep.sum(axis=1).astype(np.int32)
    assert int(row_len.max()) <= C
    pos = np.cumsum(keep, axis=1) - 1
    ind = np.full((P, C), -1, dtype=np.int32)
    rows = np.nonzero(keep)
    ind[rows[0], pos[rows]] = t[rows]
    w = np.zeros((P, C), dtype=np.float64)
    live = np.arange(C)[None, :] < row_len[:, None]
    w[live] = rng.normal(0.0, w_std, size=int(live.sum())).astype(np.float32)
    return Ragged(P, Q, C, row_len, ind, w)


def dense_readout(seed: int, K: int, N: int) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng([seed, 0xD0, K, N])
    return rng.normal(0.0, 1.0 / math.sqrt(N), size=(K, N)), np.zeros(K)


# --------------------------------------------------------------------------------------
# Topographic map inputs
# --------------------------------------------------------------------------------------

def torus_d2(a: np.ndarray, b: np.ndarray, L: int) -> np.ndarray:
    """Squared Euclidean distance between flat grid indices on an L x L torus."""
    ax, ay = a % L, a // L
    bx, by = b % L, b // L
    dx = np.abs(ax - bx)
    dy = np.abs(ay - by)
    dx = np.minimum(dx, L - dx)
    dy = np.minimum(dy, L - dy)
    return dx * dx + dy * dy


def topo_initial(seed: int, L: int, p_form: float, sigma: float, C: int, g_init: float,
                 allow_autapse: bool = True) -> Ragged:
    """Pairwise-Bernoulli initial connectivity: pair (i, j) connected with probability
    p_form * exp(-d^2 / (2 sigma^2)) (torus distance), rows capped at C."""
    rng = np.random.default_rng([seed, 0x70, L])
    N = L * L
    idx = np.arange(N)
    row_len = np.zeros(N, dtype=np.int32)
    ind = np.full((N, C), -1, dtype=np.int32)
    w = np.zeros((N, C), dtype=np.float64)
    for i in range(N):
        d2 = torus_d2(np.full(N, i), idx, L)
        prob = p_form * np.exp(-d2 / (2.0 * sigma * sigma))
        m = rng.random(N) < prob
        if not allow_autapse:
            m[i] = False
        tg = rng.permutation(np.nonzero(m)[0])[:C]
        row_len[i] = len(tg)
        ind[i, :len(tg)] = tg
        w[i, :len(tg)] = g_init
    return Ragged(N, N, C, row_len, ind, w)
