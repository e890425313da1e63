// Device code of the classifier (Sec. 2.2.1 of the paper) shared by the per-call kernels
// (classifier.cu) and the persistent multi-instance kernel (multi.cu): every kernel body
// is a device function over an explicit block / warp / element index, so both launch
// forms run the same statements and give bit-identical results.  The comments of
// classifier.cu describe the method; those here describe each piece.
#pragma once

#include "common.cuh"

namespace snn {

constexpr int BWD_THREADS = 128;

template <typename real>
struct FwdParams {
    int n_in, N, K, Win, Wh, T, t0, n_steps;
    real alpha, rho, beta, v_thr, psi_scale, inv_vthr;
    const int32_t* in_len;
    const int32_t* rec_len;
    const unsigned long long* pk;   // packed rows (see k_pack), Cf slots each
    int Cf;
    const real* b_out;
    real* v;
    real* a;
    real* y;
    real* ysum;
    uint32_t* x_bits;
    uint32_t* z_bits;
    const uint32_t* x_rec;
    uint32_t* z_rec;
    real* psi_rec;
    real* d_rec;
    real* v_rec;
    real* a_rec;
    real* y_rec;
    int record_state;
    const int32_t* trial_T;   // per-trial lengths or NULL
    const unsigned long long* colsum;   // [N + 64] |weight| sums per accumulator (k_pack)
    int32_t* status;
    int sched;                // phase A row schedule: SNN_ROWS_PAIRS, SNN_ROWS_PER_WARP or SNN_ROWS_PER_BLOCK
};

// An accumulator's sums are exact while their magnitude stays below 2^11 (2^51 in fixed
// point); the sum of |weight| over every slot aimed at it bounds any step's sum.
constexpr unsigned long long FIX_SUM_LIMIT = 1ull << 51;

struct InputParams {
    int n_in, Win, T, t0, n_steps, n_bins, n_classes, B;
    const int32_t* trial_T;
    const uint32_t* in_thr;
    uint64_t seed;
    const int32_t* labels;
    const int32_t* bin_len;
    const int64_t* trial_ids;
    uint32_t* x_rec;
    int32_t* status;
};

__device__ __forceinline__ float exp_real(float x) { return expf(x); }
__device__ __forceinline__ double exp_real(double x) { return exp(x); }

// Forward accumulators, FP64 build (wide slots): each is a pair of 32-bit words {H, L}
// summing the two parts of every added fixed-point weight w = 2^20 w_hi + w_lo (w_hi =
// bits 51..20 of the packed slot as a signed 32-bit value, w_lo = bits 19..0): both sums
// use native 32-bit shared-memory atomics and are exact: L takes at most one addend
// (< 2^20) per spiking row, rows hold no repeated target and n_in + N <= 3072 < 4096; H
// wraps modulo 2^32 like the 52-bit weights.  The total is 2^20 H + L.  The H words of
// all accumulators come first, then the L words (NA apart), so that lanes adding to
// consecutive targets hit consecutive banks: interleaved pairs would put every H word on
// an even bank and double the shared-memory wavefronts of a warp's scattered additions.
//
// FP32 build (narrow slots): one 32-bit word per accumulator and one atomic per slot.
// Accumulator t has its own grid 2^(sh_t - 40), sh_t = max(0, e_t - 30) with e_t the bit
// length of its |weight| sum in fixed point (40 fractional bits); each slot holds its
// weight rounded to its target's grid, so |any step's sum| <= 2^30 + 3072 / 2 < 2^31 and
// the 32-bit integer sums are exact on that grid.  A weight is off by at most half a grid
// step, C_t 2^-30 for an incoming |weight| sum C_t (1.3e-8 at C_t = 14): below the FP32
// rounding of the membrane update's operands at these magnitudes.  The slot carries the
// target's byte offset, so an addition is one integer add and one atomic.
template <bool NARROW>
__device__ __forceinline__ void acc_add(unsigned* acc, unsigned long long w, int NA) {
    const unsigned lo = (unsigned)w, hi = (unsigned)(w >> 32);
    if (NARROW) {
        atomicAdd((unsigned*)((char*)acc + hi), lo);          // bits 63..32: byte offset
    } else {
        unsigned* a = acc + (hi >> 20);                       // target index: bits 63..52
        atomicAdd(a, __funnelshift_r(lo, hi, 20));            // bits 51..20
        atomicAdd(a + NA, lo & 0xFFFFFu);                     // bits 19..0
    }
}
// The accumulated sum of accumulator a in real units.  Wide: 2^20 H + L (L at a + NA),
// H 2^-20 + L 2^-40, each product exact, one rounding in the sum (for double the same
// value as converting the 64-bit integer first).  Narrow: the 32-bit sum times its grid
// step `scale` (a power of two: one rounding).
template <bool NARROW, typename real>
__device__ __forceinline__ real acc_real(const unsigned* a, int NA, real scale) {
    if (NARROW) return (real)(int)a[0] * scale;
    return (real)(int)a[0] * (real)9.5367431640625e-07 + (real)a[NA] * (real)9.094947017729282e-13;
}
// Clears accumulator a.
template <bool NARROW>
__device__ __forceinline__ void acc_zero(unsigned* a, int NA) {
    a[0] = 0u;
    if (!NARROW) a[NA] = 0u;
}
// Narrow grid of an accumulator from its |weight| sum cs (fixed point): the shift sh and
// the grid step 2^(sh - 40) as a float (exact).
__device__ __forceinline__ int narrow_shift(unsigned long long cs) {
    const int e = 64 - __clzll((long long)cs);
    return e > 30 ? e - 30 : 0;
}
__device__ __forceinline__ float narrow_scale(unsigned long long cs) {
    return __int_as_float((127 - 40 + narrow_shift(cs)) << 23);
}

// Input spikes of every (trial, step) in parallel: they depend on (trial, step, channel)
// only, so they are drawn ahead of the sequential simulation.  Thread = 8 channels (one
// Philox block, one 32-bit half of a word per channel); the bytes of 4 consecutive
// threads form one 32-channel word.
__device__ __forceinline__ void input_group(const InputParams& p, const long long g) {
    const int G = p.Win * 4;
    const long long total = (long long)p.B * p.n_steps * G;
    uint32_t byte = 0;
    int gi = (int)(g % G);
    long long bt = g / G;
    if (g < total) {
        const int b = (int)(bt / p.n_steps);
        const int t = p.t0 + (int)(bt % p.n_steps);
        int label = p.labels[b], bin_len = p.bin_len[b];
        if (label < 0 || label >= p.n_classes || bin_len < 1) {
            if (gi == 0) atomicOr(p.status, ST_STATE);
            label = min(max(label, 0), p.n_classes - 1);
            bin_len = max(bin_len, 1);
        }
        if (8 * gi < p.n_in && (!p.trial_T || t < p.trial_T[b])) {
            const int bin = min(p.n_bins - 1, t / bin_len);
            const uint32_t* thr = p.in_thr + ((size_t)label * p.n_bins + bin) * p.n_in;
            const u64x4 r = philox(p.seed, PH_INPUT, (uint64_t)p.trial_ids[b], (uint64_t)t, (uint64_t)gi, 0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * gi + q;
                const uint32_t h = (uint32_t)(r[q >> 1] >> (32 * (q & 1)));
                if (c < p.n_in && h < thr[c]) byte |= 1u << q;
            }
        }
    }
    uint32_t word = byte << (8 * (gi & 3));
    word |= __shfl_xor_sync(0xffffffffu, word, 1);
    word |= __shfl_xor_sync(0xffffffffu, word, 2);
    if (g < total && (gi & 3) == 0) {
        const int b = (int)(bt / p.n_steps);
        const int t = p.t0 + (int)(bt % p.n_steps);
        p.x_rec[((size_t)b * p.T + t) * p.Win + (gi >> 2)] = word;
    }
}

// One CTA = one trial, all requested steps.  Spiking rows are kept as explicit lists
// (global row ids: input rows 0..n_in-1, hidden rows n_in + j), double-buffered by step
// parity and built where the spikes appear: hidden spikes are appended with one
// warp-aggregated shared-memory atomic per warp during the neuron update, the input
// spikes of step t (drawn ahead of time by k_input) are listed by warp 0.  Per step t:
//  (A) warps take every nwarps-th row of the lists of step t-1, FWD_ROWS at a time; each
//      slot is one packed 64-bit load (target index | fixed-point weight) and one
//      pair of 32-bit shared-memory atomics (padding slots of a row's last chunk add 0
//      to per-lane spare accumulators).  Hidden rows carry their readout column as K
//      extra slots aimed at the readout accumulators, so W_out z^{t-1} is summed by the
//      same loop.  The accumulated sums are exact while they stay below 2^11 in
//      magnitude (see acc_add).
//  (B) each thread updates its NPT neurons (state in registers) and writes psi; warp 1
//      advances the leaky readout y^t = alpha y^{t-1} + W_out z^{t-1} + b (one lane per
//      output, sequential in t) and records y^t into the d record (softmax comes later).
constexpr int FWD_ROWS = 2;   // spiking rows a warp propagates at a time (default schedule)
constexpr int FWD_CHUNKS = 5; // 32-slot chunks of each row loaded together (default schedule):
                              // a hidden row's synapses plus its readout column often pass 128

// Phase A row schedules (all add the same integers, so the sums do not depend on them).
// Row per warp: warp w takes rows w, w + nwarps, ... of the spike list, FR rows at a time,
// their blocks of CH 32-slot chunks loaded together (FR = 2, CH = 5: SNN_ROWS_PAIRS;
// 1, 4: SNN_ROWS_PER_WARP; 2, 8: SNN_ROWS_WIDE for long rows; 4, 4: SNN_ROWS_QUAD).  The
// wide forms hold 16 loads per lane in flight (fewer round trips per step, more
// registers: they suit the persistent kernel, whose CTAs have room for them).
template <bool NARROW, int FR, int nwarps, int CH = 4>
__device__ __forceinline__ void propagate_rows_warp(unsigned* acc, int NA, const int* lprv, int n_rows,
                                                    const int* lens, const unsigned long long* pk, int Cf, int R,
                                                    int warp, int lane) {
    for (int k = warp; k < n_rows; k += FR * nwarps) {
        int nr[FR];
        const unsigned long long* pr[FR];
        int nmax = 0;
#pragma unroll
        for (int u = 0; u < FR; ++u) {
            const int r = (k + u * nwarps < n_rows) ? lprv[k + u * nwarps] : R;   // R: empty row
            nr[u] = lens[r];
            pr[u] = pk + (size_t)(r < R ? r : 0) * Cf;
            nmax = nr[u] > nmax ? nr[u] : nmax;
        }
        for (int s0 = 0; s0 < nmax; s0 += 32 * CH) {
            unsigned long long wv[FR][CH];
#pragma unroll
            for (int q = 0; q < CH; ++q)
#pragma unroll
                for (int u = 0; u < FR; ++u)   // warp-uniform chunk tests; slots past a
                    wv[u][q] = s0 + q * 32 < nr[u] ? pr[u][s0 + q * 32 + lane] : 0ull;   // length are padding
#pragma unroll
            for (int q = 0; q < CH; ++q)
#pragma unroll
                for (int u = 0; u < FR; ++u)
                    if (s0 + q * 32 < nr[u]) acc_add<NARROW>(acc, wv[u][q], NA);
        }
    }
}

// Row per block: every warp works on every spiking row, warp w taking the row's 32-slot
// chunks w, w + nwarps, ...; two rows in flight (suits few long rows).
template <bool NARROW, int nwarps>
__device__ __forceinline__ void propagate_rows_block(unsigned* acc, int NA, const int* lprv, int n_rows,
                                                     const int* lens,
                                                     const unsigned long long* pk, int Cf, int warp, int lane) {
    for (int k = 0; k < n_rows; k += 2) {
        const int r0 = lprv[k];
        const int r1 = k + 1 < n_rows ? lprv[k + 1] : -1;
        const int n0 = lens[r0], n1 = r1 >= 0 ? lens[r1] : 0;
        const unsigned long long* p0 = pk + (size_t)r0 * Cf;
        const unsigned long long* p1 = pk + (size_t)(r1 >= 0 ? r1 : 0) * Cf;
        const int nmax = n0 > n1 ? n0 : n1;
        for (int s0 = warp * 32; s0 < nmax; s0 += nwarps * 32) {
            const unsigned long long a = s0 < n0 ? p0[s0 + lane] : 0ull;
            const unsigned long long b = s0 < n1 ? p1[s0 + lane] : 0ull;
            if (s0 < n0) acc_add<NARROW>(acc, a, NA);
            if (s0 < n1) acc_add<NARROW>(acc, b, NA);
        }
    }
}

// WIDE: compile the register-hungry row schedules in (the persistent kernel); without
// them SNN_ROWS_WIDE / SNN_ROWS_QUAD run as SNN_ROWS_PAIRS (the same sums).
template <typename real, int NPT, int TH, bool WIDE = false>
__device__ __forceinline__ void forward_trial(const FwdParams<real>& p, const int b, unsigned char* smem) {
    const int N = p.N, K = p.K, Win = p.Win, Wh = p.Wh, n_in = p.n_in;
    const int R = n_in + N;
    const int NA = N + 64;                        // accumulators: neurons, 32 per-lane spares, readouts
    constexpr bool NARROW = sizeof(real) == 4;    // FP32: narrow slots, one word per accumulator
    unsigned* acc = (unsigned*)smem;              // narrow [NA]; wide [2][NA]: H words, then L words
    int* lens = (int*)(acc + (NARROW ? NA : 2 * NA));   // [R + 1] packed row lengths (row R: empty)
    int* list = lens + R + 1;                     // [2][R] spiking rows by step parity
    int* lcnt = list + 2 * R;                     // [2]
    uint32_t* xw = (uint32_t*)(lcnt + 2);         // [Win] input spike words of the current step
    uint32_t* zb = xw + Win;                      // [2][Wh]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int nwarps = TH / 32;
    constexpr int RO_WARP = 1;                    // advances the readout in phase B
    const int t0 = p.t0;
    const int t_end = p.trial_T ? min(p.t0 + p.n_steps, max(p.trial_T[b], p.t0)) : p.t0 + p.n_steps;
    real vr[NPT], ar[NPT], sc[NPT];               // sc: narrow grid step of each neuron's accumulator
    {
        const int prv = (t0 - 1) & 1;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int j = tid + q * TH;
            vr[q] = j < N ? p.v[(size_t)b * N + j] : real(0);
            ar[q] = j < N ? p.a[(size_t)b * N + j] : real(0);
            sc[q] = (NARROW && j < N) ? (real)narrow_scale(p.colsum[j]) : real(0);
        }
        for (int j = tid; j < (NARROW ? NA : 2 * NA); j += TH) acc[j] = 0u;
        for (int j = tid; j < N; j += TH) lens[n_in + j] = p.rec_len[j] + K;
        for (int i = tid; i < n_in; i += TH) lens[i] = p.in_len[i];
        if (tid == 0) lens[R] = 0;
        for (int w = tid; w < Wh; w += TH) zb[prv * Wh + w] = p.z_bits[(size_t)b * Wh + w];
        if (warp == 0) {
            // lists of step t0-1 from the state's spike words
            if (lane == 0) lcnt[prv] = 0;
            __syncwarp();
            for (int w = lane; w < Win + Wh; w += 32) {
                uint32_t word = w < Win ? p.x_bits[(size_t)b * Win + w] : p.z_bits[(size_t)b * Wh + (w - Win)];
                const int base = w < Win ? w * 32 : n_in + (w - Win) * 32;
                const int pos = atomicAdd(&lcnt[prv], __popc(word));
                for (int k = 0; word; ++k, word &= word - 1u) list[prv * R + pos + k] = base + __ffs(word) - 1;
            }
        }
    }
    real yk = 0, ysk = 0, bk = 0, sck = 0;
    if (warp == RO_WARP && lane < K) {
        yk = p.y[(size_t)b * K + lane];
        ysk = p.ysum[(size_t)b * K + lane];
        bk = p.b_out[lane];
        if (NARROW) sck = (real)narrow_scale(p.colsum[N + 32 + lane]);
    }
    if (b == 0) {
        // a neuron or readout whose |weight| sum reaches 2^11 could wrap its fixed-point sum
        bool over = false;
        for (int j = tid; j < N + 64; j += TH) over |= p.colsum[j] >= FIX_SUM_LIMIT;
        if (__syncthreads_or(over) && tid == 0) atomicOr(p.status, ST_STATE);
    }
    const uint32_t* xrec_b = p.x_rec + (size_t)b * p.T * Win;
    uint32_t* zrec_b = p.z_rec + (size_t)b * p.T * Wh;
    real* psi_b = p.psi_rec ? p.psi_rec + (size_t)b * p.T * N : nullptr;   // NULL: inference, no records
    real* d_b = p.d_rec ? p.d_rec + (size_t)b * p.T * K : nullptr;
    uint32_t xnext = (warp == 0 && lane < Win && t0 < t_end) ? xrec_b[(size_t)t0 * Win + lane] : 0u;
    __syncthreads();

    for (int t = t0; t < t_end; ++t) {
        const int cur = t & 1, prv = cur ^ 1;
        const uint32_t* zprv = zb + prv * Wh;
        uint32_t* zcur = zb + cur * Wh;
        const int* lprv = list + prv * R;
        int* lcur = list + cur * R;
        // ---------------- phase A
        const int n_rows = lcnt[prv];
        if (tid >= 64 && tid - 64 < Wh) {
            const int w = tid - 64;
            if (t > t0) zrec_b[(size_t)(t - 1) * Wh + w] = zprv[w];
            zcur[w] = 0u;
        }
        if (tid == 32) lcnt[cur] = 0;
        switch (p.sched) {
            case SNN_ROWS_PER_BLOCK:
                propagate_rows_block<NARROW, nwarps>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, warp, lane);
                break;
            case SNN_ROWS_PER_WARP:
                propagate_rows_warp<NARROW, 1, nwarps>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R, warp, lane);
                break;
            case SNN_ROWS_WIDE:
                if (WIDE) propagate_rows_warp<NARROW, 2, nwarps, 8>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R, warp, lane);
                else propagate_rows_warp<NARROW, FWD_ROWS, nwarps, FWD_CHUNKS>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R, warp, lane);
                break;
            case SNN_ROWS_QUAD:
                if (WIDE) propagate_rows_warp<NARROW, 4, nwarps>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R, warp, lane);
                else propagate_rows_warp<NARROW, FWD_ROWS, nwarps, FWD_CHUNKS>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R, warp, lane);
                break;
            default:
                propagate_rows_warp<NARROW, FWD_ROWS, nwarps, FWD_CHUNKS>(acc, NA, lprv, n_rows, lens, p.pk, p.Cf, R,
                                                                         warp, lane);
                break;
        }
        __syncthreads();
        // ---------------- phase B: neurons; spike lists of step t
        if (warp == 0) {
            // x^t: one list reservation for the warp, positions by a prefix sum of the counts
            uint32_t word = lane < Win ? xnext : 0u;
            if (lane < Win && t + 1 < t_end) xnext = xrec_b[(size_t)(t + 1) * Win + lane];
            const int cnt = __popc(word);
            const int incl = warp_incl_scan(cnt);
            int base = 0;
            if (lane == 31 && incl) base = atomicAdd(&lcnt[cur], incl);
            base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
            for (int k = 0; word; ++k, word &= word - 1u) lcur[base + k] = lane * 32 + __ffs(word) - 1;
        }
        if (warp == RO_WARP && lane < K) {         // y^t from the readout sums W_out z^{t-1}
            yk = p.alpha * yk + acc_real<NARROW, real>(acc + N + 32 + lane, NA, sck) + bk;
            acc_zero<NARROW>(acc + N + 32 + lane, NA);
            ysk += yk;
            if (d_b) d_b[(size_t)t * K + lane] = yk;
            if (p.y_rec) p.y_rec[((size_t)b * p.T + t) * K + lane] = yk;
        }
        real* psi_t = psi_b ? psi_b + (size_t)t * N : nullptr;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int j = tid + q * TH;
            bool spk = false;
            if (j < N) {
                const real I = acc_real<NARROW, real>(acc + j, NA, sc[q]);
                acc_zero<NARROW>(acc + j, NA);
                const bool zp = (zprv[j >> 5] >> (j & 31)) & 1u;
                const real v = p.alpha * (zp ? vr[q] - p.v_thr : vr[q]) + I;
                const real aa = p.rho * ar[q] + (zp ? real(1) : real(0));
                const real A = p.v_thr + p.beta * aa;
                const real u = real(1) - fabs((v - A) * p.inv_vthr);
                if (psi_t) psi_t[j] = p.psi_scale * (u > real(0) ? u : real(0));
                vr[q] = v;
                ar[q] = aa;
                if (p.record_state) {
                    p.v_rec[(size_t)b * p.T * N + (size_t)t * N + j] = v;
                    p.a_rec[(size_t)b * p.T * N + (size_t)t * N + j] = aa;
                }
                spk = v >= A;
            }
            // whole warp: j >> 5 is the same word for all its lanes (TH is a multiple of 32)
            const unsigned zm = __ballot_sync(0xffffffffu, spk);
            if (zm) {
                int pos = 0;
                if (lane == 0) {
                    zcur[j >> 5] = zm;
                    pos = atomicAdd(&lcnt[cur], __popc(zm));
                }
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if (spk) lcur[pos + __popc(zm & lanemask_lt())] = n_in + j;
            }
        }
        __syncthreads();
    }
    if (t_end > t0) {
        const int last = t_end - 1;
        const int cl = last & 1;
        for (int w = tid; w < Wh; w += TH) {
            zrec_b[(size_t)last * Wh + w] = zb[cl * Wh + w];
            p.z_bits[(size_t)b * Wh + w] = zb[cl * Wh + w];
        }
        for (int w = tid; w < Win; w += TH) p.x_bits[(size_t)b * Win + w] = xrec_b[(size_t)last * Win + w];
    }
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const int j = tid + q * TH;
        if (j < N) {
            p.v[(size_t)b * N + j] = vr[q];
            p.a[(size_t)b * N + j] = ar[q];
        }
    }
    if (warp == RO_WARP && lane < K) {
        p.y[(size_t)b * K + lane] = yk;
        p.ysum[(size_t)b * K + lane] = ysk;
    }
}

template <typename real, int NPT, int TH>
__global__ void __launch_bounds__(TH, 1024 / TH) k_forward(FwdParams<real> p) {
    extern __shared__ __align__(16) unsigned char smem[];
    forward_trial<real, NPT, TH>(p, blockIdx.x, smem);
}

// d^t = softmax(y^t) - onehot(label) for every recorded (trial, step), in place over the
// y values the forward left in the d record.  A warp takes 32 consecutive steps of one
// trial: their rows are one contiguous span of 32 K values, read and written whole by
// the warp (coalesced); lane r computes row r from shared memory.
constexpr int SMX_WARPS = 4;

// One warp: the span of nr steps from ts of trial b, staged in sh (32 K values).
template <typename real>
__device__ __forceinline__ void softmax_span(real* __restrict__ d, const int32_t* __restrict__ labels, int n_classes,
                                             const int32_t* __restrict__ trial_T, int b, int T, int K, int ts, int nr,
                                             real* sh) {
    const int lane = lane_id();
    real* span = d + ((size_t)b * T + ts) * K;
    for (int e = lane; e < nr * K; e += 32) sh[e] = span[e];
    __syncwarp();
    const int t = ts + lane;
    if (lane < nr && !(trial_T && t >= trial_T[b])) {
        const int label = min(max(labels[b], 0), n_classes - 1);
        real* y = sh + lane * K;
        real mx = y[0];
        for (int k = 1; k < K; ++k) mx = y[k] > mx ? y[k] : mx;
        real ssum = 0;
        for (int k = 0; k < K; ++k) ssum += exp_real(y[k] - mx);
        for (int k = 0; k < K; ++k) y[k] = exp_real(y[k] - mx) / ssum - (k == label ? real(1) : real(0));
    }
    __syncwarp();
    for (int e = lane; e < nr * K; e += 32) span[e] = sh[e];
}

template <typename real>
__global__ void __launch_bounds__(SMX_WARPS * 32)
    k_softmax_d(real* __restrict__ d, const int32_t* __restrict__ labels, int n_classes,
                const int32_t* __restrict__ trial_T, int B, int T, int K, int t0, int n_steps) {
    extern __shared__ __align__(16) unsigned char smx_raw[];
    real* sh = (real*)smx_raw + (size_t)(threadIdx.x >> 5) * 32 * K;
    const int blocks_per_trial = (n_steps + 31) / 32;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wg >= (long long)B * blocks_per_trial) return;
    const int b = (int)(wg / blocks_per_trial);
    const int ts = t0 + (int)(wg % blocks_per_trial) * 32;          // first step of the span
    const int nr = min(32, t0 + n_steps - ts);                      // rows in the span
    softmax_span<real>(d, labels, n_classes, trial_T, b, T, K, ts, nr, sh);
}

// Packed forward rows: row r < n_in is input row r, row n_in + j is hidden row j; Cf
// slots each, one 64-bit load per slot.  Hidden row j holds its len_j synapses, then its
// readout column W_out[k][j] aimed at accumulators N + 32 + k.  Slots past a row's
// length hold weight 0 aimed at the per-lane spare N + (slot mod 32), so a warp adds a
// row's last 32-slot chunk whole, with no per-lane test and no two lanes on one address.
// Wide slots (FP64): bits 63..52 target accumulator, bits 51..0 the weight in fixed point
// (40 fractional bits, two's complement).  Narrow slots (FP32): bits 63..32 the target
// accumulator's byte offset, bits 31..0 the weight on the target's grid (see acc_add);
// they need every accumulator's |weight| sum first (colsum_slot over all slots), then
// pack_slot_narrow.

// Target accumulator and fixed-point weight of packed slot i (weight 0: padding).
template <typename real>
__device__ __forceinline__ void pack_src(const real* __restrict__ w_in, const int32_t* __restrict__ ind_in,
                                         const int32_t* __restrict__ len_in, int C_in, int n_in,
                                         const real* __restrict__ w_rec, const int32_t* __restrict__ ind_rec,
                                         const int32_t* __restrict__ len_rec, int C_rec, const real* __restrict__ W_out,
                                         int K, int N, int Cf, const long long i, unsigned& tgt, long long& f) {
    const int r = (int)(i / Cf), s = (int)(i % Cf);
    tgt = (unsigned)(N + (s & 31));
    f = 0;
    if (r < n_in) {
        if (s < len_in[r]) {
            const size_t e = (size_t)r * C_in + s;
            tgt = (unsigned)ind_in[e];
            f = to_fixed(w_in[e]);
        }
    } else {
        const int j = r - n_in, L = len_rec[j];
        if (s < L) {
            const size_t e = (size_t)j * C_rec + s;
            tgt = (unsigned)ind_rec[e];
            f = to_fixed(w_rec[e]);
        } else if (s < L + K) {
            tgt = (unsigned)(N + 32 + (s - L));
            f = to_fixed(W_out[(size_t)(s - L) * N + j]);
        }
    }
}

#define SNN_PACK_ARGS                                                                                          \
    const real *__restrict__ w_in, const int32_t *__restrict__ ind_in, const int32_t *__restrict__ len_in,    \
        int C_in, int n_in, const real *__restrict__ w_rec, const int32_t *__restrict__ ind_rec,              \
        const int32_t *__restrict__ len_rec, int C_rec, const real *__restrict__ W_out, int K, int N, int Cf
#define SNN_PACK_PASS w_in, ind_in, len_in, C_in, n_in, w_rec, ind_rec, len_rec, C_rec, W_out, K, N, Cf

// Wide slot i, and its |weight| into its accumulator's sum.
template <typename real>
__device__ __forceinline__ void pack_slot(SNN_PACK_ARGS, unsigned long long* __restrict__ pk,
                                          unsigned long long* __restrict__ colsum, const long long i) {
    unsigned tgt;
    long long f;
    pack_src<real>(SNN_PACK_PASS, i, tgt, f);
    pk[i] = ((unsigned long long)tgt << 52) | ((unsigned long long)f & ((1ull << 52) - 1));
    if (f) atomicAdd(&colsum[tgt], (unsigned long long)(f < 0 ? -f : f));
}
// The |weight| of slot i into its accumulator's sum (first pass of the narrow packing).
template <typename real>
__device__ __forceinline__ void colsum_slot(SNN_PACK_ARGS, unsigned long long* __restrict__ colsum,
                                            const long long i) {
    unsigned tgt;
    long long f;
    pack_src<real>(SNN_PACK_PASS, i, tgt, f);
    if (f) atomicAdd(&colsum[tgt], (unsigned long long)(f < 0 ? -f : f));
}
// Narrow slot i from the complete sums: the weight rounded (half up) to the target's grid.
template <typename real>
__device__ __forceinline__ void pack_slot_narrow(SNN_PACK_ARGS, unsigned long long* __restrict__ pk,
                                                 const unsigned long long* __restrict__ colsum, const long long i) {
    unsigned tgt;
    long long f;
    pack_src<real>(SNN_PACK_PASS, i, tgt, f);
    const int sh = narrow_shift(colsum[tgt]);
    const long long v = sh ? (f + (1ll << (sh - 1))) >> sh : f;
    pk[i] = ((unsigned long long)(tgt * 4u) << 32) | (unsigned)(int)v;
}

template <typename real>
__global__ void k_pack(SNN_PACK_ARGS, unsigned long long* __restrict__ pk, long long n,
                       unsigned long long* __restrict__ colsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pack_slot<real>(SNN_PACK_PASS, pk, colsum, i);
}
template <typename real>
__global__ void k_colsum(SNN_PACK_ARGS, long long n, unsigned long long* __restrict__ colsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    colsum_slot<real>(SNN_PACK_PASS, colsum, i);
}
template <typename real>
__global__ void k_pack_narrow(SNN_PACK_ARGS, unsigned long long* __restrict__ pk, long long n,
                              const unsigned long long* __restrict__ colsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pack_slot_narrow<real>(SNN_PACK_PASS, pk, colsum, i);
}

// Filtered readout error D_k^t = d_k^{t+1} + alpha D_k^{t+1} (D^{T-1} = 0), i.e.
// D_k^t = sum_{u > t} alpha^{u-t-1} d_k^u, and the bias gradient partial sum_t d_k^t.
// One warp per trial, lane k per readout (padding lanes k >= K write zeros): the warp
// walks the steps backwards reading and writing one contiguous row per step, with the
// rows of the next RS_AHEAD steps loaded ahead of the recurrence.
constexpr int RS_AHEAD = 8;

template <typename real>
__device__ __forceinline__ void readout_scan_warp(const real* __restrict__ d, real* __restrict__ Dout,
                                                  real* __restrict__ gb_part, const int b, int T, int K, int Kp,
                                                  real alpha) {
    const int k = lane_id();
    if (k >= Kp) return;
    const real* db = d + (size_t)b * T * K;
    real* Db = Dout + (size_t)b * T * Kp;
    const bool live = k < K;
    real E = 0, gsum = 0;
    real dn = 0;                                     // d^{t+1}
    // steps in blocks of RS_AHEAD, from the end: the block's d rows are loaded first
    for (int t1 = T; t1 > 0; t1 -= RS_AHEAD) {
        const int t0 = t1 - RS_AHEAD > 0 ? t1 - RS_AHEAD : 0;
        real dv[RS_AHEAD];
#pragma unroll
        for (int r = 0; r < RS_AHEAD; ++r) {
            const int t = t1 - 1 - r;
            dv[r] = (live && t >= t0) ? db[(size_t)t * K + k] : real(0);
        }
#pragma unroll
        for (int r = 0; r < RS_AHEAD; ++r) {
            const int t = t1 - 1 - r;
            if (t >= t0) {
                E = (t == T - 1) ? real(0) : dn + alpha * E;
                Db[(size_t)t * Kp + k] = E;
                gsum += dv[r];
                dn = dv[r];
            }
        }
    }
    if (live) gb_part[(size_t)b * K + k] = gsum;
}

template <typename real>
__global__ void k_readout_scan(const real* __restrict__ d, real* __restrict__ Dout, real* __restrict__ gb_part,
                               int B, int T, int K, int Kp, real alpha) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    readout_scan_warp<real>(d, Dout, gb_part, b, T, K, Kp, alpha);
}

// Gather order of a ragged row: its live slots as keys (target << 11) | slot, sorted
// ascending (targets are distinct within a row).  With sorted targets the 32 lanes of
// one gather chunk read a narrow band of the adjoint row, so the chunks of one spike
// event touch few 32-byte sectors more than once.  Warp per row, rank by counting;
// blockDim.x / 32 warps per CTA, each with a C-word shared-memory row.
__device__ __forceinline__ void sort_row_warp(const int32_t* __restrict__ len, const int32_t* __restrict__ ind,
                                              const int i, int C, int32_t* __restrict__ keys, int32_t* row) {
    const int lane = lane_id();
    const int n = len[i];
    for (int s = lane; s < n; s += 32) row[s] = (ind[(size_t)i * C + s] << 11) | s;
    __syncwarp();
    for (int s = lane; s < n; s += 32) {
        const int32_t key = row[s];
        int rank = 0;
        for (int e = 0; e < n; ++e) rank += row[e] < key ? 1 : 0;
        keys[(size_t)i * C + rank] = key;
    }
}

// Gather: grid (spike-word columns x 32 / ROWS, KS, slot groups).  CTA = ROWS presynaptic
// rows of one bit word (input words first, then hidden words) for one group of 128 slots;
// one warp per row, 4 slot chunks per lane.  The CTA stages the spike words of its whole
// (trial, step) range in shared memory; each warp walks its bit through them with
// ballots, collects EV spike times (across as many 32-step windows as it takes) and then
// issues their delta loads together, so a sparse row still keeps 4 EV loads in flight
// per lane.  The group-0 warps of hidden rows also sum D into the
// readout gradient.  CTAs whose rows all end before their group exit before staging.
constexpr int GATHER_SPAN = 4096;   // (trial, step) entries per K-split: ~16 MB of adjoint rows per
                                    // split stays in L2 while the splits in flight read it (8192: 5 % slower)
constexpr int GATHER_ROWS = 16;   // rows (warps) per CTA: 32, 16 or 8
constexpr int GATHER_EV = 4;      // spike events whose loads are issued together

template <typename real, int ROWS, int EV, bool DIRECT>
__device__ __forceinline__ void gather_block(const uint32_t* __restrict__ x_rec, const uint32_t* __restrict__ z_rec, int Win, int Wh,
             const int32_t* __restrict__ in_len, const int32_t* __restrict__ in_keys, int in_C, int n_in,
             const int32_t* __restrict__ rec_len, const int32_t* __restrict__ rec_keys, int rec_C, int N,
             const real* __restrict__ delta, const real* __restrict__ D, int K, int Kp, long long BT,
             long long bt_per, real* __restrict__ part_in, real* __restrict__ part_rec,
             real* __restrict__ part_out, const int bx, const int ks, const int g, uint32_t* words) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    constexpr int SPLIT = 32 / ROWS;
    const int col = bx / SPLIT;
    const int r0 = (bx % SPLIT) * ROWS;            // first row of the word this CTA owns
    // g: slot group, slots [128 g, 128 g + 128)
    const bool is_in = col < Win;
    const int wi = is_in ? col : col - Win;
    const int i = wi * 32 + r0 + warp;
    const int P = is_in ? n_in : N;
    const bool row_ok = i < P;
    const int len = row_ok ? (is_in ? in_len[i] : rec_len[i]) : 0;
    const int s_base = 128 * g;
    const bool readout = !is_in && g == 0;
    const bool active = row_ok && (len > s_base || readout);
    if (!__syncthreads_or(active)) return;
    const uint32_t* bits = is_in ? x_rec : z_rec;
    const int W = is_in ? Win : Wh;
    const int C = is_in ? in_C : rec_C;
    const long long bt0 = (long long)ks * bt_per;
    const long long bt1 = min(BT, bt0 + bt_per);
    // the walk below reads words [0, roundup32(bt1 - bt0)) only
    const int n_stage = bt1 > bt0 ? (int)min((long long)GATHER_SPAN, (bt1 - bt0 + 31) / 32 * 32) : 0;
    for (int k = threadIdx.x; k < n_stage; k += ROWS * 32) {
        const long long my = bt0 + k;
        words[k] = (my < bt1) ? bits[my * W + wi] : 0u;
    }
    const int32_t* rk = (is_in ? in_keys : rec_keys) + (size_t)(row_ok ? i : 0) * C;
    const int nq = len > s_base ? min(4, (len - s_base + 31) >> 5) : 0;   // warp-uniform
    int key[4];                                     // (target << 11) | slot, or -1
    real acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int s = s_base + q * 32 + lane;
        key[q] = (q < nq && s < len) ? rk[s] : -1;
        acc[q] = 0;
    }
    real acc_o = 0;
    const bool do_out = readout && row_ok && lane < K;
    const uint32_t bit = 1u << (r0 + warp);
    __syncthreads();
    if (!active) return;
    const int span = bt1 > bt0 ? (int)(bt1 - bt0) : 0;
    const real* delta0 = delta + bt0 * N;
    const real* D0 = D + bt0 * Kp;
    int sub = 0, wbase = 0;
    uint32_t spk = 0u;                               // warp-uniform (a ballot)
    for (;;) {
        int off[EV];
        int nv = 0;
#pragma unroll
        for (int k = 0; k < EV; ++k) {
            while (spk == 0u && sub < span) {
                spk = __ballot_sync(0xffffffffu, (words[sub + lane] & bit) != 0u);
                wbase = sub;
                sub += 32;
            }
            off[k] = wbase + (spk ? __ffs(spk) - 1 : 0);
            if (spk) {
                spk &= spk - 1u;
                ++nv;
            }
        }
        if (nv == 0) break;
        real v[EV][4];
#pragma unroll
        for (int k = 0; k < EV; ++k) {
            const real* rowp = delta0 + (size_t)off[k] * N;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[k][q] = (k < nv && q < nq && key[q] >= 0) ? rowp[key[q] >> 11] : real(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            real s = 0;
#pragma unroll
            for (int k = 0; k < EV; k += 4) s += (v[k][q] + v[k + 1][q]) + (v[k + 2][q] + v[k + 3][q]);
            acc[q] += s;
        }
        if (do_out) {
            real o = 0;
#pragma unroll
            for (int k = 0; k < EV; ++k)
                if (k < nv) o += D0[(size_t)off[k] * Kp + lane];
            acc_o += o;
        }
    }
    real* part = is_in ? part_in : part_rec;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int s = s_base + q * 32 + lane;
        if (q < nq && s < len) part[((size_t)ks * P + i) * C + (key[q] & 2047)] = acc[q];
    }
    if (do_out) {
        if (DIRECT) part_out[(size_t)lane * N + i] = acc_o;      // one K-split: G_out[k][j] directly
        else part_out[((size_t)ks * N + i) * K + lane] = acc_o;
    }
}

template <typename real, int ROWS, int EV>
__global__ void __launch_bounds__(ROWS * 32, 1)
    k_gather(const uint32_t* __restrict__ x_rec, const uint32_t* __restrict__ z_rec, int Win, int Wh,
             const int32_t* __restrict__ in_len, const int32_t* __restrict__ in_keys, int in_C, int n_in,
             const int32_t* __restrict__ rec_len, const int32_t* __restrict__ rec_keys, int rec_C, int N,
             const real* __restrict__ delta, const real* __restrict__ D, int K, int Kp, long long BT,
             long long bt_per, real* __restrict__ part_in, real* __restrict__ part_rec,
             real* __restrict__ part_out) {
    __shared__ uint32_t words[GATHER_SPAN];
    gather_block<real, ROWS, EV, false>(x_rec, z_rec, Win, Wh, in_len, in_keys, in_C, n_in, rec_len, rec_keys, rec_C,
                                        N, delta, D, K, Kp, BT, bt_per, part_in, part_rec, part_out, blockIdx.x,
                                        blockIdx.y, blockIdx.z, words);
}

// ------------------------------------------------------------------ Adam (+ L1)
// omb1 = 1 - beta1 and omb2 = 1 - beta2 come from the host in double precision: forming
// 1 - 0.999f in float would put a 1.3e-5 relative error on the second-moment update.
template <typename real>
__device__ __forceinline__ void adam_update(real& w, real& m, real& v, real g, real lr, real b1, real b2, real omb1,
                                            real omb2, real eps, real bc1, real bc2) {
    m = b1 * m + omb1 * g;
    v = b2 * v + omb2 * g * g;
    real mh = m / bc1;
    real vh = v / bc2;
    w = w - lr * mh / (sqrt(vh) + eps);
}

// bias_dev (optional): device {beta1^t, beta2^t}; replaces bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
template <typename real>
__device__ __forceinline__ void bias_from_device(const double* bias_dev, real& bc1, real& bc2) {
    if (bias_dev) {
        bc1 = (real)(1.0 - bias_dev[0]);
        bc2 = (real)(1.0 - bias_dev[1]);
    }
}

// DEEP R noise of slot (i, s): standard normal by the Box-Muller transform of two
// Philox words, in double precision.
__device__ __forceinline__ double deepr_noise(uint64_t seed, uint64_t noise_idx, int i, int s) {
    const u64x4 u = philox(seed, PH_DEEPR_NOISE, noise_idx, (uint64_t)i, (uint64_t)s, 0);
    const double u1 = (double)((u.x >> 11) + 1) * 0x1p-53;      // (0, 1], exact: the log stays finite
    const double u2 = (double)(u.y >> 11) * 0x1p-53;            // [0, 1)
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

struct NoiseK {
    double amp;                    // sqrt(2 lr temperature); 0 = off
    uint64_t seed, idx;
    const int64_t* idx_dev;
};

template <typename real>
__device__ __forceinline__ void adam_ragged_elem(const int32_t* __restrict__ len, const int32_t* __restrict__ ind,
                                                 int C, int Qw, real* __restrict__ w, real* __restrict__ m,
                                                 real* __restrict__ v, const real* __restrict__ grad,
                                                 const uint32_t* __restrict__ sign, real l1, real lr, real b1, real b2,
                                                 real omb1, real omb2, real eps, real bc1, real bc2,
                                                 const double* __restrict__ bias_dev, const NoiseK& nz,
                                                 const long long idx) {
    bias_from_device(bias_dev, bc1, bc2);
    int i = (int)(idx / C), s = (int)(idx % C);
    if (s >= len[i]) return;
    real g = grad[idx];
    if (sign) {
        int j = ind[idx];
        bool pos = (sign[(size_t)i * Qw + (j >> 5)] >> (j & 31)) & 1u;
        g += pos ? l1 : -l1;
    }
    real ww = w[idx], mm = m[idx], vv = v[idx];
    adam_update(ww, mm, vv, g, lr, b1, b2, omb1, omb2, eps, bc1, bc2);
    if (nz.amp > 0.0) {
        const uint64_t k = nz.idx_dev ? (uint64_t)*nz.idx_dev : nz.idx;
        ww = (real)((double)ww + nz.amp * deepr_noise(nz.seed, k, i, s));
    }
    w[idx] = ww;
    m[idx] = mm;
    v[idx] = vv;
}

template <typename real>
__device__ __forceinline__ void adam_dense_elem(real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                                                const real* __restrict__ grad, real lr, real b1, real b2, real omb1,
                                                real omb2, real eps, real bc1, real bc2,
                                                const double* __restrict__ bias_dev, const int idx) {
    bias_from_device(bias_dev, bc1, bc2);
    real ww = w[idx], mm = m[idx], vv = v[idx];
    adam_update(ww, mm, vv, grad[idx], lr, b1, b2, omb1, omb2, eps, bc1, bc2);
    w[idx] = ww;
    m[idx] = mm;
    v[idx] = vv;
}

template <typename real>
__global__ void k_adam_ragged(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, int P, int C, int Qw,
                              real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                              const real* __restrict__ grad, const uint32_t* __restrict__ sign, real l1, real lr,
                              real b1, real b2, real omb1, real omb2, real eps, real bc1, real bc2,
                              const double* __restrict__ bias_dev, NoiseK nz) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * C) return;
    adam_ragged_elem<real>(len, ind, C, Qw, w, m, v, grad, sign, l1, lr, b1, b2, omb1, omb2, eps, bc1, bc2, bias_dev,
                           nz, idx);
}

template <typename real>
__global__ void k_adam_dense(real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                             const real* __restrict__ grad, int n, real lr, real b1, real b2, real omb1,
                             real omb2, real eps, real bc1, real bc2, const double* __restrict__ bias_dev) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    adam_dense_elem<real>(w, m, v, grad, lr, b1, b2, omb1, omb2, eps, bc1, bc2, bias_dev, idx);
}

// Packed FP32 pairs (Blackwell f32x2 arithmetic; each half is rounded exactly like the
// scalar operation).  Low half = first value.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float f2_lo(unsigned long long a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float f2_hi(unsigned long long a) { return __uint_as_float((unsigned)(a >> 32)); }
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// FP32 adjoint scan with two neurons per thread (N even): the same recurrences as
// k_backward on neuron pairs (2 jp, 2 jp + 1) in packed f32x2 arithmetic, psi and delta
// moved as 8-byte pairs.  lam of each neuron is summed over readout pairs (k, k + 1)
// with one packed FMA per pair: lam = (sum over even k) + (sum over odd k).
constexpr int BWD2_TCH = 4;    // steps per chunk of the packed kernel

// One CTA (TH threads) of the scan: neuron pairs blk * TH .. blk * TH + TH - 1 of trial b;
// D_smem: 2 * BWD2_TCH * 4 KV floats of shared memory, 16-byte aligned.
template <int KV, int TH>
__device__ __forceinline__ void backward_x2_block(const float* __restrict__ psi, const float* __restrict__ Dg,
                                                  const float* __restrict__ W_out, float* __restrict__ delta, int T,
                                                  int N, int K, float alpha, float rho, float beta, const int blk,
                                                  const int b, float* D_smem) {
    constexpr int KP = 4 * KV;
    float (*D_s)[BWD2_TCH][KP] = reinterpret_cast<float (*)[BWD2_TCH][KP]>(D_smem);
    const int tid = threadIdx.x;
    const int jp = blk * TH + tid;                    // neuron pair
    const int N2 = N >> 1;
    const bool ok = jp < N2;
    unsigned long long wa[KP / 2], wb[KP / 2];         // (W[2m][j], W[2m+1][j]) for j = 2 jp, 2 jp + 1
#pragma unroll
    for (int m = 0; m < KP / 2; ++m) {
        const int k0 = 2 * m, k1 = 2 * m + 1;
        const float a0 = (k0 < K && ok) ? W_out[(size_t)k0 * N + 2 * jp] : 0.f;
        const float a1 = (k1 < K && ok) ? W_out[(size_t)k1 * N + 2 * jp] : 0.f;
        const float b0 = (k0 < K && ok) ? W_out[(size_t)k0 * N + 2 * jp + 1] : 0.f;
        const float b1 = (k1 < K && ok) ? W_out[(size_t)k1 * N + 2 * jp + 1] : 0.f;
        wa[m] = f2_pack(a0, a1);
        wb[m] = f2_pack(b0, b1);
    }
    const unsigned long long* pb = (const unsigned long long*)psi + (size_t)b * T * N2 + (ok ? jp : 0);
    const float* Db = Dg + (size_t)b * T * KP;
    unsigned long long* db = (unsigned long long*)delta + (size_t)b * T * N2 + (ok ? jp : 0);
    const int n_chunks = (T + BWD2_TCH - 1) / BWD2_TCH;
    unsigned long long pcur[BWD2_TCH], pnext[BWD2_TCH];
    auto load_chunk = [&](int ch, unsigned long long (&dst)[BWD2_TCH], int buf) {
        const int tb = ch * BWD2_TCH, nt = min(BWD2_TCH, T - tb);
#pragma unroll
        for (int r = 0; r < BWD2_TCH; ++r) dst[r] = (r < nt && ok) ? pb[(size_t)(tb + r) * N2] : 0ull;
        for (int idx = tid; idx < nt * KP; idx += TH) D_s[buf][idx / KP][idx % KP] = Db[(size_t)tb * KP + idx];
    };
    const unsigned long long alpha2 = f2_pack(alpha, alpha), beta2 = f2_pack(beta, beta);
    const unsigned long long rho2 = f2_pack(rho, rho), nbeta2 = f2_pack(-beta, -beta);
    load_chunk(n_chunks - 1, pcur, (n_chunks - 1) & 1);
    __syncthreads();
    unsigned long long lam_next = 0, psi_next = 0, mu = 0, h_next = 0, dl = 0;
    for (int ch = n_chunks - 1; ch >= 0; --ch) {
        const int tb = ch * BWD2_TCH, nt = min(BWD2_TCH, T - tb);
        const int buf = ch & 1;
        if (ch > 0) load_chunk(ch - 1, pnext, buf ^ 1);
#pragma unroll
        for (int r = BWD2_TCH - 1; r >= 0; --r) {
            if (r < nt) {
                const int t = tb + r;
                const unsigned long long ps = pcur[r];
                const unsigned long long* Dr = (const unsigned long long*)D_s[buf][r];
                unsigned long long sa = 0, sb = 0;
#pragma unroll
                for (int m = 0; m < KP / 2; ++m) {
                    const unsigned long long dk = Dr[m];           // (D_2m, D_2m+1)
                    sa = f2_fma(wa[m], dk, sa);
                    sb = f2_fma(wb[m], dk, sb);
                }
                const unsigned long long lam = f2_pack(f2_lo(sa) + f2_hi(sa), f2_lo(sb) + f2_hi(sb));
                if (t == T - 1) {
                    mu = 0;
                    dl = 0;
                } else {
                    // mu = beta lam' psi' + (rho - beta psi') mu ;  delta = h' + alpha delta'
                    mu = f2_fma(beta2, f2_mul(lam_next, psi_next), f2_mul(f2_fma(nbeta2, psi_next, rho2), mu));
                    dl = f2_fma(alpha2, dl, h_next);
                }
                const unsigned long long h = f2_mul(ps, f2_sub(lam, mu));
                if (ok) db[(size_t)t * N2] = dl;
                h_next = h;
                lam_next = lam;
                psi_next = ps;
            }
        }
#pragma unroll
        for (int r = 0; r < BWD2_TCH; ++r) pcur[r] = pnext[r];
        __syncthreads();
    }
}

template <int KV>
__global__ void __launch_bounds__(BWD_THREADS)
    k_backward_x2(const float* __restrict__ psi, const float* __restrict__ Dg, const float* __restrict__ W_out,
                  float* __restrict__ delta, int T, int N, int K, float alpha, float rho, float beta) {
    __shared__ __align__(16) float D_s[2 * BWD2_TCH * 4 * KV];
    backward_x2_block<KV, BWD_THREADS>(psi, Dg, W_out, delta, T, N, K, alpha, rho, beta, blockIdx.x, blockIdx.y, D_s);
}

// beta1^t, beta2^t for the step count t, kept in device state: one multiplication per
// call when t advances by one (graph replay), a fresh running product otherwise.  At most
// 2^24 multiplications per call: a larger jump sets the invalid-state flag and keeps the
// partial product (a later call continues it).  One thread.
__device__ __forceinline__ void adam_bias_step(long long t, double beta1, double beta2, AdamBias* st,
                                               int32_t* status) {
    if (t < 1) {
        atomicOr(status, ST_STATE);
        t = 1;
    }
    if (st->t == t && st->beta1 == beta1 && st->beta2 == beta2) return;
    double b1 = 1.0, b2 = 1.0;
    long long t0 = 0;
    if (st->beta1 == beta1 && st->beta2 == beta2 && st->t >= 0 && st->t < t) {
        b1 = st->b1t;
        b2 = st->b2t;
        t0 = st->t;
    }
    const long long lim = 1ll << 24;
    adam_bias_advance(beta1, beta2, t0, b1, b2, t, lim);
    long long reached = t;
    if (t - t0 > lim && (b1 != 0.0 || b2 != 0.0)) {
        atomicOr(status, ST_STATE);
        reached = t0 + lim;
    }
    st->b1t = b1;
    st->b2t = b2;
    st->beta1 = beta1;
    st->beta2 = beta2;
    st->t = reached;
}

}  // namespace snn
