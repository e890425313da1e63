// Recurrent LIF/ALIF classifier with e-prop and Adam (Sec. 2.2.1 of the paper).
//
// Forward: one CTA owns one trial and runs every requested step inside one launch.
// Per step it propagates the previous step's input and hidden spikes through the two
// ragged matrices into shared-memory fixed-point accumulators (sums independent of the
// order of the atomic additions), draws the new input spikes from Philox, updates the
// neurons and the leaky readout, and records spikes (bits), psi and y; a second kernel
// turns the recorded y into d = softmax(y) - onehot(label) for all steps in parallel.
//
// Gradient: e-prop's traces are linear in the presynaptic filtered spike train zbar_i
// with coefficients that depend only on the postsynaptic neuron j, so
//   G_ji = sum_t L_j^{t+1} ebar_ji^t = sum_{(b,t): z_i^{b,t} = 1} delta_j^{b,t}
// where delta is produced by a reverse-time scan per hidden neuron:
//   D_k^t  = d_k^{t+1} + alpha D_k^{t+1}               (filtered readout error)
//   lam^t  = sum_k W_out[k][j] D_k^t
//   mu^t   = beta lam^{t+1} psi^{t+1} + (rho - beta psi^{t+1}) mu^{t+1}
//   h^t    = psi^t (lam^t - mu^t)
//   delta^t = h^{t+1} + alpha delta^{t+1}
// (with zero values beyond the last step), and G_out[k][j] = sum over spikes of j of
// D_k.  The gather walks each presynaptic row's spike times and sums delta at the row's
// targets, so the per-synapse work is proportional to synaptic events, not to
// synapses x steps.  Partial sums over K-splits are reduced in a fixed order.
#include "common.cuh"

#include <cmath>
#include <type_traits>

namespace snn {


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

// Forward accumulators: each is a pair of 32-bit words {H, L} summing the two parts of
// every added fixed-point weight w = 2^20 w_hi + w_lo (w_hi = bits 51..20 of the packed
// slot as a signed 32-bit value, w_lo = bits 19..0): both sums use native 32-bit
// shared-memory atomics and are exact: L takes at most one addend (< 2^20) per spiking
// row, rows hold no repeated target and n_in + N <= 3072 < 4096; H wraps modulo 2^32
// like the 52-bit weights.  The total is 2^20 H + L.
__device__ __forceinline__ void acc_add(unsigned* acc, unsigned long long w) {
    const unsigned lo = (unsigned)w, hi = (unsigned)(w >> 32);
    unsigned* a = acc + 2 * (hi >> 20);                   // target index: bits 63..52
    atomicAdd(a, __funnelshift_r(lo, hi, 20));            // bits 51..20
    atomicAdd(a + 1, lo & 0xFFFFFu);                      // bits 19..0
}
// The accumulated sum 2^20 H + L in real units (40 fractional bits): H 2^-20 + L 2^-40,
// each product exact, one rounding in the sum (for double the same value as converting
// the 64-bit integer first).
template <typename real>
__device__ __forceinline__ real acc_real(const long long* acc) {
    const unsigned* a = (const unsigned*)acc;
    return (real)(int)a[0] * (real)9.5367431640625e-07 + (real)a[1] * (real)9.094947017729282e-13;
}

// Input spikes of every (trial, step) in parallel: they depend on (trial, step, channel)
// only, so they are drawn ahead of the sequential simulation.  Thread = 8 channels (one
// Philox block, one 32-bit half of a word per channel); the bytes of 4 consecutive
// threads form one 32-channel word.
__global__ void k_input(InputParams p) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
constexpr int FWD_ROWS = 2;   // spiking rows a warp propagates at a time

template <typename real, int NPT, int TH>
__global__ void __launch_bounds__(TH, 1024 / TH) k_forward(FwdParams<real> p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, K = p.K, Win = p.Win, Wh = p.Wh, n_in = p.n_in;
    const int R = n_in + N;
    long long* Iacc = (long long*)smem;           // [N + 64]: neurons, 32 per-lane spares, readouts
    int* lens = (int*)(Iacc + N + 64);            // [R + 1] packed row lengths (row R: empty)
    int* list = lens + R + 1;                     // [2][R] spiking rows by step parity
    int* lcnt = list + 2 * R;                     // [2]
    uint32_t* xw = (uint32_t*)(lcnt + 2);         // [Win] input spike words of the current step
    uint32_t* zb = xw + Win;                      // [2][Wh]

    const int b = blockIdx.x;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int nwarps = TH / 32;
    constexpr int RO_WARP = 1;                    // advances the readout in phase B
    const int t0 = p.t0;
    const int t_end = p.trial_T ? min(p.t0 + p.n_steps, max(p.trial_T[b], p.t0)) : p.t0 + p.n_steps;
    real vr[NPT], ar[NPT];
    {
        const int prv = (t0 - 1) & 1;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int j = tid + q * TH;
            vr[q] = j < N ? p.v[(size_t)b * N + j] : real(0);
            ar[q] = j < N ? p.a[(size_t)b * N + j] : real(0);
        }
        for (int j = tid; j < N + 64; j += TH) Iacc[j] = 0;
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
    real yk = 0, ysk = 0, bk = 0;
    if (warp == RO_WARP && lane < K) {
        yk = p.y[(size_t)b * K + lane];
        ysk = p.ysum[(size_t)b * K + lane];
        bk = p.b_out[lane];
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
    unsigned* acc = (unsigned*)Iacc;

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
        for (int k = warp; k < n_rows; k += FWD_ROWS * nwarps) {
            // FWD_ROWS rows per warp at a time, their packed chunks loaded together
            int nr[FWD_ROWS];
            const unsigned long long* pr[FWD_ROWS];
            int nmax = 0;
#pragma unroll
            for (int u = 0; u < FWD_ROWS; ++u) {
                const int r = (k + u * nwarps < n_rows) ? lprv[k + u * nwarps] : R;   // R: empty row
                nr[u] = lens[r];
                pr[u] = p.pk + (size_t)(r < R ? r : 0) * p.Cf;
                nmax = nr[u] > nmax ? nr[u] : nmax;
            }
            for (int s0 = 0; s0 < nmax; s0 += 128) {
                unsigned long long wv[FWD_ROWS][4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int u = 0; u < FWD_ROWS; ++u)   // warp-uniform chunk tests; slots past a
                        wv[u][q] = s0 + q * 32 < nr[u] ? pr[u][s0 + q * 32 + lane] : 0ull;   // length are padding
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int u = 0; u < FWD_ROWS; ++u)
                        if (s0 + q * 32 < nr[u]) acc_add(acc, wv[u][q]);
            }
        }
        __syncthreads();
        // ---------------- phase B: neurons; spike lists of step t
        if (warp == 0 && lane < Win) {
            uint32_t word = xnext;                 // x^t
            if (t + 1 < t_end) xnext = xrec_b[(size_t)(t + 1) * Win + lane];
            const int pos = atomicAdd(&lcnt[cur], __popc(word));
            for (int k = 0; word; ++k, word &= word - 1u) lcur[pos + k] = lane * 32 + __ffs(word) - 1;
            xw[lane] = 0u;
        }
        if (warp == RO_WARP && lane < K) {         // y^t from the readout sums W_out z^{t-1}
            yk = p.alpha * yk + acc_real<real>(Iacc + N + 32 + lane) + bk;
            Iacc[N + 32 + lane] = 0;
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
                const real I = acc_real<real>(Iacc + j);
                Iacc[j] = 0;
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

// d^t = softmax(y^t) - onehot(label) for every recorded (trial, step), in place over the
// y values the forward left in the d record.  A warp takes 32 consecutive steps of one
// trial: their rows are one contiguous span of 32 K values, read and written whole by
// the warp (coalesced); lane r computes row r from shared memory.
constexpr int SMX_WARPS = 4;

template <typename real>
__global__ void __launch_bounds__(SMX_WARPS * 32)
    k_softmax_d(real* __restrict__ d, const int32_t* __restrict__ labels, int n_classes,
                const int32_t* __restrict__ trial_T, int B, int T, int K, int t0, int n_steps) {
    extern __shared__ __align__(16) unsigned char smx_raw[];
    real* sh = (real*)smx_raw + (size_t)(threadIdx.x >> 5) * 32 * K;
    const int lane = lane_id();
    const int blocks_per_trial = (n_steps + 31) / 32;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wg >= (long long)B * blocks_per_trial) return;
    const int b = (int)(wg / blocks_per_trial);
    const int ts = t0 + (int)(wg % blocks_per_trial) * 32;          // first step of the span
    const int nr = min(32, t0 + n_steps - ts);                      // rows in the span
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

// Packed forward rows: row r < n_in is input row r, row n_in + j is hidden row j; Cf
// slots each.  A slot is bits 63..52 target accumulator, bits 51..0 the weight in fixed
// point (40 fractional bits, two's complement): one 64-bit load per slot, added with
// acc_add.  Hidden row j holds its len_j synapses, then its readout column W_out[k][j]
// aimed at accumulators N + 32 + k.  Slots past a row's length hold weight 0 aimed at
// the per-lane spare N + (slot mod 32), so a warp adds a row's last 32-slot chunk whole,
// with no per-lane test and no two lanes on one address.
template <typename real>
__global__ void k_pack(const real* __restrict__ w_in, const int32_t* __restrict__ ind_in,
                       const int32_t* __restrict__ len_in, int C_in, int n_in, const real* __restrict__ w_rec,
                       const int32_t* __restrict__ ind_rec, const int32_t* __restrict__ len_rec, int C_rec,
                       const real* __restrict__ W_out, int K, int N, int Cf, unsigned long long* __restrict__ pk,
                       long long n, unsigned long long* __restrict__ colsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = (int)(i / Cf), s = (int)(i % Cf);
    unsigned tgt = (unsigned)(N + (s & 31));
    long long f = 0;
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
    pk[i] = ((unsigned long long)tgt << 52) | ((unsigned long long)f & ((1ull << 52) - 1));
    if (f) atomicAdd(&colsum[tgt], (unsigned long long)(f < 0 ? -f : f));
}

// ------------------------------------------------------------------ backward
// G_b[k] = sum over trials of the per-trial partials: one CTA per readout, a strided
// sum per thread, then a fixed-order tree (deterministic).
constexpr int RGB_THREADS = 256;

template <typename real>
__global__ void __launch_bounds__(RGB_THREADS)
    k_reduce_gb(const real* __restrict__ gb_part, real* __restrict__ G_b, int B, int K) {
    __shared__ real red[RGB_THREADS];
    const int k = blockIdx.x;
    real s = 0;
    for (int b = threadIdx.x; b < B; b += RGB_THREADS) s += gb_part[(size_t)b * K + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = RGB_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) G_b[k] = red[0];
}

// Filtered readout error D_k^t = d_k^{t+1} + alpha D_k^{t+1} (D^{T-1} = 0), i.e.
// D_k^t = sum_{u > t} alpha^{u-t-1} d_k^u, and the bias gradient partial sum_t d_k^t.
// One warp per trial, lane k per readout (padding lanes k >= K write zeros): the warp
// walks the steps backwards reading and writing one contiguous row per step, with the
// rows of the next RS_AHEAD steps loaded ahead of the recurrence.
constexpr int RS_AHEAD = 8;

template <typename real>
__global__ void k_readout_scan(const real* __restrict__ d, real* __restrict__ Dout, real* __restrict__ gb_part,
                               int B, int T, int K, int Kp, real alpha) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int k = lane_id();
    if (b >= B || k >= Kp) return;
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

// The adjoint scan.  CTA = (trial, BWD_THREADS hidden neurons); steps are walked backwards
// in chunks of BWD_TCH.  Each thread prefetches its neuron's psi for the next chunk into
// registers while it runs the current chunk; the chunk's filtered readout error D
// [BWD_TCH][KP] is double-buffered in shared memory (one barrier per chunk).  Per step:
//   lam = sum_k W_out[k][j] D_k,  mu = beta lam' psi' + (rho - beta psi') mu',
//   h = psi (lam - mu),  delta = h' + alpha delta'   (primes: step t+1; zero after T-1).
constexpr int BWD_THREADS = 128;
constexpr int BWD_TCH = 8;

template <typename real, int KV>
__global__ void __launch_bounds__(BWD_THREADS)
    k_backward(const real* __restrict__ psi, const real* __restrict__ Dg, const real* __restrict__ W_out,
               real* __restrict__ delta, int T, int N, int K, real alpha, real rho, real beta) {
    constexpr int KP = 4 * KV;
    __shared__ __align__(16) real D_s[2][BWD_TCH][KP];
    const int tid = threadIdx.x;
    const int j = blockIdx.x * BWD_THREADS + tid;
    const int b = blockIdx.y;
    const bool ok = j < N;
    real wc[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) wc[k] = (k < K && ok) ? W_out[(size_t)k * N + j] : real(0);
    const real* pb = psi + (size_t)b * T * N + (ok ? j : 0);
    const real* Db = Dg + (size_t)b * T * KP;
    real* db = delta + (size_t)b * T * N + (ok ? j : 0);
    const int n_chunks = (T + BWD_TCH - 1) / BWD_TCH;
    real pcur[BWD_TCH], pnext[BWD_TCH];
    auto load_chunk = [&](int ch, real (&dst)[BWD_TCH], int buf) {
        const int tb = ch * BWD_TCH, nt = min(BWD_TCH, T - tb);
#pragma unroll
        for (int r = 0; r < BWD_TCH; ++r) dst[r] = (r < nt && ok) ? pb[(size_t)(tb + r) * N] : real(0);
        for (int idx = tid; idx < nt * KP; idx += BWD_THREADS) D_s[buf][idx / KP][idx % KP] = Db[(size_t)tb * KP + idx];
    };
    load_chunk(n_chunks - 1, pcur, (n_chunks - 1) & 1);
    __syncthreads();
    real lam_next = 0, psi_next = 0, mu = 0, h_next = 0, dl = 0;
    for (int ch = n_chunks - 1; ch >= 0; --ch) {
        const int tb = ch * BWD_TCH, nt = min(BWD_TCH, T - tb);
        const int buf = ch & 1;
        if (ch > 0) load_chunk(ch - 1, pnext, buf ^ 1);
#pragma unroll
        for (int r = BWD_TCH - 1; r >= 0; --r) {
            if (r < nt) {
                const int t = tb + r;
                const real ps = pcur[r];
                real lam = 0;
#pragma unroll
                for (int k = 0; k < KP; ++k) lam += wc[k] * D_s[buf][r][k];
                if (t == T - 1) {
                    mu = 0;
                    dl = 0;
                } else {
                    mu = beta * lam_next * psi_next + (rho - beta * psi_next) * mu;
                    dl = h_next + alpha * dl;
                }
                const real h = ps * (lam - mu);
                if (ok) db[(size_t)t * N] = dl;
                h_next = h;
                lam_next = lam;
                psi_next = ps;
            }
        }
#pragma unroll
        for (int r = 0; r < BWD_TCH; ++r) pcur[r] = pnext[r];
        __syncthreads();
    }
}

// Gather order of a ragged row: its live slots as keys (target << 11) | slot, sorted
// ascending (targets are distinct within a row).  With sorted targets the 32 lanes of
// one gather chunk read a narrow band of the adjoint row, so the chunks of one spike
// event touch few 32-byte sectors more than once.  Warp per row, rank by counting;
// blockDim.x / 32 warps per CTA, each with a C-word shared-memory row.
__global__ void __launch_bounds__(256)
    k_sort_rows(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, int P, int C,
                int32_t* __restrict__ keys) {
    extern __shared__ int32_t sk[];                  // [warps][C]
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= P) return;
    int32_t* row = sk + (size_t)warp * C;
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
constexpr int GATHER_SPAN = 8192;
constexpr int GATHER_ROWS = 16;   // rows (warps) per CTA: 32, 16 or 8
constexpr int GATHER_EV = 4;      // spike events whose loads are issued together

template <typename real, int ROWS, int EV>
__global__ void __launch_bounds__(ROWS * 32, 1)
    k_gather(const uint32_t* __restrict__ x_rec, const uint32_t* __restrict__ z_rec, int Win, int Wh,
             const int32_t* __restrict__ in_len, const int32_t* __restrict__ in_keys, int in_C, int n_in,
             const int32_t* __restrict__ rec_len, const int32_t* __restrict__ rec_keys, int rec_C, int N,
             const real* __restrict__ delta, const real* __restrict__ D, int K, int Kp, long long BT,
             long long bt_per, real* __restrict__ part_in, real* __restrict__ part_rec,
             real* __restrict__ part_out) {
    __shared__ uint32_t words[GATHER_SPAN];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    constexpr int SPLIT = 32 / ROWS;
    const int col = blockIdx.x / SPLIT;
    const int r0 = (blockIdx.x % SPLIT) * ROWS;    // first row of the word this CTA owns
    const int ks = blockIdx.y;
    const int g = blockIdx.z;                       // slot group: slots [128 g, 128 g + 128)
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
    for (int k = threadIdx.x; k < GATHER_SPAN; k += ROWS * 32) {
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
    if (do_out) part_out[((size_t)ks * N + i) * K + lane] = acc_o;
}

template <typename real>
__global__ void k_reduce_ragged(const real* __restrict__ part, const int32_t* __restrict__ len, int P, int C, int KS,
                                real* __restrict__ grad) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * C) return;
    int i = (int)(idx / C), s = (int)(idx % C);
    real g = 0;
    if (s < len[i])
        for (int k = 0; k < KS; ++k) g += part[(size_t)k * P * C + idx];
    grad[idx] = g;
}

template <typename real>
__global__ void k_reduce_out(const real* __restrict__ part, int N, int K, int KS, real* __restrict__ G_out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * K) return;
    int j = idx / K, k = idx % K;
    real g = 0;
    for (int s = 0; s < KS; ++s) g += part[((size_t)s * N + j) * K + k];
    G_out[(size_t)k * N + j] = g;
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

// beta1^t, beta2^t for a step count read from device memory, kept in the handle's device
// state: one multiplication per call when t advances by one (graph replay), a fresh
// running product otherwise.  At most 2^24 multiplications per call: a larger jump sets
// the invalid-state flag and keeps the partial product (a later call continues it).
__global__ void k_adam_bias(const long long* __restrict__ step_dev, double beta1, double beta2, AdamBias* st,
                            int32_t* status) {
    long long t = *step_dev;
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

struct NoiseK {
    double amp;                    // sqrt(2 lr temperature); 0 = off
    uint64_t seed, idx;
    const int64_t* idx_dev;
};

template <typename real>
__global__ void k_adam_ragged(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, int P, int C, int Qw,
                              real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                              const real* __restrict__ grad, const uint32_t* __restrict__ sign, real l1, real lr,
                              real b1, real b2, real omb1, real omb2, real eps, real bc1, real bc2,
                              const double* __restrict__ bias_dev, NoiseK nz) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * C) return;
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
__global__ void k_adam_dense(real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                             const real* __restrict__ grad, int n, real lr, real b1, real b2, real omb1,
                             real omb2, real eps, real bc1, real bc2, const double* __restrict__ bias_dev) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    bias_from_device(bias_dev, bc1, bc2);
    real ww = w[idx], mm = m[idx], vv = v[idx];
    adam_update(ww, mm, vv, grad[idx], lr, b1, b2, omb1, omb2, eps, bc1, bc2);
    w[idx] = ww;
    m[idx] = mm;
    v[idx] = vv;
}

// ------------------------------------------------------------------ host side
static size_t fwd_smem(int n_in, int N, int Win, int Wh) {
    return (size_t)(N + 64) * 8 + (size_t)(n_in + N + 1) * 4 + (size_t)(n_in + N) * 4 * 2 + 8 +
           (size_t)(Win + 2 * Wh) * 4;
}

template <typename real, int NPT, int TH>
static snn_status launch_forward(const FwdParams<real>& p, int B, size_t smem, cudaStream_t s) {
    // raise the dynamic shared-memory limit once per device and size (not inside graph capture)
    static int set_for[64] = {0};
    int dev = 0;
    SNN_CUDA(cudaGetDevice(&dev));
    if (smem > 48 * 1024 && dev < 64 && set_for[dev] < (int)smem) {
        SNN_CUDA(cudaFuncSetAttribute(k_forward<real, NPT, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        set_for[dev] = (int)smem;
    }
    k_forward<real, NPT, TH><<<B, TH, smem, s>>>(p);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

// Row schedule: TH threads (TH / 32 warps) share one trial's spiking rows.
template <typename real, int TH>
static snn_status launch_forward_th(const FwdParams<real>& p, int B, size_t smem, cudaStream_t s) {
    const int npt = (p.N + TH - 1) / TH;
    if (npt <= 1) return launch_forward<real, 1, TH>(p, B, smem, s);
    if (npt <= 2) return launch_forward<real, 2, TH>(p, B, smem, s);
    if (npt <= 4) return launch_forward<real, 4, TH>(p, B, smem, s);
    if (npt <= 8) return launch_forward<real, 8, TH>(p, B, smem, s);
    SNN_REQUIRE(false, "snn_step_neurons: N = %d too large for %d threads per trial", p.N, TH);
}

template <typename real>
static snn_status refresh_fixed(snn_classifier* c, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const long long n = (long long)(d.n_in + d.N) * c->Cf;
    SNN_CUDA(cudaMemsetAsync(c->colsum, 0, (size_t)(d.N + 64) * sizeof(unsigned long long), s));
    k_pack<real><<<ceil_div(n, 256), 256, 0, s>>>(
        (const real*)d.w_in->d.w, d.w_in->d.ind, d.w_in->d.row_len, d.w_in->d.C, d.n_in, (const real*)d.w_rec->d.w,
        d.w_rec->d.ind, d.w_rec->d.row_len, d.w_rec->d.C, (const real*)d.W_out, d.K, d.N, c->Cf,
        (unsigned long long*)c->pk, n, c->colsum);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

static snn_status draw_impl(snn_classifier* c, const snn_batch* bt, int t0, int n_steps, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const int Win = (d.n_in + 31) / 32;
    InputParams ip;
    ip.n_in = d.n_in;
    ip.Win = Win;
    ip.T = bt->T;
    ip.t0 = t0;
    ip.n_steps = n_steps;
    ip.n_bins = d.n_bins;
    ip.n_classes = d.n_classes;
    ip.B = bt->B;
    ip.in_thr = d.in_thr;
    ip.seed = d.in_seed;
    ip.labels = bt->labels;
    ip.bin_len = bt->bin_len;
    ip.trial_ids = bt->trial_ids;
    ip.x_rec = bt->x_rec;
    ip.status = d.w_in->status;
    ip.trial_T = bt->trial_T;
    const long long groups = (long long)bt->B * n_steps * Win * 4;
    k_input<<<ceil_div(groups, 256), 256, 0, s>>>(ip);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

template <typename real>
static snn_status step_impl(snn_classifier* c, const snn_batch* bt, int t0, int n_steps, bool inputs_ready,
                            cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const int Win = (d.n_in + 31) / 32, Wh = (d.N + 31) / 32;
    if (!inputs_ready) {
        const snn_status st = draw_impl(c, bt, t0, n_steps, s);
        if (st != SNN_OK) return st;
    }

    FwdParams<real> p;
    p.n_in = d.n_in;
    p.N = d.N;
    p.K = d.K;
    p.Win = Win;
    p.Wh = Wh;
    p.T = bt->T;
    p.t0 = t0;
    p.n_steps = n_steps;
    p.alpha = (real)c->alpha;
    p.rho = (real)c->rho;
    p.beta = (real)d.beta;
    p.v_thr = (real)d.v_thr;
    p.psi_scale = (real)(0.3 / d.v_thr);
    p.inv_vthr = (real)(1.0 / d.v_thr);
    p.in_len = d.w_in->d.row_len;
    p.rec_len = d.w_rec->d.row_len;
    p.pk = (const unsigned long long*)c->pk;
    p.Cf = c->Cf;
    p.b_out = (const real*)d.b_out;
    p.v = (real*)bt->v;
    p.a = (real*)bt->a;
    p.y = (real*)bt->y;
    p.ysum = (real*)bt->ysum;
    p.x_bits = bt->x_bits;
    p.z_bits = bt->z_bits;
    p.x_rec = bt->x_rec;
    p.z_rec = bt->z_rec;
    p.psi_rec = (real*)bt->psi_rec;
    p.d_rec = (real*)bt->d_rec;
    p.v_rec = (real*)bt->v_rec;
    p.a_rec = (real*)bt->a_rec;
    p.y_rec = (real*)bt->y_rec;
    p.record_state = (bt->v_rec && bt->a_rec) ? 1 : 0;
    p.trial_T = bt->trial_T;
    p.colsum = c->colsum;
    p.status = d.w_in->status;
    const size_t smem = fwd_smem(d.n_in, d.N, Win, Wh);
    snn_status st = refresh_fixed<real>(c, s);
    if (st != SNN_OK) return st;
    SNN_REQUIRE(smem <= 227 * 1024, "snn_step_neurons: n_in = %d, N = %d need %zu bytes of shared memory (max 227 KB)",
                d.n_in, d.N, smem);
    switch (c->fwd_threads) {
        case 128: st = launch_forward_th<real, 128>(p, bt->B, smem, s); break;
        case 512: st = launch_forward_th<real, 512>(p, bt->B, smem, s); break;
        default: st = launch_forward_th<real, 256>(p, bt->B, smem, s); break;
    }
    if (st != SNN_OK || !bt->d_rec) return st;
    const long long warps = (long long)bt->B * ((n_steps + 31) / 32);
    const size_t smx = (size_t)SMX_WARPS * 32 * d.K * sizeof(real);   // <= 32 KB (K <= 32)
    k_softmax_d<real><<<ceil_div(warps, SMX_WARPS), SMX_WARPS * 32, smx, s>>>(
        (real*)bt->d_rec, bt->labels, d.n_classes, bt->trial_T, bt->B, bt->T, d.K, t0, n_steps);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
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

template <int KV>
__global__ void __launch_bounds__(BWD_THREADS)
    k_backward_x2(const float* __restrict__ psi, const float* __restrict__ Dg, const float* __restrict__ W_out,
                  float* __restrict__ delta, int T, int N, int K, float alpha, float rho, float beta) {
    constexpr int KP = 4 * KV;
    __shared__ __align__(16) float D_s[2][BWD2_TCH][KP];
    const int tid = threadIdx.x;
    const int jp = blockIdx.x * BWD_THREADS + tid;     // neuron pair
    const int N2 = N >> 1;
    const int b = blockIdx.y;
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
        for (int idx = tid; idx < nt * KP; idx += BWD_THREADS) D_s[buf][idx / KP][idx % KP] = Db[(size_t)tb * KP + idx];
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

// ---- bulk-copy staging of the adjoint scan (TMA 1-D copies into shared memory)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait for the barrier's phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
    return done != 0;
}
// Failure-detection probe: one warp waits, bounded, on an mbarrier that completes only
// if `arrive` is set; a wait that gives up sets ST_TIMEOUT, as the adjoint scan does.
// No copy is in flight, so giving up leaves nothing behind.
__global__ void k_wait_probe(int arrive, int limit, int32_t* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncwarp();
    if (threadIdx.x == 0 && arrive)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    __syncwarp();
    const bool got = mbar_wait(&bar, 0u, limit);
    if (threadIdx.x == 0 && !got) atomicOr(status, ST_TIMEOUT);
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) that
// completes its byte count on the barrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// FP32 adjoint scan, two neurons per thread, psi and D staged by bulk copies: CTA =
// (trial, 256 neurons); steps walked backwards in chunks of BB_S, BB_NST chunks in
// flight.  Thread 0 issues, per chunk, one bulk copy per step row of the CTA's psi slice
// (up to 1 KB) and one for the chunk's D rows, all completing on that stage's mbarrier;
// every thread reads its neuron pair's psi from shared memory.  The same recurrences
// and arithmetic as k_backward_x2 (bit-identical results).  Needs N % 4 == 0.  A wait
// that gives up sets SNN_ETIMEOUT's flag, lets the copies in flight land (bounded) and
// ends the CTA.
constexpr bool BWD_BULK = true;
constexpr int BB_THREADS = 128;
constexpr int BB_S = 8;
constexpr int BB_NST = 3;
constexpr int BB_WAIT = 1 << 22;

template <int KV>
__global__ void __launch_bounds__(BB_THREADS)
    k_backward_bulk(const float* __restrict__ psi, const float* __restrict__ Dg, const float* __restrict__ W_out,
                    float* __restrict__ delta, int T, int N, int K, float alpha, float rho, float beta,
                    int32_t* status) {
    constexpr int KP = 4 * KV;
    __shared__ __align__(128) float ps_s[BB_NST][BB_S][2 * BB_THREADS];
    __shared__ __align__(16) float D_s[BB_NST][BB_S][KP];
    __shared__ __align__(8) uint64_t bar[BB_NST];
    const int tid = threadIdx.x;
    const int j0 = blockIdx.x * 2 * BB_THREADS;             // first neuron of the CTA
    const int ncols = min(2 * BB_THREADS, N - j0);          // multiple of 4 (N % 4 == 0)
    const int jp = blockIdx.x * BB_THREADS + tid;            // neuron pair
    const int N2 = N >> 1;
    const int b = blockIdx.y;
    const bool ok = jp < N2;
    unsigned long long wa[KP / 2], wb[KP / 2];
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
    const float* pb = psi + (size_t)b * T * N + j0;
    const float* Db = Dg + (size_t)b * T * KP;
    unsigned long long* db = (unsigned long long*)delta + (size_t)b * T * N2 + (ok ? jp : 0);
    const int n_chunks = (T + BB_S - 1) / BB_S;
    if (tid == 0) {
        for (int st = 0; st < BB_NST; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // chunk q (0 = last in time) -> chunk index n_chunks-1-q, stage q % BB_NST
    auto issue = [&](int q) {
        const int ch = n_chunks - 1 - q, st = q % BB_NST;
        const int tb = ch * BB_S, nt = min(BB_S, T - tb);
        mbar_expect_tx(&bar[st], (uint32_t)(nt * ncols * 4 + nt * KP * 4));
        for (int r = 0; r < nt; ++r)
            bulk_g2s(ps_s[st][r], pb + (size_t)(tb + r) * N, (uint32_t)(ncols * 4), &bar[st]);
        bulk_g2s(D_s[st][0], Db + (size_t)tb * KP, (uint32_t)(nt * KP * 4), &bar[st]);
    };
    if (tid == 0)
        for (int q = 0; q < BB_NST && q < n_chunks; ++q) issue(q);
    const unsigned long long alpha2 = f2_pack(alpha, alpha), beta2 = f2_pack(beta, beta);
    const unsigned long long rho2 = f2_pack(rho, rho), nbeta2 = f2_pack(-beta, -beta);
    unsigned long long lam_next = 0, psi_next = 0, mu = 0, h_next = 0, dl = 0;
    for (int q = 0; q < n_chunks; ++q) {
        const int ch = n_chunks - 1 - q, st = q % BB_NST;
        const int tb = ch * BB_S, nt = min(BB_S, T - tb);
        const bool got = mbar_wait(&bar[st], (uint32_t)((q / BB_NST) & 1), BB_WAIT);
        if (__syncthreads_or(!got)) {
            // give up: record it, let every copy still in flight land, end the CTA
            if (tid == 0) {
                atomicOr(status, ST_TIMEOUT);
                for (int q2 = q; q2 < n_chunks && q2 < q + BB_NST; ++q2)
                    mbar_wait(&bar[q2 % BB_NST], (uint32_t)((q2 / BB_NST) & 1), BB_WAIT);
            }
            __syncthreads();
            return;
        }
#pragma unroll
        for (int r = BB_S - 1; r >= 0; --r) {
            if (r < nt) {
                const int t = tb + r;
                const unsigned long long ps = ((const unsigned long long*)ps_s[st][r])[tid];
                const unsigned long long* Dr = (const unsigned long long*)D_s[st][r];
                unsigned long long sa = 0, sb = 0;
#pragma unroll
                for (int m = 0; m < KP / 2; ++m) {
                    const unsigned long long dk = Dr[m];
                    sa = f2_fma(wa[m], dk, sa);
                    sb = f2_fma(wb[m], dk, sb);
                }
                const unsigned long long lam = f2_pack(f2_lo(sa) + f2_hi(sa), f2_lo(sb) + f2_hi(sb));
                if (t == T - 1) {
                    mu = 0;
                    dl = 0;
                } else {
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
        __syncthreads();                                     // stage st fully read
        if (tid == 0 && q + BB_NST < n_chunks) issue(q + BB_NST);
    }
}

template <typename real, int KV>
static void launch_backward(const snn_classifier* c, const snn_batch* bt, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    if (std::is_same<real, float>::value && d.N % 4 == 0 && BWD_BULK) {
        dim3 g(ceil_div(d.N, 2 * BB_THREADS), bt->B);
        k_backward_bulk<KV><<<g, BB_THREADS, 0, s>>>((const float*)bt->psi_rec, (const float*)bt->Dout,
                                                      (const float*)d.W_out, (float*)bt->delta, bt->T, d.N, d.K,
                                                      (float)c->alpha, (float)c->rho, (float)d.beta,
                                                      d.w_rec->status);
        return;
    }
    if (std::is_same<real, float>::value && d.N % 2 == 0) {
        dim3 g(ceil_div(d.N / 2, BWD_THREADS), bt->B);
        k_backward_x2<KV><<<g, BWD_THREADS, 0, s>>>((const float*)bt->psi_rec, (const float*)bt->Dout,
                                                     (const float*)d.W_out, (float*)bt->delta, bt->T, d.N, d.K,
                                                     (float)c->alpha, (float)c->rho, (float)d.beta);
        return;
    }
    dim3 g(ceil_div(d.N, BWD_THREADS), bt->B);
    k_backward<real, KV><<<g, BWD_THREADS, 0, s>>>((const real*)bt->psi_rec, (const real*)bt->Dout,
                                                   (const real*)d.W_out, (real*)bt->delta, bt->T, d.N, d.K,
                                                   (real)c->alpha, (real)c->rho, (real)d.beta);
}

template <typename real>
static snn_status grad_impl(snn_classifier* c, const snn_batch* bt, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const int B = bt->B, T = bt->T, N = d.N, K = d.K, Kp = (K + 3) & ~3;
    const int Win = (d.n_in + 31) / 32, Wh = (N + 31) / 32;
    real* gb_part = (real*)c->part_out + (size_t)c->KS * N * K;
    k_readout_scan<real><<<ceil_div((long long)B * 32, 128), 128, 0, s>>>(
        (const real*)bt->d_rec, (real*)bt->Dout, gb_part, B, T, K, Kp, (real)c->alpha);
    SNN_LAUNCH_CHECK();
    switch (Kp / 4) {
        case 1: launch_backward<real, 1>(c, bt, s); break;
        case 2: launch_backward<real, 2>(c, bt, s); break;
        case 3: launch_backward<real, 3>(c, bt, s); break;
        case 4: launch_backward<real, 4>(c, bt, s); break;
        case 5: launch_backward<real, 5>(c, bt, s); break;
        case 6: launch_backward<real, 6>(c, bt, s); break;
        case 7: launch_backward<real, 7>(c, bt, s); break;
        default: launch_backward<real, 8>(c, bt, s); break;
    }
    SNN_LAUNCH_CHECK();
    k_reduce_gb<real><<<K, RGB_THREADS, 0, s>>>(gb_part, (real*)d.G_b, B, K);
    SNN_LAUNCH_CHECK();
    const long long BT = (long long)B * T;
    const int KS = c->KS;
    const long long bt_per = ((BT + KS - 1) / KS + 31) / 32 * 32;
    SNN_REQUIRE(bt_per <= GATHER_SPAN, "snn_eprop_update: internal K-split too small");
    const snn_ragged_desc& ri = d.w_in->d;
    const snn_ragged_desc& rr = d.w_rec->d;
    const int Cmax = ri.C > rr.C ? ri.C : rr.C;
    int32_t* keys_in = c->gkeys;
    int32_t* keys_rec = c->gkeys + (size_t)ri.P * ri.C;
    for (int m = 0; m < 2; ++m) {
        const snn_ragged_desc& rd = m == 0 ? ri : rr;
        const int sw = rd.C <= 1536 ? 8 : 6;       // warps per CTA: at most 48 KB of rows
        k_sort_rows<<<ceil_div(rd.P, sw), sw * 32, (size_t)sw * rd.C * 4, s>>>(rd.row_len, rd.ind, rd.P, rd.C,
                                                                                  m == 0 ? keys_in : keys_rec);
        SNN_LAUNCH_CHECK();
    }
    dim3 gg((Win + Wh) * (32 / GATHER_ROWS), KS, (Cmax + 127) / 128);
    k_gather<real, GATHER_ROWS, GATHER_EV><<<gg, GATHER_ROWS * 32, 0, s>>>(
        bt->x_rec, bt->z_rec, Win, Wh, ri.row_len, keys_in, ri.C, d.n_in,
        rr.row_len, keys_rec, rr.C, N, (const real*)bt->delta, (const real*)bt->Dout, K, Kp, BT, bt_per,
        (real*)c->part_in, (real*)c->part_rec, (real*)c->part_out);
    SNN_LAUNCH_CHECK();
    k_reduce_ragged<real><<<ceil_div((long long)ri.P * ri.C, 256), 256, 0, s>>>((const real*)c->part_in, ri.row_len,
                                                                                ri.P, ri.C, KS, (real*)ri.grad);
    SNN_LAUNCH_CHECK();
    k_reduce_ragged<real><<<ceil_div((long long)rr.P * rr.C, 256), 256, 0, s>>>(
        (const real*)c->part_rec, rr.row_len, rr.P, rr.C, KS, (real*)rr.grad);
    SNN_LAUNCH_CHECK();
    k_reduce_out<real><<<ceil_div(N * K, 256), 256, 0, s>>>((const real*)c->part_out, N, K, KS, (real*)d.G_out);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

// beta1^t, beta2^t on the host, continued from the handle's cache when it matches.
static void host_adam_bias(snn_classifier* c, double beta1, double beta2, long long t, double& b1t, double& b2t) {
    if (!(c->h_beta1 == beta1 && c->h_beta2 == beta2 && c->h_t >= 0 && c->h_t <= t)) {
        c->h_b1t = c->h_b2t = 1.0;
        c->h_t = 0;
        c->h_beta1 = beta1;
        c->h_beta2 = beta2;
    }
    adam_bias_advance(beta1, beta2, c->h_t, c->h_b1t, c->h_b2t, t, 1ll << 62);
    c->h_t = t;
    b1t = c->h_b1t;
    b2t = c->h_b2t;
}

template <typename real>
static snn_status apply_impl(snn_classifier* c, const snn_adam* ad, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const real lr = (real)ad->lr, b1 = (real)ad->beta1, b2 = (real)ad->beta2, eps = (real)ad->eps;
    double b1t = 1.0, b2t = 1.0;
    const double* bias_dev = nullptr;
    if (ad->step_dev) {
        k_adam_bias<<<1, 1, 0, s>>>((const long long*)ad->step_dev, ad->beta1, ad->beta2, (AdamBias*)c->adam_dev,
                                    d.w_in->status);
        SNN_LAUNCH_CHECK();
        bias_dev = (const double*)c->adam_dev;          // {beta1^t, beta2^t} at its start
    } else {
        host_adam_bias(c, ad->beta1, ad->beta2, ad->step, b1t, b2t);
    }
    const real bc1 = (real)(1.0 - b1t), bc2 = (real)(1.0 - b2t);
    const real omb1 = (real)(1.0 - ad->beta1), omb2 = (real)(1.0 - ad->beta2);
    for (snn_ragged* r : {d.w_in, d.w_rec}) {
        const snn_ragged_desc& rd = r->d;
        const uint32_t* sign = (ad->l1 != 0.0) ? rd.sign_bits : nullptr;
        NoiseK nz;
        nz.amp = ad->temperature > 0.0 ? std::sqrt(2.0 * ad->lr * ad->temperature) : 0.0;
        nz.seed = rd.seed;
        nz.idx = (uint64_t)ad->noise_idx;
        nz.idx_dev = ad->noise_idx_dev;
        k_adam_ragged<real><<<ceil_div((long long)rd.P * rd.C, 256), 256, 0, s>>>(
            rd.row_len, rd.ind, rd.P, rd.C, r->Qw, (real*)rd.w, (real*)rd.m, (real*)rd.v, (const real*)rd.grad, sign,
            (real)ad->l1, lr, b1, b2, omb1, omb2, eps, bc1, bc2, bias_dev, nz);
        SNN_LAUNCH_CHECK();
    }
    k_adam_dense<real><<<ceil_div(d.K * d.N, 256), 256, 0, s>>>((real*)d.W_out, (real*)d.W_out_m, (real*)d.W_out_v,
                                                                (const real*)d.G_out, d.K * d.N, lr, b1, b2, omb1,
                                                                omb2, eps, bc1, bc2, bias_dev);
    SNN_LAUNCH_CHECK();
    k_adam_dense<real><<<1, 32, 0, s>>>((real*)d.b_out, (real*)d.b_m, (real*)d.b_v, (const real*)d.G_b, d.K, lr, b1,
                                        b2, omb1, omb2, eps, bc1, bc2, bias_dev);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // namespace snn

using namespace snn;

extern "C" {

snn_status snn_create_classifier(const snn_classifier_desc* d, snn_classifier** out) {
    clear_error();
    SNN_REQUIRE(d && out, "snn_create_classifier: NULL argument");
    *out = nullptr;
    SNN_REQUIRE(d->n_in > 0 && d->N > 0 && d->K > 0 && d->K <= 32, "snn_create_classifier: need n_in, N > 0 and 0 < K <= 32");
    SNN_REQUIRE(d->dtype == SNN_F32 || d->dtype == SNN_F64, "snn_create_classifier: bad dtype");
    SNN_REQUIRE(d->w_in && d->w_rec, "snn_create_classifier: w_in and w_rec handles are required");
    SNN_REQUIRE(d->w_in->d.P == d->n_in && d->w_in->d.Q == d->N, "snn_create_classifier: w_in must be n_in x N");
    SNN_REQUIRE(d->w_rec->d.P == d->N && d->w_rec->d.Q == d->N, "snn_create_classifier: w_rec must be N x N");
    SNN_REQUIRE(d->w_in->d.dtype == d->dtype && d->w_rec->d.dtype == d->dtype,
                "snn_create_classifier: ragged dtypes must match the classifier dtype");
    SNN_REQUIRE(d->in_thr && d->W_out && d->b_out && d->G_out && d->G_b, "snn_create_classifier: NULL array");
    SNN_REQUIRE(d->n_classes > 0 && d->n_bins > 0, "snn_create_classifier: n_classes, n_bins must be > 0");
    SNN_REQUIRE(d->tau_m > 0 && d->dt > 0 && d->v_thr > 0, "snn_create_classifier: tau_m, dt, v_thr must be > 0");
    SNN_REQUIRE(d->max_B > 0 && d->max_T > 0, "snn_create_classifier: max_B, max_T must be > 0");
    SNN_REQUIRE(d->w_in->d.C <= 2048 && d->w_rec->d.C <= 2048, "snn_create_classifier: row capacity must be <= 2048");
    SNN_REQUIRE(d->N <= 8 * 256, "snn_create_classifier: N must be <= 2048");
    SNN_REQUIRE(d->N + 64 <= 4096, "snn_create_classifier: N + 64 accumulators must fit the 12-bit packed target");
    SNN_REQUIRE(d->n_in <= 1024, "snn_create_classifier: n_in must be <= 1024");
    snn_classifier* c = (snn_classifier*)calloc(1, sizeof(snn_classifier));
    if (!c) {
        set_error("snn_create_classifier: out of host memory");
        return SNN_ENOMEM;
    }
    c->d = *d;
    c->fwd_threads = 256;
    c->alpha = std::exp(-d->dt / d->tau_m);
    c->rho = d->tau_a > 0 ? std::exp(-d->dt / d->tau_a) : 0.0;
    long long BT = (long long)d->max_B * d->max_T;
    // K-splits of the gather: each CTA stages at most 8192 (trial, step) spike words
    c->KS = (int)((BT + 8191) / 8192);
    const int c_rec = d->w_rec->d.C + d->K;
    c->Cf = ((d->w_in->d.C > c_rec ? d->w_in->d.C : c_rec) + 31) / 32 * 32;
    size_t rsz = d->dtype == SNN_F32 ? 4 : 8;
    size_t n_in_part = (size_t)c->KS * d->w_in->d.P * d->w_in->d.C * rsz;
    size_t n_rec_part = (size_t)c->KS * d->w_rec->d.P * d->w_rec->d.C * rsz;
    size_t n_out_part = ((size_t)c->KS * d->N * d->K + (size_t)d->max_B * d->K) * rsz;
    cudaError_t e = cudaMalloc(&c->part_in, n_in_part);
    if (e == cudaSuccess) e = cudaMalloc(&c->part_rec, n_rec_part);
    if (e == cudaSuccess) e = cudaMalloc(&c->part_out, n_out_part);
    if (e == cudaSuccess) e = cudaMalloc(&c->pk, (size_t)(d->n_in + d->N) * c->Cf * 8);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->gkeys, ((size_t)d->w_in->d.P * d->w_in->d.C + (size_t)d->w_rec->d.P * d->w_rec->d.C) * 4);
    c->h_b1t = c->h_b2t = 1.0;
    c->h_beta1 = c->h_beta2 = -1.0;
    c->h_t = 0;
    if (e == cudaSuccess) e = cudaMalloc(&c->adam_dev, sizeof(AdamBias));
    if (e == cudaSuccess) e = cudaMalloc(&c->colsum, (size_t)(d->N + 64) * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        const AdamBias init = {1.0, 1.0, -1.0, -1.0, 0, 0};
        e = cudaMemcpy(c->adam_dev, &init, sizeof(AdamBias), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        snn_destroy_classifier(c);
        set_error("snn_create_classifier: cudaMalloc failed: %s", cudaGetErrorString(e));
        return SNN_ENOMEM;
    }
    *out = c;
    return SNN_OK;
}

snn_status snn_classifier_set_schedule(snn_classifier* c, int32_t warps_per_trial) {
    clear_error();
    SNN_REQUIRE(c, "snn_classifier_set_schedule: NULL classifier");
    SNN_REQUIRE(warps_per_trial == 4 || warps_per_trial == 8 || warps_per_trial == 16,
                "snn_classifier_set_schedule: warps_per_trial must be 4, 8 or 16");
    SNN_REQUIRE(c->d.N <= 8 * 32 * warps_per_trial, "snn_classifier_set_schedule: N = %d needs more warps", c->d.N);
    c->fwd_threads = 32 * warps_per_trial;
    return SNN_OK;
}

snn_status snn_destroy_classifier(snn_classifier* c) {
    if (!c) return SNN_OK;
    cudaFree(c->part_in);
    cudaFree(c->part_rec);
    cudaFree(c->part_out);
    cudaFree(c->pk);
    cudaFree(c->gkeys);
    cudaFree(c->adam_dev);
    cudaFree(c->colsum);
    free(c);
    return SNN_OK;
}

static snn_status check_batch(const snn_classifier* c, const snn_batch* b) {
    SNN_REQUIRE(b, "NULL batch");
    SNN_REQUIRE(b->B > 0 && b->T > 0, "batch B and T must be > 0");
    SNN_REQUIRE(b->B <= c->d.max_B && b->T <= c->d.max_T, "batch (B=%d, T=%d) exceeds the classifier's max (%d, %d)",
                b->B, b->T, c->d.max_B, c->d.max_T);
    SNN_REQUIRE(b->labels && b->bin_len && b->trial_ids && b->v && b->a && b->y && b->ysum && b->x_bits &&
                    b->z_bits && b->x_rec && b->z_rec,
                "batch has a NULL required array");
    return SNN_OK;
}

snn_status snn_step_neurons_ex(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps, int32_t flags,
                               snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_step_neurons: NULL classifier");
    snn_status st = check_batch(c, b);
    if (st != SNN_OK) return st;
    SNN_REQUIRE(t0 >= 0 && n_steps >= 0 && t0 + n_steps <= b->T, "snn_step_neurons: steps [%d, %d) outside [0, %d)",
                t0, t0 + n_steps, b->T);
    SNN_REQUIRE((flags & ~SNN_STEP_INPUTS_READY) == 0, "snn_step_neurons_ex: unknown flags 0x%x", flags);
    if (n_steps == 0) return SNN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool ready = (flags & SNN_STEP_INPUTS_READY) != 0;
    return c->d.dtype == SNN_F32 ? step_impl<float>(c, b, t0, n_steps, ready, s)
                                 : step_impl<double>(c, b, t0, n_steps, ready, s);
}

snn_status snn_step_neurons(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps, snn_stream stream) {
    return snn_step_neurons_ex(c, b, t0, n_steps, 0, stream);
}

snn_status snn_draw_inputs(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_draw_inputs: NULL classifier");
    snn_status st = check_batch(c, b);
    if (st != SNN_OK) return st;
    SNN_REQUIRE(t0 >= 0 && n_steps >= 0 && t0 + n_steps <= b->T, "snn_draw_inputs: steps [%d, %d) outside [0, %d)",
                t0, t0 + n_steps, b->T);
    if (n_steps == 0) return SNN_OK;
    return draw_impl(c, b, t0, n_steps, (cudaStream_t)stream);
}

snn_status snn_adam_bias(double beta1, double beta2, int64_t step, double* out) {
    clear_error();
    SNN_REQUIRE(out, "snn_adam_bias: NULL output");
    SNN_REQUIRE(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0, "snn_adam_bias: betas must be in [0, 1)");
    SNN_REQUIRE(step >= 0, "snn_adam_bias: step must be >= 0");
    double b1 = 1.0, b2 = 1.0;
    adam_bias_advance(beta1, beta2, 0, b1, b2, step, 1ll << 62);
    out[0] = b1;
    out[1] = b2;
    return SNN_OK;
}

snn_status snn_test_wait_timeout(snn_ragged* r, int32_t arrive, int32_t limit, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && limit > 0 && limit <= (1 << 24), "snn_test_wait_timeout: bad argument");
    k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(arrive ? 1 : 0, limit, r->status);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_eprop_update(snn_classifier* c, const snn_batch* b, int32_t phase, const snn_adam* adam,
                            snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_eprop_update: NULL classifier");
    cudaStream_t s = (cudaStream_t)stream;
    if (phase == SNN_EPROP_GRAD) {
        snn_status st = check_batch(c, b);
        if (st != SNN_OK) return st;
        SNN_REQUIRE(b->delta && b->Dout && b->psi_rec && b->d_rec,
                    "snn_eprop_update: GRAD needs the psi/d records and the delta/Dout workspace");
        SNN_REQUIRE(!b->trial_T, "snn_eprop_update: GRAD needs every trial to run all T steps (trial_T must be NULL)");
        SNN_REQUIRE(c->d.w_in->d.grad && c->d.w_rec->d.grad, "snn_eprop_update: ragged grad arrays missing");
        return c->d.dtype == SNN_F32 ? grad_impl<float>(c, b, s) : grad_impl<double>(c, b, s);
    }
    if (phase == SNN_EPROP_APPLY) {
        SNN_REQUIRE(adam, "snn_eprop_update: APPLY needs Adam parameters");
        for (snn_ragged* r : {c->d.w_in, c->d.w_rec})
            SNN_REQUIRE(r->d.m && r->d.v && r->d.grad, "snn_eprop_update: ragged m, v, grad required for APPLY");
        SNN_REQUIRE(c->d.W_out_m && c->d.W_out_v && c->d.b_m && c->d.b_v, "snn_eprop_update: readout moments missing");
        SNN_REQUIRE(adam->beta1 >= 0.0 && adam->beta1 < 1.0 && adam->beta2 >= 0.0 && adam->beta2 < 1.0,
                    "snn_eprop_update: beta1, beta2 must be in [0, 1)");
        SNN_REQUIRE(adam->step_dev || adam->step >= 1, "snn_eprop_update: the Adam step count must be >= 1");
        SNN_REQUIRE(adam->temperature >= 0.0 && (adam->temperature == 0.0 || adam->noise_idx >= 0),
                    "snn_eprop_update: temperature must be >= 0 (and noise_idx >= 0 when it is > 0)");
        return c->d.dtype == SNN_F32 ? apply_impl<float>(c, adam, s) : apply_impl<double>(c, adam, s);
    }
    SNN_REQUIRE(false, "snn_eprop_update: unknown phase %d", phase);
}

}  // extern "C"
