// Recurrent LIF/ALIF classifier with e-prop and Adam (Sec. 2.2.1 of the paper).
//
// Forward: one CTA owns one trial and runs every requested step inside one launch.
// Per step it propagates the previous step's input and hidden spikes through the two
// ragged matrices into shared-memory fixed-point accumulators (sums independent of the
// order of the atomic additions), draws the new input spikes from Philox, updates the
// neurons, the leaky readout and its softmax, and records spikes (bits), psi and d.
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

namespace snn {

constexpr int FWD_THREADS = 256;
constexpr int GATHER_WARPS = 8;

template <typename real>
struct FwdParams {
    int n_in, N, K, Win, Wh, T, t0, n_steps;
    real alpha, rho, beta, v_thr, psi_scale, inv_vthr;
    const uint64_t* in_thr;
    int n_bins, n_classes;
    uint64_t in_seed;
    int32_t* status;
    const int32_t* labels;
    const int32_t* bin_len;
    const int64_t* trial_ids;
    const int32_t* in_len;
    const int32_t* in_ind;
    const real* in_w;
    int in_C;
    const int32_t* rec_len;
    const int32_t* rec_ind;
    const real* rec_w;
    int rec_C;
    const real* W_out;
    const real* b_out;
    real* v;
    real* a;
    real* y;
    real* ysum;
    uint32_t* x_bits;
    uint32_t* z_bits;
    uint32_t* x_rec;
    uint32_t* z_rec;
    real* psi_rec;
    real* d_rec;
    real* v_rec;
    real* a_rec;
    real* y_rec;
};

__device__ __forceinline__ float exp_real(float x) { return expf(x); }
__device__ __forceinline__ double exp_real(double x) { return exp(x); }

template <typename real>
__device__ __forceinline__ void propagate_word(uint32_t word, int row0, const int32_t* __restrict__ len,
                                               const int32_t* __restrict__ ind, const real* __restrict__ w, int C,
                                               unsigned long long* acc) {
    while (word) {
        int i = row0 + __ffs(word) - 1;
        word &= word - 1u;
        int n = len[i];
        const int32_t* ri = ind + (size_t)i * C;
        const real* rw = w + (size_t)i * C;
        int s = lane_id();
        // four independent loads in flight per lane before the atomics
        for (; s + 96 < n; s += 128) {
            int j0 = ri[s], j1 = ri[s + 32], j2 = ri[s + 64], j3 = ri[s + 96];
            real w0 = rw[s], w1 = rw[s + 32], w2 = rw[s + 64], w3 = rw[s + 96];
            atomicAdd(acc + j0, (unsigned long long)to_fixed(w0));
            atomicAdd(acc + j1, (unsigned long long)to_fixed(w1));
            atomicAdd(acc + j2, (unsigned long long)to_fixed(w2));
            atomicAdd(acc + j3, (unsigned long long)to_fixed(w3));
        }
        for (; s < n; s += 32) atomicAdd(acc + ri[s], (unsigned long long)to_fixed(rw[s]));
    }
}

template <typename real>
__global__ void __launch_bounds__(FWD_THREADS) k_forward(FwdParams<real> p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, K = p.K, Win = p.Win, Wh = p.Wh;
    long long* Iacc = (long long*)smem;
    real* vs = (real*)(Iacc + N);
    real* as = vs + N;
    real* yacc = as + N;                        // [32]
    uint32_t* xb = (uint32_t*)(yacc + 32);      // [2][Win]
    uint32_t* zb = xb + 2 * Win;                // [2][Wh]

    const int b = blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, nwarps = nthr >> 5, lane = tid & 31;
    int label = p.labels[b];
    int bin_len = p.bin_len[b];
    if (label < 0 || label >= p.n_classes || bin_len < 1) {
        // invalid per-trial input: report it and simulate a valid stand-in instead of
        // reading outside the threshold table
        if (tid == 0) atomicOr(p.status, ST_STATE);
        label = min(max(label, 0), p.n_classes - 1);
        bin_len = max(bin_len, 1);
    }
    const uint64_t trial = (uint64_t)p.trial_ids[b];
    const int t0 = p.t0;
    {
        const int prv = (t0 - 1) & 1, cur = t0 & 1;
        for (int j = tid; j < N; j += nthr) {
            Iacc[j] = 0;
            vs[j] = p.v[(size_t)b * N + j];
            as[j] = p.a[(size_t)b * N + j];
        }
        for (int w = tid; w < Win; w += nthr) {
            xb[prv * Win + w] = p.x_bits[(size_t)b * Win + w];
            xb[cur * Win + w] = 0u;
        }
        for (int w = tid; w < Wh; w += nthr) {
            zb[prv * Wh + w] = p.z_bits[(size_t)b * Wh + w];
            zb[cur * Wh + w] = 0u;
        }
    }
    real yk = 0, ysk = 0, bk = 0;
    if (warp == 0 && lane < K) {
        yk = p.y[(size_t)b * K + lane];
        ysk = p.ysum[(size_t)b * K + lane];
        bk = p.b_out[lane];
    }
    __syncthreads();
    unsigned long long* acc = (unsigned long long*)Iacc;
    const int n_groups = (p.n_in + 3) >> 2;
    for (int t = t0; t < t0 + p.n_steps; ++t) {
        const int cur = t & 1, prv = cur ^ 1;
        uint32_t* xprv = xb + prv * Win;
        uint32_t* xcur = xb + cur * Win;
        uint32_t* zprv = zb + prv * Wh;
        uint32_t* zcur = zb + cur * Wh;
        // ---------------- phase A: propagate step t-1, readout sum, input of step t
        for (int wi = warp; wi < Win + Wh; wi += nwarps) {
            if (wi < Win)
                propagate_word<real>(xprv[wi], wi * 32, p.in_len, p.in_ind, p.in_w, p.in_C, acc);
            else
                propagate_word<real>(zprv[wi - Win], (wi - Win) * 32, p.rec_len, p.rec_ind, p.rec_w, p.rec_C, acc);
        }
        for (int k = warp; k < K; k += nwarps) {
            real part = 0;
            for (int wi = lane; wi < Wh; wi += 32) {
                uint32_t word = zprv[wi];
                while (word) {
                    int j = wi * 32 + __ffs(word) - 1;
                    word &= word - 1u;
                    part += p.W_out[(size_t)k * N + j];
                }
            }
            part = warp_sum(part);
            if (lane == 0) yacc[k] = part;
        }
        {
            const int bin = min(p.n_bins - 1, t / bin_len);
            const uint64_t* thr = p.in_thr + ((size_t)label * p.n_bins + bin) * p.n_in;
            for (int g = tid; g < n_groups; g += nthr) {
                u64x4 r = philox(p.in_seed, PH_INPUT, trial, (uint64_t)t, (uint64_t)g, 0);
                uint32_t nib = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int c = 4 * g + q;
                    if (c < p.n_in && r[q] < thr[c]) nib |= 1u << q;
                }
                if (nib) atomicOr(&xcur[(4 * g) >> 5], nib << ((4 * g) & 31));
            }
        }
        for (int w = tid; w < Wh; w += nthr) zcur[w] = 0u;
        if (t > t0)
            for (int w = tid; w < Wh; w += nthr) p.z_rec[((size_t)b * p.T + (t - 1)) * Wh + w] = zprv[w];
        __syncthreads();
        // ---------------- phase B: neurons, readout softmax, records
        const size_t rec_off = ((size_t)b * p.T + t) * N;
        for (int j = tid; j < N; j += nthr) {
            real I = from_fixed<real>(Iacc[j]);
            Iacc[j] = 0;
            const bool zp = (zprv[j >> 5] >> (j & 31)) & 1u;
            real v = p.alpha * (zp ? vs[j] - p.v_thr : vs[j]) + I;
            real aa = p.rho * as[j] + (zp ? real(1) : real(0));
            real A = p.v_thr + p.beta * aa;
            bool z = v >= A;
            real u = real(1) - fabs((v - A) * p.inv_vthr);
            real psi = p.psi_scale * (u > real(0) ? u : real(0));
            vs[j] = v;
            as[j] = aa;
            p.psi_rec[rec_off + j] = psi;
            if (p.v_rec) p.v_rec[rec_off + j] = v;
            if (p.a_rec) p.a_rec[rec_off + j] = aa;
            if (z) atomicOr(&zcur[j >> 5], 1u << (j & 31));
        }
        if (warp == 0) {
            real ynew = 0, e = 0;
            if (lane < K) {
                yk = p.alpha * yk + yacc[lane] + bk;
                ynew = yk;
                ysk += yk;
            }
            real mx = warp_max(lane < K ? ynew : -INFINITY);
            if (lane < K) e = exp_real(ynew - mx);
            real ssum = warp_sum(e);
            if (lane < K) {
                real pi = e / ssum;
                p.d_rec[((size_t)b * p.T + t) * K + lane] = pi - (lane == label ? real(1) : real(0));
                if (p.y_rec) p.y_rec[((size_t)b * p.T + t) * K + lane] = ynew;
            }
        }
        for (int w = tid; w < Win; w += nthr) {
            p.x_rec[((size_t)b * p.T + t) * Win + w] = xcur[w];
            xprv[w] = 0u;
        }
        __syncthreads();
    }
    const int last = t0 + p.n_steps - 1;
    const int cl = last & 1;
    for (int w = tid; w < Wh; w += nthr) {
        p.z_rec[((size_t)b * p.T + last) * Wh + w] = zb[cl * Wh + w];
        p.z_bits[(size_t)b * Wh + w] = zb[cl * Wh + w];
    }
    for (int w = tid; w < Win; w += nthr) p.x_bits[(size_t)b * Win + w] = xb[cl * Win + w];
    for (int j = tid; j < N; j += nthr) {
        p.v[(size_t)b * N + j] = vs[j];
        p.a[(size_t)b * N + j] = as[j];
    }
    if (warp == 0 && lane < K) {
        p.y[(size_t)b * K + lane] = yk;
        p.ysum[(size_t)b * K + lane] = ysk;
    }
}

// ------------------------------------------------------------------ backward
// One thread per (trial, readout): D^{T-1} = 0, D^t = d^{t+1} + alpha D^{t+1};
// gb_part[b][k] = sum_t d^t.
template <typename real>
__global__ void k_readout_backward(const real* __restrict__ d, real* __restrict__ D, real* __restrict__ gb_part,
                                   int B, int T, int K, int Kp, real alpha) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * Kp) return;
    int b = idx / Kp, k = idx % Kp;
    real Dk = 0, gsum = 0;
    for (int t = T - 1; t >= 0; --t) {
        real dnext = 0;
        if (k < K) {
            if (t + 1 < T) dnext = d[((size_t)b * T + t + 1) * K + k];
            gsum += d[((size_t)b * T + t) * K + k];
        }
        Dk = (t == T - 1) ? real(0) : dnext + alpha * Dk;
        D[((size_t)b * T + t) * Kp + k] = (k < K) ? Dk : real(0);
    }
    if (k < K) gb_part[(size_t)b * K + k] = gsum;
}

template <typename real>
__global__ void k_reduce_gb(const real* __restrict__ gb_part, real* __restrict__ G_b, int B, int K) {
    int k = threadIdx.x;
    if (k >= K) return;
    real s = 0;
    for (int b = 0; b < B; ++b) s += gb_part[(size_t)b * K + k];
    G_b[k] = s;
}

// One thread per (trial, hidden neuron): the reverse-time adjoint scan.
template <typename real>
__global__ void k_neuron_backward(const real* __restrict__ psi, const real* __restrict__ D,
                                  const real* __restrict__ W_out, real* __restrict__ delta, int B, int T, int N,
                                  int K, int Kp, real alpha, real rho, real beta) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int b = blockIdx.y;
    if (j >= N) return;
    real wc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) wc[k] = (k < K) ? W_out[(size_t)k * N + j] : real(0);
    real lam_next = 0, psi_next = 0, mu = 0, h_next = 0, dl = 0;
    for (int t = T - 1; t >= 0; --t) {
        const size_t o = (size_t)b * T + t;
        real ps = psi[o * N + j];
        const real* Dt = D + o * Kp;
        real lam = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (k < K) lam += wc[k] * Dt[k];
        if (t == T - 1) {
            mu = 0;
            dl = 0;
        } else {
            mu = beta * lam_next * psi_next + (rho - beta * psi_next) * mu;
            dl = h_next + alpha * dl;
        }
        real h = ps * (lam - mu);
        delta[o * N + j] = dl;
        h_next = h;
        lam_next = lam;
        psi_next = ps;
    }
}

// Gather: grid (row blocks, KS).  Warp = one presynaptic row (input rows first, then
// hidden rows); it scans its K-range of (trial, step) for its spike bit, and for every
// spike sums delta at its targets (and, for hidden rows, D into the readout gradient).
template <typename real, int MAXCH>
__global__ void __launch_bounds__(GATHER_WARPS * 32)
    k_gather(const uint32_t* __restrict__ x_rec, const uint32_t* __restrict__ z_rec, int Win, int Wh,
             const int32_t* __restrict__ in_len, const int32_t* __restrict__ in_ind, int in_C, int n_in,
             const int32_t* __restrict__ rec_len, const int32_t* __restrict__ rec_ind, int rec_C, int N,
             const real* __restrict__ delta, const real* __restrict__ D, int K, int Kp, long long BT,
             long long bt_per, real* __restrict__ part_in, real* __restrict__ part_rec,
             real* __restrict__ part_out) {
    const int lane = lane_id();
    const int r = blockIdx.x * GATHER_WARPS + (threadIdx.x >> 5);
    const int ks = blockIdx.y;
    if (r >= n_in + N) return;
    const bool is_in = r < n_in;
    const int i = is_in ? r : r - n_in;
    const uint32_t* bits = is_in ? x_rec : z_rec;
    const int W = is_in ? Win : Wh;
    const int C = is_in ? in_C : rec_C;
    const int len = is_in ? in_len[i] : rec_len[i];
    const int32_t* ri = (is_in ? in_ind : rec_ind) + (size_t)i * C;
    int tgt[MAXCH];
    real acc[MAXCH];
#pragma unroll
    for (int c = 0; c < MAXCH; ++c) {
        int s = c * 32 + lane;
        tgt[c] = (s < len) ? ri[s] : -1;
        acc[c] = 0;
    }
    real acc_o = 0;
    const bool do_out = !is_in && lane < K;
    const int wi = i >> 5;
    const uint32_t bit = 1u << (i & 31);
    const long long bt0 = (long long)ks * bt_per;
    const long long bt1 = min(BT, bt0 + bt_per);
    for (long long base = bt0; base < bt1; base += 32) {
        long long my = base + lane;
        uint32_t word = (my < bt1) ? bits[my * W + wi] : 0u;
        uint32_t spk = __ballot_sync(0xffffffffu, (word & bit) != 0u);
        while (spk) {
            long long e = base + __ffs(spk) - 1;
            spk &= spk - 1u;
            const real* dl = delta + e * N;
#pragma unroll
            for (int c = 0; c < MAXCH; ++c)
                if (tgt[c] >= 0) acc[c] += dl[tgt[c]];
            if (do_out) acc_o += D[e * Kp + lane];
        }
    }
    real* part = is_in ? part_in : part_rec;
    const size_t P = is_in ? (size_t)n_in : (size_t)N;
#pragma unroll
    for (int c = 0; c < MAXCH; ++c) {
        int s = c * 32 + lane;
        if (s < len) part[((size_t)ks * P + i) * C + s] = acc[c];
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

template <typename real>
__global__ void k_adam_ragged(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, int P, int C, int Qw,
                              real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                              const real* __restrict__ grad, const uint32_t* __restrict__ sign, real l1, real lr,
                              real b1, real b2, real omb1, real omb2, real eps, real bc1, real bc2) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * C) return;
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
    w[idx] = ww;
    m[idx] = mm;
    v[idx] = vv;
}

template <typename real>
__global__ void k_adam_dense(real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                             const real* __restrict__ grad, int n, real lr, real b1, real b2, real omb1,
                             real omb2, real eps, real bc1, real bc2) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    real ww = w[idx], mm = m[idx], vv = v[idx];
    adam_update(ww, mm, vv, grad[idx], lr, b1, b2, omb1, omb2, eps, bc1, bc2);
    w[idx] = ww;
    m[idx] = mm;
    v[idx] = vv;
}

// ------------------------------------------------------------------ host side
static size_t fwd_smem(int N, int Win, int Wh, size_t rsz) {
    return (size_t)N * 8 + 2 * (size_t)N * rsz + 32 * rsz + (size_t)(2 * Win + 2 * Wh) * 4;
}

template <typename real>
static snn_status step_impl(snn_classifier* c, const snn_batch* bt, int t0, int n_steps, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    FwdParams<real> p;
    p.n_in = d.n_in;
    p.N = d.N;
    p.K = d.K;
    p.Win = (d.n_in + 31) / 32;
    p.Wh = (d.N + 31) / 32;
    p.T = bt->T;
    p.t0 = t0;
    p.n_steps = n_steps;
    p.alpha = (real)c->alpha;
    p.rho = (real)c->rho;
    p.beta = (real)d.beta;
    p.v_thr = (real)d.v_thr;
    p.psi_scale = (real)(0.3 / d.v_thr);
    p.inv_vthr = (real)(1.0 / d.v_thr);
    p.in_thr = d.in_thr;
    p.n_bins = d.n_bins;
    p.n_classes = d.n_classes;
    p.in_seed = d.in_seed;
    p.status = d.w_in->status;
    p.labels = bt->labels;
    p.bin_len = bt->bin_len;
    p.trial_ids = bt->trial_ids;
    p.in_len = d.w_in->d.row_len;
    p.in_ind = d.w_in->d.ind;
    p.in_w = (const real*)d.w_in->d.w;
    p.in_C = d.w_in->d.C;
    p.rec_len = d.w_rec->d.row_len;
    p.rec_ind = d.w_rec->d.ind;
    p.rec_w = (const real*)d.w_rec->d.w;
    p.rec_C = d.w_rec->d.C;
    p.W_out = (const real*)d.W_out;
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
    size_t smem = fwd_smem(d.N, p.Win, p.Wh, sizeof(real));
    SNN_REQUIRE(smem <= 227 * 1024, "snn_step_neurons: N = %d needs %zu bytes of shared memory (max 227 KB)", d.N,
                smem);
    if (smem > 48 * 1024)
        SNN_CUDA(cudaFuncSetAttribute(k_forward<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_forward<real><<<bt->B, FWD_THREADS, smem, s>>>(p);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

template <typename real>
static snn_status grad_impl(snn_classifier* c, const snn_batch* bt, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const int B = bt->B, T = bt->T, N = d.N, K = d.K, Kp = (K + 3) & ~3;
    const int Win = (d.n_in + 31) / 32, Wh = (N + 31) / 32;
    const real alpha = (real)c->alpha, rho = (real)c->rho, beta = (real)d.beta;
    real* gb_part = (real*)c->part_out + (size_t)c->KS * N * K;
    k_readout_backward<real><<<ceil_div((long long)B * Kp, 128), 128, 0, s>>>(
        (const real*)bt->d_rec, (real*)bt->Dout, gb_part, B, T, K, Kp, alpha);
    SNN_LAUNCH_CHECK();
    k_reduce_gb<real><<<1, 32, 0, s>>>(gb_part, (real*)d.G_b, B, K);
    SNN_LAUNCH_CHECK();
    dim3 gb(ceil_div(N, 128), B);
    k_neuron_backward<real><<<gb, 128, 0, s>>>((const real*)bt->psi_rec, (const real*)bt->Dout,
                                               (const real*)d.W_out, (real*)bt->delta, B, T, N, K, Kp, alpha, rho,
                                               beta);
    SNN_LAUNCH_CHECK();
    const long long BT = (long long)B * T;
    const int KS = c->KS;
    long long bt_per = ((BT + KS - 1) / KS + 31) / 32 * 32;
    dim3 gg(ceil_div(d.n_in + N, GATHER_WARPS), KS);
    const snn_ragged_desc& ri = d.w_in->d;
    const snn_ragged_desc& rr = d.w_rec->d;
    int Cmax = ri.C > rr.C ? ri.C : rr.C;
#define SNN_GATHER(MC)                                                                                        \
    k_gather<real, MC><<<gg, GATHER_WARPS * 32, 0, s>>>(                                                       \
        bt->x_rec, bt->z_rec, Win, Wh, ri.row_len, ri.ind, ri.C, d.n_in, rr.row_len, rr.ind, rr.C, N,          \
        (const real*)bt->delta, (const real*)bt->Dout, K, Kp, BT, bt_per, (real*)c->part_in, (real*)c->part_rec, \
        (real*)c->part_out)
    if (Cmax <= 64) SNN_GATHER(2);
    else if (Cmax <= 128) SNN_GATHER(4);
    else if (Cmax <= 320) SNN_GATHER(10);
    else if (Cmax <= 512) SNN_GATHER(16);
    else SNN_GATHER(64);
#undef SNN_GATHER
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

template <typename real>
static snn_status apply_impl(snn_classifier* c, const snn_adam* ad, cudaStream_t s) {
    const snn_classifier_desc& d = c->d;
    const real lr = (real)ad->lr, b1 = (real)ad->beta1, b2 = (real)ad->beta2, eps = (real)ad->eps;
    const real bc1 = (real)(1.0 - ad->b1t), bc2 = (real)(1.0 - ad->b2t);
    const real omb1 = (real)(1.0 - ad->beta1), omb2 = (real)(1.0 - ad->beta2);
    for (snn_ragged* r : {d.w_in, d.w_rec}) {
        const snn_ragged_desc& rd = r->d;
        const uint32_t* sign = (ad->l1 != 0.0) ? rd.sign_bits : nullptr;
        k_adam_ragged<real><<<ceil_div((long long)rd.P * rd.C, 256), 256, 0, s>>>(
            rd.row_len, rd.ind, rd.P, rd.C, r->Qw, (real*)rd.w, (real*)rd.m, (real*)rd.v, (const real*)rd.grad, sign,
            (real)ad->l1, lr, b1, b2, omb1, omb2, eps, bc1, bc2);
        SNN_LAUNCH_CHECK();
    }
    k_adam_dense<real><<<ceil_div(d.K * d.N, 256), 256, 0, s>>>((real*)d.W_out, (real*)d.W_out_m, (real*)d.W_out_v,
                                                                (const real*)d.G_out, d.K * d.N, lr, b1, b2, omb1,
                                                                omb2, eps, bc1, bc2);
    SNN_LAUNCH_CHECK();
    k_adam_dense<real><<<1, 32, 0, s>>>((real*)d.b_out, (real*)d.b_m, (real*)d.b_v, (const real*)d.G_b, d.K, lr, b1,
                                        b2, omb1, omb2, eps, bc1, bc2);
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
    snn_classifier* c = (snn_classifier*)calloc(1, sizeof(snn_classifier));
    if (!c) {
        set_error("snn_create_classifier: out of host memory");
        return SNN_ENOMEM;
    }
    c->d = *d;
    c->alpha = std::exp(-d->dt / d->tau_m);
    c->rho = d->tau_a > 0 ? std::exp(-d->dt / d->tau_a) : 0.0;
    long long BT = (long long)d->max_B * d->max_T;
    c->KS = BT >= 65536 ? 16 : (BT >= 4096 ? 4 : 1);
    size_t rsz = d->dtype == SNN_F32 ? 4 : 8;
    size_t n_in_part = (size_t)c->KS * d->w_in->d.P * d->w_in->d.C * rsz;
    size_t n_rec_part = (size_t)c->KS * d->w_rec->d.P * d->w_rec->d.C * rsz;
    size_t n_out_part = ((size_t)c->KS * d->N * d->K + (size_t)d->max_B * d->K) * rsz;
    cudaError_t e = cudaMalloc(&c->part_in, n_in_part);
    if (e == cudaSuccess) e = cudaMalloc(&c->part_rec, n_rec_part);
    if (e == cudaSuccess) e = cudaMalloc(&c->part_out, n_out_part);
    if (e != cudaSuccess) {
        snn_destroy_classifier(c);
        set_error("snn_create_classifier: cudaMalloc failed: %s", cudaGetErrorString(e));
        return SNN_ENOMEM;
    }
    *out = c;
    return SNN_OK;
}

snn_status snn_destroy_classifier(snn_classifier* c) {
    if (!c) return SNN_OK;
    cudaFree(c->part_in);
    cudaFree(c->part_rec);
    cudaFree(c->part_out);
    free(c);
    return SNN_OK;
}

static snn_status check_batch(const snn_classifier* c, const snn_batch* b) {
    SNN_REQUIRE(b, "NULL batch");
    SNN_REQUIRE(b->B > 0 && b->T > 0, "batch B and T must be > 0");
    SNN_REQUIRE(b->B <= c->d.max_B && b->T <= c->d.max_T, "batch (B=%d, T=%d) exceeds the classifier's max (%d, %d)",
                b->B, b->T, c->d.max_B, c->d.max_T);
    SNN_REQUIRE(b->labels && b->bin_len && b->trial_ids && b->v && b->a && b->y && b->ysum && b->x_bits &&
                    b->z_bits && b->x_rec && b->z_rec && b->psi_rec && b->d_rec,
                "batch has a NULL required array");
    return SNN_OK;
}

snn_status snn_step_neurons(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_step_neurons: NULL classifier");
    snn_status st = check_batch(c, b);
    if (st != SNN_OK) return st;
    SNN_REQUIRE(t0 >= 0 && n_steps >= 0 && t0 + n_steps <= b->T, "snn_step_neurons: steps [%d, %d) outside [0, %d)",
                t0, t0 + n_steps, b->T);
    if (n_steps == 0) return SNN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    return c->d.dtype == SNN_F32 ? step_impl<float>(c, b, t0, n_steps, s) : step_impl<double>(c, b, t0, n_steps, s);
}

snn_status snn_eprop_update(snn_classifier* c, const snn_batch* b, int32_t phase, const snn_adam* adam,
                            snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_eprop_update: NULL classifier");
    cudaStream_t s = (cudaStream_t)stream;
    if (phase == SNN_EPROP_GRAD) {
        snn_status st = check_batch(c, b);
        if (st != SNN_OK) return st;
        SNN_REQUIRE(b->delta && b->Dout, "snn_eprop_update: batch workspace delta/Dout missing");
        SNN_REQUIRE(c->d.w_in->d.grad && c->d.w_rec->d.grad, "snn_eprop_update: ragged grad arrays missing");
        return c->d.dtype == SNN_F32 ? grad_impl<float>(c, b, s) : grad_impl<double>(c, b, s);
    }
    if (phase == SNN_EPROP_APPLY) {
        SNN_REQUIRE(adam, "snn_eprop_update: APPLY needs Adam parameters");
        for (snn_ragged* r : {c->d.w_in, c->d.w_rec})
            SNN_REQUIRE(r->d.m && r->d.v && r->d.grad, "snn_eprop_update: ragged m, v, grad required for APPLY");
        SNN_REQUIRE(c->d.W_out_m && c->d.W_out_v && c->d.b_m && c->d.b_v, "snn_eprop_update: readout moments missing");
        SNN_REQUIRE(adam->b1t < 1.0 && adam->b2t < 1.0, "snn_eprop_update: b1t, b2t must be beta^t with t >= 1");
        return c->d.dtype == SNN_F32 ? apply_impl<float>(c, adam, s) : apply_impl<double>(c, adam, s);
    }
    SNN_REQUIRE(false, "snn_eprop_update: unknown phase %d", phase);
}

}  // extern "C"
