// Recurrent LIF/ALIF classifier with e-prop and Adam (Sec. 2.2.1 of the paper).
//
// Forward: one CTA owns one trial and runs every requested step inside one launch.
// Per step it propagates the previous step's input and hidden spikes through the two
// ragged matrices into shared-memory integer accumulators (sums independent of the
// order of the atomic additions; FP64 on the 2^-40 fixed-point grid, FP32 on a grid per
// accumulator set by its incoming |weight| sum), updates the neurons and the leaky
// readout, and records spikes (bits), psi and y; the input spikes of every step are drawn
// from Philox ahead of the step loop (k_input, all steps in parallel); a second kernel
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
#include "classifier_dev.cuh"

#include <cmath>
#include <type_traits>

namespace snn {


__global__ void k_input(InputParams p) { input_group(p, (long long)blockIdx.x * blockDim.x + threadIdx.x); }

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

// The adjoint scan.  CTA = (trial, BWD_THREADS hidden neurons); steps are walked backwards
// in chunks of BWD_TCH.  Each thread prefetches its neuron's psi for the next chunk into
// registers while it runs the current chunk; the chunk's filtered readout error D
// [BWD_TCH][KP] is double-buffered in shared memory (one barrier per chunk).  Per step:
//   lam = sum_k W_out[k][j] D_k,  mu = beta lam' psi' + (rho - beta psi') mu',
//   h = psi (lam - mu),  delta = h' + alpha delta'   (primes: step t+1; zero after T-1).
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

__global__ void __launch_bounds__(256)
    k_sort_rows(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, int P, int C,
                int32_t* __restrict__ keys) {
    extern __shared__ int32_t sk[];                  // [warps][C]
    const int warp = threadIdx.x >> 5;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= P) return;
    sort_row_warp(len, ind, i, C, keys, sk + (size_t)warp * C);
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

__global__ void k_adam_bias(const long long* __restrict__ step_dev, double beta1, double beta2, AdamBias* st,
                            int32_t* status) {
    adam_bias_step(*step_dev, beta1, beta2, st, status);
}


// ------------------------------------------------------------------ host side
// Shared memory of the forward: accumulators (one word each for FP32, a pair for FP64),
// row lengths, two spike lists, their counts, the spike words.
static size_t fwd_smem(int n_in, int N, int Win, int Wh, bool narrow) {
    return (size_t)(N + 64) * (narrow ? 4 : 8) + (size_t)(n_in + N + 1) * 4 + (size_t)(n_in + N) * 4 * 2 + 8 +
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
#define SNN_PACK_SRC                                                                                               \
    (const real*)d.w_in->d.w, d.w_in->d.ind, d.w_in->d.row_len, d.w_in->d.C, d.n_in, (const real*)d.w_rec->d.w, \
        d.w_rec->d.ind, d.w_rec->d.row_len, d.w_rec->d.C, (const real*)d.W_out, d.K, d.N, c->Cf
    if (sizeof(real) == 4) {
        // narrow slots: every accumulator's |weight| sum first, then the slots on its grid
        k_colsum<real><<<ceil_div(n, 256), 256, 0, s>>>(SNN_PACK_SRC, n, c->colsum);
        SNN_LAUNCH_CHECK();
        k_pack_narrow<real><<<ceil_div(n, 256), 256, 0, s>>>(SNN_PACK_SRC, (unsigned long long*)c->pk, n, c->colsum);
    } else {
        k_pack<real><<<ceil_div(n, 256), 256, 0, s>>>(SNN_PACK_SRC, (unsigned long long*)c->pk, n, c->colsum);
    }
#undef SNN_PACK_SRC
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
                            bool packed_ready, cudaStream_t s) {
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
    p.sched = c->row_sched;
    const size_t smem = fwd_smem(d.n_in, d.N, Win, Wh, sizeof(real) == 4);
    snn_status st = packed_ready ? SNN_OK : refresh_fixed<real>(c, s);
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
    // K-splits of the gather: each CTA stages at most GATHER_SPAN (trial, step) spike words
    c->KS = (int)((BT + GATHER_SPAN - 1) / GATHER_SPAN);
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

snn_status snn_classifier_set_row_schedule(snn_classifier* c, int32_t mode) {
    clear_error();
    SNN_REQUIRE(c, "snn_classifier_set_row_schedule: NULL classifier");
    SNN_REQUIRE(mode >= SNN_ROWS_PAIRS && mode <= SNN_ROWS_QUAD, "snn_classifier_set_row_schedule: unknown mode %d",
                mode);
    c->row_sched = mode;
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
    SNN_REQUIRE((flags & ~(SNN_STEP_INPUTS_READY | SNN_STEP_PACKED_READY)) == 0,
                "snn_step_neurons_ex: unknown flags 0x%x", flags);
    if (n_steps == 0) return SNN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool ready = (flags & SNN_STEP_INPUTS_READY) != 0;
    const bool packed = (flags & SNN_STEP_PACKED_READY) != 0;
    return c->d.dtype == SNN_F32 ? step_impl<float>(c, b, t0, n_steps, ready, packed, s)
                                 : step_impl<double>(c, b, t0, n_steps, ready, packed, s);
}

snn_status snn_classifier_pack(snn_classifier* c, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(c, "snn_classifier_pack: NULL classifier");
    cudaStream_t s = (cudaStream_t)stream;
    return c->d.dtype == SNN_F32 ? refresh_fixed<float>(c, s) : refresh_fixed<double>(c, s);
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
