// Batched form: many independent classifier instances (Sec. 2.2.1 networks of different
// sizes and trial lengths, each with its own ragged matrices and DEEP R state, Sec. 2.1.2)
// trained together in ONE persistent kernel launch per iteration.
//
// An iteration of one instance is the same sequence of operations as its per-call path
// (bookkeeping, snn_step_neurons over the whole trial, snn_eprop_update GRAD and APPLY,
// snn_rewire_deepr on both projections), split into phases whose work is cut into items:
//   PREP    1 item       trial id / label / time warp of the iteration, state reset
//   PRE     n items      input spikes of the trial, |weight| sums of the accumulators
//   PACK    n items      packed forward rows (narrow slots, on each accumulator's grid)
//   FWD     1 + n items  the whole trial (forward_trial), and beside it the gather order
//                        of every row (needed only by GATHER)
//   SCAN    1 item       softmax of the readout, filtered readout error, bias gradient,
//                        Adam's running products
//   BWD     N/1024 items the adjoint scan, 1024 hidden neurons per item (two per thread)
//   GATHER  Win+Wh items e-prop gradients of one spike-bit word (32 presynaptic rows)
//   ADAM    n items      L1 + Adam (+ DEEP R noise) on 8192 elements per item
//   ELIM    n items      DEEP R elimination, 32 rows per item
//   DIST    2 items      DEEP R redistribution of each projection (one CTA)
//   FORM    n items      DEEP R formation, 32 rows per item
// Items sit in a device work queue (slots plus per-slot publication stamps).  Every CTA
// loops: take the next slot index, wait (bounded) until that slot is published, run the
// item, and if it was the last item of its instance's phase, publish the next phase's
// items.  A phase starts only when the previous one is complete, so items never wait on
// each other; the only waits are those for queue slots, and each gives up after the
// run's time limit (status SNN_ETIMEOUT, every CTA leaves).  All instances' phases
// interleave freely, so short instances' gradient and rewiring work fills the SMs while
// long instances simulate.  The items run the same device functions as the per-call
// kernels (classifier_dev.cuh, deepr_dev.cuh), so results are bit-identical to them.
//
// The first phase is seeded by the kernel itself, or, with SNN_MULTI_HOST_POSTS, from a
// mailbox in mapped host memory that a host producer fills after the launch
// (snn_multi_post): the kernel waits for it with the same bounded wait.
#include "classifier_dev.cuh"
#include "deepr_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace snn {

enum : int {
    MP_PREP = 0, MP_PRE = 1, MP_PACK = 2, MP_FWD = 3, MP_SCAN = 4, MP_BWD = 5, MP_GATHER = 6, MP_ADAM = 7,
    MP_ELIM = 8, MP_DIST = 9, MP_FORM = 10, MP_N = 11,
};

constexpr int MT = 512;                          // threads per CTA (one CTA per SM: a trial's forward
                                                 // gets 16 warps; 256 threads: 1.18x longer iterations)
constexpr int MW = MT / 32;                      // warps per CTA
constexpr int M_INPUT_PER_ITEM = 8 * MT;         // input groups (8 channels each) per item
constexpr int M_PACK_PER_ITEM = 32 * MT;         // packed slots per item
constexpr int M_ROWS_PER_ITEM = 32;              // rows per sort / elimination / formation item
constexpr int M_ADAM_PER_ITEM = 16 * MT;         // optimiser elements per item
constexpr int M_BWD_PER_ITEM = 2 * MT;           // hidden neurons per adjoint item

struct MRag {
    int32_t* len;
    int32_t* ind;
    float* w;
    float* m;
    float* v;
    float* grad;
    uint32_t* sign;
    uint32_t* conn;
    uint32_t* tag;
    int32_t* dormant;
    int32_t* taken;
    int32_t* room;
    int32_t* cnt;
    unsigned long long* dsum;                    // [2]
    int32_t* status;
    snn_rewire_stats* stats;
    int32_t* keys;                               // gather order
    uint64_t seed;
    int P, Q, C, Qw, no_autapse;
};

struct MInst {
    int n_in, N, K, Kp, Win, Wh, T, Cf, n_classes, n_bins, sched, Cmax;
    float alpha, rho, beta, v_thr, psi_scale, inv_vthr;
    const uint32_t* in_thr;
    uint64_t in_seed;
    unsigned long long* pk;
    unsigned long long* colsum;
    AdamBias* adam_state;
    float *W_out, *b_out, *W_out_m, *W_out_v, *b_m, *b_v, *G_out, *G_b;
    int32_t* labels;
    int32_t* bin_len;
    int64_t* trial_ids;
    float *v, *a, *y, *ysum;
    uint32_t *x_bits, *z_bits, *x_rec, *z_rec;
    float *psi, *d, *delta, *Dout;
    long long* iter;
    const int32_t* label_table;
    const int32_t* bin_table;
    int n_label, n_bin;
    double lr, beta1, beta2, eps, l1, temperature;
    MRag rg[2];
    int n_items[MP_N];
    int n_input, n_pack, n_sort0;                // MP_PRE: input, sums; MP_PACK; MP_FWD: sort items of input rows first
    int n_rows0;                                 // MP_ELIM / MP_FORM: items of the input projection
    int orig;                                    // the instance's index in the caller's array
};

// Queue header.  gen = completed runs; run r uses stamp r + 1 for its published slots.
struct MQueue {
    unsigned int head, tail, exit_count, gen;
    unsigned int total, total_stamp, abort_stamp, pad;
    int32_t status;
    int32_t pad2[7];
};

__device__ __forceinline__ unsigned long long m_item(int inst, int phase, int idx) {
    return ((unsigned long long)inst << 40) | ((unsigned long long)phase << 32) | (unsigned)idx;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys_i32(const volatile int* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct MArgs {
    const MInst* inst;
    int n_inst;
    int* remaining;                   // [n_inst] items left in the instance's current phase
    MQueue* q;
    unsigned long long* slots;        // [cap]
    unsigned* ready;                  // [cap] publication stamps
    unsigned cap;
    const int* mailbox;               // mapped host memory: {stamp, n, instance ids...} or NULL
    long long limit_ns;
    long long* trace;                 // [n_inst][MP_N + 1] global-timer stamps, or NULL
};

// Publishes all items of `phase` of instance i (the whole CTA calls it).
__device__ void m_push(const MArgs& A, int i, int phase, unsigned stamp, unsigned* s_base) {
    const int n = A.inst[i].n_items[phase];
    if (threadIdx.x == 0) {
        atomicExch(&A.remaining[i], n);
        __threadfence();
        *s_base = atomicAdd(&A.q->tail, (unsigned)n);
    }
    __syncthreads();
    const unsigned base = *s_base;
    for (int k = threadIdx.x; k < n; k += MT) {
        if (base + k < A.cap) {
            A.slots[base + k] = m_item(i, phase, k);
            __threadfence();
            st_release_u32(&A.ready[base + k], stamp);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- the phases' items
__device__ void m_prep(const MInst& I) {
    const long long it = *I.iter;
    const int tid = threadIdx.x;
    if (tid == 0) {
        I.trial_ids[0] = it;
        I.labels[0] = I.label_table[(int)(it % I.n_label)];
        I.bin_len[0] = I.bin_table[(int)(it % I.n_bin)];
    }
    for (int j = tid; j < I.N; j += MT) {
        I.v[j] = 0.f;
        I.a[j] = 0.f;
    }
    for (int k = tid; k < I.K; k += MT) {
        I.y[k] = 0.f;
        I.ysum[k] = 0.f;
    }
    for (int w = tid; w < I.Win; w += MT) I.x_bits[w] = 0u;
    for (int w = tid; w < I.Wh; w += MT) I.z_bits[w] = 0u;
    for (int j = tid; j < I.N + 64; j += MT) I.colsum[j] = 0ull;
    if (tid < 2) {
        I.rg[tid].dsum[0] = 0ull;
        I.rg[tid].dsum[1] = 0ull;
    }
}

__device__ void m_pre(const MInst& I, int k, unsigned char* smem) {
    const int tid = threadIdx.x;
    if (k < I.n_input) {
        InputParams p;
        p.n_in = I.n_in;
        p.Win = I.Win;
        p.T = I.T;
        p.t0 = 0;
        p.n_steps = I.T;
        p.n_bins = I.n_bins;
        p.n_classes = I.n_classes;
        p.B = 1;
        p.trial_T = nullptr;
        p.in_thr = I.in_thr;
        p.seed = I.in_seed;
        p.labels = I.labels;
        p.bin_len = I.bin_len;
        p.trial_ids = I.trial_ids;
        p.x_rec = I.x_rec;
        p.status = I.rg[0].status;
        const long long g0 = (long long)k * M_INPUT_PER_ITEM;
        for (int r = 0; r < M_INPUT_PER_ITEM / MT; ++r) input_group(p, g0 + (long long)r * MT + tid);
        return;
    }
    k -= I.n_input;
    if (k < I.n_pack) {
        const long long n = (long long)(I.n_in + I.N) * I.Cf;
        const MRag &ri = I.rg[0], &rr = I.rg[1];
        for (int r = 0; r < M_PACK_PER_ITEM / MT; ++r) {
            const long long s = (long long)k * M_PACK_PER_ITEM + (long long)r * MT + tid;
            if (s < n)
                colsum_slot<float>(ri.w, ri.ind, ri.len, ri.C, I.n_in, rr.w, rr.ind, rr.len, rr.C, I.W_out, I.K, I.N,
                                   I.Cf, I.colsum, s);
        }
        return;
    }
}

// Packed forward rows, slots [k M_PACK_PER_ITEM, (k + 1) M_PACK_PER_ITEM), from the
// complete |weight| sums of the PRE phase.
__device__ void m_pack(const MInst& I, int k) {
    const long long n = (long long)(I.n_in + I.N) * I.Cf;
    const MRag &ri = I.rg[0], &rr = I.rg[1];
    for (int r = 0; r < M_PACK_PER_ITEM / MT; ++r) {
        const long long s = (long long)k * M_PACK_PER_ITEM + (long long)r * MT + threadIdx.x;
        if (s < n)
            pack_slot_narrow<float>(ri.w, ri.ind, ri.len, ri.C, I.n_in, rr.w, rr.ind, rr.len, rr.C, I.W_out, I.K,
                                    I.N, I.Cf, I.pk, I.colsum, s);
    }
}

// Gather order of 32 rows (item k of the FWD phase's sort items).
__device__ void m_sort(const MInst& I, int k, unsigned char* smem) {
    const int tid = threadIdx.x;
    const int proj = k < I.n_sort0 ? 0 : 1;
    const int kk = proj == 0 ? k : k - I.n_sort0;
    const MRag& r = I.rg[proj];
    const int warp = tid >> 5;
    int32_t* row = (int32_t*)smem + (size_t)warp * r.C;
    for (int u = warp; u < M_ROWS_PER_ITEM; u += MW) {
        const int i = kk * M_ROWS_PER_ITEM + u;
        if (i < r.P) sort_row_warp(r.len, r.ind, i, r.C, r.keys, row);
        __syncwarp();
    }
}

template <int NPT>
__device__ void m_fwd_npt(const FwdParams<float>& p, unsigned char* smem) {
    forward_trial<float, NPT, MT, true>(p, 0, smem);
}

__device__ void m_fwd(const MInst& I, unsigned char* smem) {
    FwdParams<float> p;
    p.n_in = I.n_in;
    p.N = I.N;
    p.K = I.K;
    p.Win = I.Win;
    p.Wh = I.Wh;
    p.T = I.T;
    p.t0 = 0;
    p.n_steps = I.T;
    p.alpha = I.alpha;
    p.rho = I.rho;
    p.beta = I.beta;
    p.v_thr = I.v_thr;
    p.psi_scale = I.psi_scale;
    p.inv_vthr = I.inv_vthr;
    p.in_len = I.rg[0].len;
    p.rec_len = I.rg[1].len;
    p.pk = I.pk;
    p.Cf = I.Cf;
    p.b_out = I.b_out;
    p.v = I.v;
    p.a = I.a;
    p.y = I.y;
    p.ysum = I.ysum;
    p.x_bits = I.x_bits;
    p.z_bits = I.z_bits;
    p.x_rec = I.x_rec;
    p.z_rec = I.z_rec;
    p.psi_rec = I.psi;
    p.d_rec = I.d;
    p.v_rec = p.a_rec = p.y_rec = nullptr;
    p.record_state = 0;
    p.trial_T = nullptr;
    p.colsum = I.colsum;
    p.status = I.rg[0].status;
    p.sched = I.sched;
    const int npt = (I.N + MT - 1) / MT;
    if (npt <= 1) m_fwd_npt<1>(p, smem);
    else if (npt <= 2) m_fwd_npt<2>(p, smem);
    else if (npt <= 4) m_fwd_npt<4>(p, smem);
    else m_fwd_npt<8>(p, smem);
}

__device__ void m_scan(const MInst& I, unsigned char* smem) {
    const int warp = threadIdx.x >> 5;
    float* sh = (float*)smem + (size_t)warp * 32 * I.K;
    const int n_span = (I.T + 31) / 32;
    for (int s = warp; s < n_span; s += MW) {
        const int ts = s * 32;
        softmax_span<float>(I.d, I.labels, I.n_classes, nullptr, 0, I.T, I.K, ts, min(32, I.T - ts), sh);
    }
    __syncthreads();
    // one trial: the bias gradient is the scan's per-trial sum itself
    if (warp == 0) readout_scan_warp<float>(I.d, I.Dout, I.G_b, 0, I.T, I.K, I.Kp, I.alpha);
    if (threadIdx.x == 32) adam_bias_step(*I.iter + 1, I.beta1, I.beta2, I.adam_state, I.rg[0].status);
}

template <int KV>
__device__ void m_bwd_kv(const MInst& I, int k, unsigned char* smem) {
    backward_x2_block<KV, MT>(I.psi, I.Dout, I.W_out, I.delta, I.T, I.N, I.K, I.alpha, I.rho, I.beta, k, 0,
                              (float*)smem);
}

__device__ void m_bwd(const MInst& I, int k, unsigned char* smem) {
    switch (I.Kp / 4) {
        case 1: m_bwd_kv<1>(I, k, smem); break;
        case 2: m_bwd_kv<2>(I, k, smem); break;
        case 3: m_bwd_kv<3>(I, k, smem); break;
        case 4: m_bwd_kv<4>(I, k, smem); break;
        case 5: m_bwd_kv<5>(I, k, smem); break;
        case 6: m_bwd_kv<6>(I, k, smem); break;
        case 7: m_bwd_kv<7>(I, k, smem); break;
        default: m_bwd_kv<8>(I, k, smem); break;
    }
}

// One spike-bit word (input words first, then hidden words): its 32 rows in groups of
// MW warps, each over all 128-slot groups; one K-split (B = 1, T <= GATHER_SPAN), gradients
// written in place.
__device__ void m_gather(const MInst& I, int col, unsigned char* smem) {
    const MRag &ri = I.rg[0], &rr = I.rg[1];
    const long long BT = I.T;
    const long long bt_per = (BT + 31) / 32 * 32;
    const int n_groups = (I.Cmax + 127) / 128;
    constexpr int SPLIT = 32 / MW;
    for (int part = 0; part < SPLIT; ++part)
        for (int g = 0; g < n_groups; ++g) {
            gather_block<float, MW, GATHER_EV, true>(I.x_rec, I.z_rec, I.Win, I.Wh, ri.len, ri.keys, ri.C, I.n_in,
                                                     rr.len, rr.keys, rr.C, I.N, I.delta, I.Dout, I.K, I.Kp, BT,
                                                     bt_per, ri.grad, rr.grad, I.G_out, col * SPLIT + part, 0, g,
                                                     (uint32_t*)smem);
            __syncthreads();
        }
}

__device__ void m_adam(const MInst& I, int k) {
    const long long n0 = (long long)I.rg[0].P * I.rg[0].C, n1 = (long long)I.rg[1].P * I.rg[1].C;
    const long long n2 = (long long)I.K * I.N, n3 = I.K;
    const float lr = (float)I.lr, b1 = (float)I.beta1, b2 = (float)I.beta2, eps = (float)I.eps;
    const float omb1 = (float)(1.0 - I.beta1), omb2 = (float)(1.0 - I.beta2);
    const double* bias = (const double*)I.adam_state;
    for (int r = 0; r < M_ADAM_PER_ITEM / MT; ++r) {
        long long e = (long long)k * M_ADAM_PER_ITEM + (long long)r * MT + threadIdx.x;
        if (e < n0 + n1) {
            const int pj = e < n0 ? 0 : 1;
            if (pj) e -= n0;
            const MRag& rg = I.rg[pj];
            NoiseK nz;
            nz.amp = I.temperature > 0.0 ? sqrt(2.0 * I.lr * I.temperature) : 0.0;
            nz.seed = rg.seed;
            nz.idx = 0;
            nz.idx_dev = (const int64_t*)I.iter;
            const uint32_t* sign = I.l1 != 0.0 ? rg.sign : nullptr;
            const int i = (int)(e / rg.C), s = (int)(e % rg.C);
            if (s < rg.len[i])
                adam_ragged_elem<float>(rg.len, rg.ind, rg.C, rg.Qw, rg.w, rg.m, rg.v, rg.grad, sign, (float)I.l1, lr,
                                        b1, b2, omb1, omb2, eps, 1.f, 1.f, bias, nz, e);
        } else if (e < n0 + n1 + n2) {
            adam_dense_elem<float>(I.W_out, I.W_out_m, I.W_out_v, I.G_out, lr, b1, b2, omb1, omb2, eps, 1.f, 1.f, bias,
                                   (int)(e - n0 - n1));
        } else if (e < n0 + n1 + n2 + n3) {
            adam_dense_elem<float>(I.b_out, I.b_m, I.b_v, I.G_b, lr, b1, b2, omb1, omb2, eps, 1.f, 1.f, bias,
                                   (int)(e - n0 - n1 - n2));
        }
    }
}

__device__ void m_elim(const MInst& I, int k, long long* red) {
    const int proj = k < I.n_rows0 ? 0 : 1;
    const int kk = proj == 0 ? k : k - I.n_rows0;
    const MRag& r = I.rg[proj];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    long long removed = 0;
    for (int u = warp; u < M_ROWS_PER_ITEM; u += MW) {
        const int i = kk * M_ROWS_PER_ITEM + u;
        if (i < r.P) {
            eliminate_row<float>(r.len, r.ind, r.w, r.m, r.v, r.sign, r.conn, r.tag, r.dormant, r.cnt, i, r.C, r.Qw);
            if (lane == 0) removed += r.dormant[i];
        }
    }
    const long long t = block_sum_ll(lane == 0 ? removed : 0, red);
    if (threadIdx.x == 0 && t) atomicAdd(r.dsum, (unsigned long long)t);
}

__device__ void m_dist(const MInst& I, int proj, long long* red) {
    const MRag& r = I.rg[proj];
    const long long D = (long long)*(volatile unsigned long long*)r.dsum;
    redistribute_block(r.len, r.cnt, r.room, r.taken, D, r.P, r.C, r.Q, r.no_autapse, r.seed,
                       (uint64_t)*I.iter, r.status, r.stats, red);
}

__device__ void m_form(const MInst& I, int k, unsigned char* smem) {
    const int proj = k < I.n_rows0 ? 0 : 1;
    const int kk = proj == 0 ? k : k - I.n_rows0;
    const MRag& r = I.rg[proj];
    const int warp = threadIdx.x >> 5;
    const int NC = (r.Qw + 31) >> 5;
    int32_t* F = (int32_t*)smem + (size_t)warp * (NC + 1);
    for (int u = warp; u < M_ROWS_PER_ITEM; u += MW) {
        const int i = kk * M_ROWS_PER_ITEM + u;
        if (i < r.P)
            form_row_warp<float>(r.len, r.ind, r.w, r.m, r.v, r.conn, r.taken, i, r.C, r.Q, r.Qw, r.no_autapse,
                                 r.seed, (uint64_t)*I.iter, r.status, r.stats, F);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- the persistent kernel
__global__ void __launch_bounds__(MT, 1) k_multi(MArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_item;
    __shared__ int s_flag;
    __shared__ unsigned s_base;
    __shared__ long long red[32];
    const int tid = threadIdx.x;
    __shared__ unsigned s_stamp;
    if (tid == 0) s_stamp = *(volatile unsigned*)&A.q->gen + 1u;
    __syncthreads();
    const unsigned stamp = s_stamp;
    // ---- seeding (CTA 0): the first phase of every instance, or of the posted ones
    if (blockIdx.x == 0) {
        if (tid == 0) {
            s_flag = 1;
            if (A.mailbox) {
                const unsigned long long t0 = global_ns();
                while ((unsigned)ld_acquire_sys_i32(A.mailbox) != stamp) {
                    if ((long long)(global_ns() - t0) > A.limit_ns) {
                        atomicOr(&A.q->status, ST_TIMEOUT);
                        st_release_u32(&A.q->abort_stamp, stamp);
                        s_flag = 0;
                        break;
                    }
                    __nanosleep(1000);
                }
            }
            unsigned total = 0;
            if (s_flag) {
                const int n = A.mailbox ? ld_acquire_sys_i32(A.mailbox + 1) : A.n_inst;
                for (int k = 0; k < n; ++k) {
                    const int i = A.mailbox ? A.mailbox[2 + k] : k;
                    if (i < 0 || i >= A.n_inst) {
                        atomicOr(&A.q->status, ST_STATE);
                        continue;
                    }
                    for (int ph = 0; ph < MP_N; ++ph) total += (unsigned)A.inst[i].n_items[ph];
                }
                if (total > A.cap) {                       // a posted instance twice: refuse the run
                    atomicOr(&A.q->status, ST_STATE);
                    total = 0;
                }
            }
            A.q->total = total;
            __threadfence();
            st_release_u32(&A.q->total_stamp, stamp);
            s_item = total > 0 ? (unsigned long long)(A.mailbox ? ld_acquire_sys_i32(A.mailbox + 1) : A.n_inst) : 0ull;
        }
        __syncthreads();
        const int n_seed = (int)s_item;                // same value in every thread
        __syncthreads();
        for (int k = 0; k < n_seed; ++k) {
            // thread 0 reads the posted instance and shares it, so all threads agree
            if (tid == 0) s_flag = A.mailbox ? A.mailbox[2 + k] : k;
            __syncthreads();
            const int i = s_flag;
            __syncthreads();
            if (i >= 0 && i < A.n_inst) {
                if (A.trace && tid == 0) A.trace[(size_t)A.inst[i].orig * (MP_N + 1)] = (long long)global_ns();
                m_push(A, i, MP_PREP, stamp, &s_base);
            }
        }
        __syncthreads();
    }
    // ---- the work loop
    for (;;) {
        if (tid == 0) {
            const unsigned h = atomicAdd(&A.q->head, 1u);
            const unsigned long long t0 = global_ns();
            int flag = 0;
            for (;;) {
                if (ld_acquire_u32(&A.q->total_stamp) == stamp && h >= *(volatile unsigned*)&A.q->total) break;
                if (h < A.cap && ld_acquire_u32(&A.ready[h]) == stamp) {
                    s_item = *(volatile unsigned long long*)&A.slots[h];
                    flag = 1;
                    break;
                }
                if (ld_acquire_u32(&A.q->abort_stamp) == stamp) break;
                if ((long long)(global_ns() - t0) > A.limit_ns) {
                    atomicOr(&A.q->status, ST_TIMEOUT);
                    st_release_u32(&A.q->abort_stamp, stamp);
                    break;
                }
                __nanosleep(200);
            }
            __threadfence();
            s_flag = flag;
        }
        __syncthreads();
        if (!s_flag) break;
        const unsigned long long item = s_item;
        const int i = (int)(item >> 40);
        const int phase = (int)((item >> 32) & 0xff);
        const int k = (int)(item & 0xffffffffu);
        const MInst& I = A.inst[i];
        switch (phase) {
            case MP_PREP: m_prep(I); break;
            case MP_PRE: m_pre(I, k, smem); break;
            case MP_PACK: m_pack(I, k); break;
            case MP_FWD:
                if (k == 0) m_fwd(I, smem);
                else m_sort(I, k - 1, smem);
                break;
            case MP_SCAN: m_scan(I, smem); break;
            case MP_BWD: m_bwd(I, k, smem); break;
            case MP_GATHER: m_gather(I, k, smem); break;
            case MP_ADAM: m_adam(I, k); break;
            case MP_ELIM: m_elim(I, k, red); break;
            case MP_DIST: m_dist(I, k, red); break;
            default: m_form(I, k, smem); break;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_flag = atomicSub(&A.remaining[i], 1) == 1;
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            if (A.trace && tid == 0) A.trace[(size_t)I.orig * (MP_N + 1) + 1 + phase] = (long long)global_ns();
            if (phase + 1 < MP_N) {
                m_push(A, i, phase + 1, stamp, &s_base);
            } else if (tid == 0) {
                *I.iter += 1;                          // the instance's iteration is complete
                __threadfence();
            }
        }
        __syncthreads();
    }
    // ---- the last CTA out resets the queue for the next run
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&A.q->exit_count, 1u) == gridDim.x - 1) {
            A.q->head = 0;
            A.q->tail = 0;
            A.q->exit_count = 0;
            __threadfence();
            atomicAdd(&A.q->gen, 1u);
        }
    }
}

}  // namespace snn

using namespace snn;

struct snn_multi {
    int n;
    MInst* d_inst;
    int* d_remaining;
    MQueue* d_q;
    unsigned long long* d_slots;
    unsigned* d_ready;
    unsigned cap;
    int* h_mailbox;               // mapped pinned host memory
    int* d_mailbox;
    unsigned runs;                // snn_multi_run calls so far (= the device's completed runs)
    long long* trace;             // caller's device buffer of phase completion times, or NULL
    size_t smem;
    int grid;
    std::vector<int> order;       // seeding order (longest instances first)
};

static snn_status multi_fill(const snn_multi_instance& s, MInst& I, size_t& smem) {
    SNN_REQUIRE(s.cls, "snn_multi_create: NULL classifier");
    const snn_classifier* c = s.cls;
    const snn_classifier_desc& d = c->d;
    const snn_batch& b = s.batch;
    SNN_REQUIRE(d.dtype == SNN_F32, "snn_multi_create: FP32 classifiers only");
    SNN_REQUIRE(d.N % 2 == 0, "snn_multi_create: N must be even");
    SNN_REQUIRE(b.B == 1 && b.T > 0 && b.T <= d.max_T && b.T <= GATHER_SPAN,
                "snn_multi_create: each instance trains one trial (B = 1) of 1 <= T <= min(max_T, %d) steps", GATHER_SPAN);
    SNN_REQUIRE(b.labels && b.bin_len && b.trial_ids && b.v && b.a && b.y && b.ysum && b.x_bits && b.z_bits &&
                    b.x_rec && b.z_rec && b.psi_rec && b.d_rec && b.delta && b.Dout && !b.trial_T,
                "snn_multi_create: the batch needs state, records and workspace (and no trial_T)");
    SNN_REQUIRE(s.label_table && s.n_label > 0 && s.bin_table && s.n_bin > 0 && s.iter,
                "snn_multi_create: label / bin tables and the iteration counter are required");
    SNN_REQUIRE(s.beta1 >= 0 && s.beta1 < 1 && s.beta2 >= 0 && s.beta2 < 1 && s.temperature >= 0,
                "snn_multi_create: bad optimiser parameters");
    SNN_REQUIRE(d.W_out_m && d.W_out_v && d.b_m && d.b_v, "snn_multi_create: readout Adam moments required");
    const snn_ragged* rg[2] = {d.w_in, d.w_rec};
    for (int p = 0; p < 2; ++p) {
        const snn_ragged_desc& r = rg[p]->d;
        SNN_REQUIRE(r.m && r.v && r.grad && r.sign_bits && r.conn_bits && rg[p]->stag,
                    "snn_multi_create: ragged handles need m, v, grad and DEEP R bitfields");
        SNN_REQUIRE(!rg[p]->guide_on, "snn_multi_create: distance-guided formation is not supported here");
        SNN_REQUIRE((size_t)(MT / 32) * ((rg[p]->Qw + 31) / 32 + 1) * 4 <= 48 * 1024,
                    "snn_multi_create: Q too large for the formation chunk table");
        MRag& m = I.rg[p];
        m.len = r.row_len;
        m.ind = r.ind;
        m.w = (float*)r.w;
        m.m = (float*)r.m;
        m.v = (float*)r.v;
        m.grad = (float*)r.grad;
        m.sign = r.sign_bits;
        m.conn = r.conn_bits;
        m.tag = rg[p]->stag;
        m.dormant = rg[p]->dormant;
        m.taken = rg[p]->taken;
        m.room = rg[p]->room;
        m.cnt = rg[p]->cnt;
        m.dsum = (unsigned long long*)rg[p]->scal;
        m.status = rg[p]->status;
        m.stats = s.stats ? s.stats + p : nullptr;
        m.seed = r.seed;
        m.P = r.P;
        m.Q = r.Q;
        m.C = r.C;
        m.Qw = rg[p]->Qw;
        m.no_autapse = r.no_autapse;
    }
    I.rg[0].keys = c->gkeys;
    I.rg[1].keys = c->gkeys + (size_t)d.w_in->d.P * d.w_in->d.C;
    I.n_in = d.n_in;
    I.N = d.N;
    I.K = d.K;
    I.Kp = (d.K + 3) & ~3;
    I.Win = (d.n_in + 31) / 32;
    I.Wh = (d.N + 31) / 32;
    I.T = b.T;
    I.Cf = c->Cf;
    I.Cmax = std::max(d.w_in->d.C, d.w_rec->d.C);
    I.n_classes = d.n_classes;
    I.n_bins = d.n_bins;
    I.sched = c->row_sched;
    I.alpha = (float)c->alpha;
    I.rho = (float)c->rho;
    I.beta = (float)d.beta;
    I.v_thr = (float)d.v_thr;
    I.psi_scale = (float)(0.3 / d.v_thr);
    I.inv_vthr = (float)(1.0 / d.v_thr);
    I.in_thr = d.in_thr;
    I.in_seed = d.in_seed;
    I.pk = (unsigned long long*)c->pk;
    I.colsum = c->colsum;
    I.adam_state = (AdamBias*)c->adam_dev;
    I.W_out = (float*)d.W_out;
    I.b_out = (float*)d.b_out;
    I.W_out_m = (float*)d.W_out_m;
    I.W_out_v = (float*)d.W_out_v;
    I.b_m = (float*)d.b_m;
    I.b_v = (float*)d.b_v;
    I.G_out = (float*)d.G_out;
    I.G_b = (float*)d.G_b;
    I.labels = (int32_t*)b.labels;
    I.bin_len = (int32_t*)b.bin_len;
    I.trial_ids = (int64_t*)b.trial_ids;
    I.v = (float*)b.v;
    I.a = (float*)b.a;
    I.y = (float*)b.y;
    I.ysum = (float*)b.ysum;
    I.x_bits = b.x_bits;
    I.z_bits = b.z_bits;
    I.x_rec = b.x_rec;
    I.z_rec = b.z_rec;
    I.psi = (float*)b.psi_rec;
    I.d = (float*)b.d_rec;
    I.delta = (float*)b.delta;
    I.Dout = (float*)b.Dout;
    I.iter = (long long*)s.iter;
    I.label_table = s.label_table;
    I.bin_table = s.bin_table;
    I.n_label = s.n_label;
    I.n_bin = s.n_bin;
    I.lr = s.lr;
    I.beta1 = s.beta1;
    I.beta2 = s.beta2;
    I.eps = s.eps;
    I.l1 = s.l1;
    I.temperature = s.temperature;
    // items per phase
    const int rows0 = ceil_div(d.n_in, M_ROWS_PER_ITEM), rows1 = ceil_div(d.N, M_ROWS_PER_ITEM);
    I.n_input = ceil_div((long long)b.T * I.Win * 4, M_INPUT_PER_ITEM);
    I.n_pack = ceil_div((long long)(d.n_in + d.N) * c->Cf, M_PACK_PER_ITEM);
    I.n_sort0 = rows0;
    I.n_rows0 = rows0;
    I.n_items[MP_PREP] = 1;
    I.n_items[MP_PRE] = I.n_input + I.n_pack;
    I.n_items[MP_PACK] = I.n_pack;
    I.n_items[MP_FWD] = 1 + rows0 + rows1;
    I.n_items[MP_SCAN] = 1;
    I.n_items[MP_BWD] = ceil_div(d.N, M_BWD_PER_ITEM);
    I.n_items[MP_GATHER] = I.Win + I.Wh;
    I.n_items[MP_ADAM] = ceil_div((long long)d.w_in->d.P * d.w_in->d.C + (long long)d.w_rec->d.P * d.w_rec->d.C +
                                      (long long)d.K * d.N + d.K,
                                  M_ADAM_PER_ITEM);
    I.n_items[MP_ELIM] = rows0 + rows1;
    I.n_items[MP_DIST] = 2;
    I.n_items[MP_FORM] = rows0 + rows1;
    // shared memory of the largest phase
    const size_t fwd = (size_t)(d.N + 64) * 4 + (size_t)(d.n_in + d.N + 1) * 4 + (size_t)(d.n_in + d.N) * 4 * 2 + 8 +
                       (size_t)(I.Win + 2 * I.Wh) * 4;   // narrow accumulators: one word each
    const size_t sort = (size_t)MW * I.Cmax * 4;
    const size_t gat = (size_t)((b.T + 31) / 32 * 32) * 4;
    const size_t scan = (size_t)MW * 32 * d.K * 4;
    const size_t form = (size_t)MW * ((std::max(rg[0]->Qw, rg[1]->Qw) + 31) / 32 + 1) * 4;
    const size_t bwd = (size_t)2 * BWD2_TCH * I.Kp * 4;
    smem = std::max({smem, fwd, sort, gat, scan, form, bwd});
    return SNN_OK;
}

extern "C" {

snn_status snn_multi_create(const snn_multi_instance* inst, int32_t n, snn_multi** out) {
    clear_error();
    SNN_REQUIRE(inst && out && n > 0 && n < 65536, "snn_multi_create: need 1 <= n < 65536 instances");
    *out = nullptr;
    std::vector<MInst> h(n);
    size_t smem = 0;
    unsigned long long cap = 0;
    for (int i = 0; i < n; ++i) {
        std::memset(&h[i], 0, sizeof(MInst));
        const snn_status st = multi_fill(inst[i], h[i], smem);
        if (st != SNN_OK) return st;
        for (int ph = 0; ph < MP_N; ++ph) cap += (unsigned long long)h[i].n_items[ph];
        for (int j = 0; j < i; ++j)
            SNN_REQUIRE(inst[j].cls != inst[i].cls, "snn_multi_create: instance %d repeats a classifier", i);
    }
    SNN_REQUIRE(cap < (1ull << 31), "snn_multi_create: too many work items");
    SNN_REQUIRE(smem <= 227 * 1024, "snn_multi_create: an instance needs %zu bytes of shared memory", smem);
    snn_multi* m = new snn_multi();
    m->n = n;
    m->cap = (unsigned)cap;
    m->smem = std::max(smem, (size_t)16);
    // seeding order: longest trials (then largest networks) first, so their forwards start early
    m->order.resize(n);
    for (int i = 0; i < n; ++i) m->order[i] = i;
    std::stable_sort(m->order.begin(), m->order.end(), [&](int a, int b) {
        const double ca = (double)h[a].T * (1.0 + h[a].N / 1024.0), cb = (double)h[b].T * (1.0 + h[b].N / 1024.0);
        return ca > cb;
    });
    std::vector<MInst> ho(n);
    for (int k = 0; k < n; ++k) {
        ho[k] = h[m->order[k]];
        ho[k].orig = m->order[k];
    }
    cudaError_t e = cudaMalloc(&m->d_inst, sizeof(MInst) * n);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_remaining, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_q, sizeof(MQueue));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_slots, sizeof(unsigned long long) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_ready, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaHostAlloc(&m->h_mailbox, sizeof(int) * (2 + n), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&m->d_mailbox, m->h_mailbox, 0);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_inst, ho.data(), sizeof(MInst) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_q, 0, sizeof(MQueue));
    if (e == cudaSuccess) e = cudaMemset(m->d_ready, 0, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMemset(m->d_remaining, 0, sizeof(int) * n);
    // the limit is a ceiling only (occupancy follows each launch's own size): the device's
    // opt-in maximum less the kernel's static shared memory serves every plan
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_multi);
    if (e == cudaSuccess && m->smem + fa.sharedSizeBytes > (size_t)optin) {
        set_error("snn_multi_create: %zu bytes of shared memory needed, %d available", m->smem + fa.sharedSizeBytes,
                  optin);
        snn_multi_destroy(m);
        return SNN_EINVAL;
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi, MT, m->smem);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess || per_sm < 1) {
        set_error("snn_multi_create: %s", e != cudaSuccess ? cudaGetErrorString(e) : "kernel does not fit on an SM");
        snn_multi_destroy(m);
        return e != cudaSuccess ? SNN_ECUDA : SNN_EINVAL;
    }
    std::memset(m->h_mailbox, 0, sizeof(int) * (2 + n));
    m->grid = per_sm * sm_count();
    m->runs = 0;
    m->trace = nullptr;
    *out = m;
    return SNN_OK;
}

snn_status snn_multi_run(snn_multi* m, int32_t flags, int64_t wait_limit_ns, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(m, "snn_multi_run: NULL handle");
    SNN_REQUIRE((flags & ~SNN_MULTI_HOST_POSTS) == 0, "snn_multi_run: unknown flags 0x%x", flags);
    SNN_REQUIRE(wait_limit_ns > 0 && wait_limit_ns <= 60ll * 1000000000ll,
                "snn_multi_run: wait_limit_ns must be in (0, 60 s]");
    MArgs a;
    a.inst = m->d_inst;
    a.n_inst = m->n;
    a.remaining = m->d_remaining;
    a.q = m->d_q;
    a.slots = m->d_slots;
    a.ready = m->d_ready;
    a.cap = m->cap;
    a.mailbox = (flags & SNN_MULTI_HOST_POSTS) ? m->d_mailbox : nullptr;
    a.limit_ns = wait_limit_ns;
    a.trace = m->trace;
    k_multi<<<m->grid, MT, m->smem, (cudaStream_t)stream>>>(a);
    SNN_LAUNCH_CHECK();
    m->runs += 1;
    return SNN_OK;
}

snn_status snn_multi_set_trace(snn_multi* m, int64_t* times) {
    clear_error();
    SNN_REQUIRE(m, "snn_multi_set_trace: NULL handle");
    m->trace = (long long*)times;
    return SNN_OK;
}

snn_status snn_multi_post(snn_multi* m, const int32_t* instances, int32_t n) {
    clear_error();
    SNN_REQUIRE(m && n >= 0 && n <= m->n && (instances || n == 0), "snn_multi_post: bad argument");
    for (int k = 0; k < n; ++k) {
        SNN_REQUIRE(instances[k] >= 0 && instances[k] < m->n, "snn_multi_post: instance %d out of range",
                    instances[k]);
        for (int j = 0; j < k; ++j) SNN_REQUIRE(instances[j] != instances[k], "snn_multi_post: instance posted twice");
    }
    volatile int* mb = m->h_mailbox;
    // instance numbers in the caller's order map to the device table's (seeding) order
    for (int k = 0; k < n; ++k) {
        int pos = 0;
        while (m->order[pos] != instances[k]) ++pos;
        mb[2 + k] = pos;
    }
    mb[1] = n;
    __sync_synchronize();
    mb[0] = (int)m->runs;                      // the stamp of the last launched run
    __sync_synchronize();
    return SNN_OK;
}

snn_status snn_multi_status(snn_multi* m, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(m, "snn_multi_status: NULL handle");
    SNN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int32_t st = 0;
    SNN_CUDA(cudaMemcpy(&st, &m->d_q->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    SNN_CUDA(cudaMemset(&m->d_q->status, 0, sizeof(int32_t)));
    if (st & ST_TIMEOUT) {
        set_error("snn_multi_run: a bounded wait for work gave up");
        return SNN_ETIMEOUT;
    }
    if (st & ST_STATE) {
        set_error("snn_multi_run: invalid posted instances");
        return SNN_ESTATE;
    }
    return SNN_OK;
}

snn_status snn_multi_destroy(snn_multi* m) {
    if (!m) return SNN_OK;
    cudaFree(m->d_inst);
    cudaFree(m->d_remaining);
    cudaFree(m->d_q);
    cudaFree(m->d_slots);
    cudaFree(m->d_ready);
    if (m->h_mailbox) cudaFreeHost(m->h_mailbox);
    delete m;
    return SNN_OK;
}

}  // extern "C"
