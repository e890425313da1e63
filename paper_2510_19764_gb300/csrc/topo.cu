// Topographic map (Sec. 2.1.3, Sec. 2.2.2, Tab. 1-2 of the paper): correlated Poisson
// source sheet, conductance LIF target sheet with exponential Euler, all-to-all STDP
// without a transpose (rows are scanned against the post-spike bitmask) and the
// parallel rewiring rule (distance-dependent formation, weight-dependent elimination).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace snn {

struct TopoK {
    int L, L_f, t_stim, n_ref, N, Nw;
    float ds, dplus, dminus, dt_over_tau_m, V_rest, E_exc, V_theta, V_reset, g_leak, g_max, A_plus, A_minus;
};

// Input thresholds by squared distance to the focus: thr[min(d2, n - 1)] (the host
// checks that the profile is flat from entry n - 1 on).  Passed by value (8 KB of kernel
// parameters) and copied to shared memory by each CTA: lanes index it with their own d2,
// which in the constant bank would serialise.
constexpr int TOPO_IN_TAB = 1024;
struct TopoIn {
    uint64_t thr[TOPO_IN_TAB];
    int n;
};

// Tab. 2D / 2F: refractory steps round(tau_ref / dt); A_+ = A_plus_rel g_max and
// A_- = B A_+ tau_+ / tau_-, in double precision on the host.
static snn_topo_derived topo_derived(const snn_topo_params* p) {
    snn_topo_derived d;
    d.n_ref = (int32_t)std::llround(p->tau_ref / p->dt);
    d.reserved = 0;
    d.A_plus = p->A_plus_rel * p->g_max;
    d.A_minus = p->B * d.A_plus * p->tau_plus / p->tau_minus;
    return d;
}

static TopoK topo_consts(const snn_topo_params* p) {
    const snn_topo_derived dv = topo_derived(p);
    TopoK k;
    k.L = p->L;
    k.L_f = p->L_f;
    k.t_stim = p->t_stim;
    k.n_ref = dv.n_ref;
    k.N = p->L * p->L;
    k.Nw = (k.N + 31) / 32;
    k.ds = (float)std::exp(-p->dt / p->tau_s);
    k.dplus = (float)std::exp(-p->dt / p->tau_plus);
    k.dminus = (float)std::exp(-p->dt / p->tau_minus);
    k.dt_over_tau_m = (float)(p->dt / p->tau_m);
    k.V_rest = (float)p->V_rest;
    k.E_exc = (float)p->E_exc;
    k.V_theta = (float)p->V_theta;
    k.V_reset = (float)p->V_reset;
    k.g_leak = (float)p->g_leak;
    k.g_max = (float)p->g_max;
    k.A_plus = (float)dv.A_plus;
    k.A_minus = (float)dv.A_minus;
    return k;
}

// Rate threshold of squared focus distance d2: the disc (sigma_stim = 0) or the Gaussian
// profile of Tab. 1 "Input", floor(rate dt 1e-3 2^64) in double on the host.
static uint64_t input_threshold(const snn_topo_params* p, int d2) {
    if (p->sigma_stim > 0.0)
        return prob_threshold((p->f_base + p->f_in * std::exp(-(double)d2 / (2.0 * p->sigma_stim * p->sigma_stim))) *
                              p->dt * 1e-3);
    return prob_threshold((d2 <= p->radius2 ? p->f_in : p->f_base) * p->dt * 1e-3);
}

// The threshold table of the input profile; rebuilt only when the parameters that
// define it change (the per-step calls would otherwise evaluate it every step).
static snn_status topo_input_table(const snn_topo_params* p, TopoIn& in) {
    struct Key {
        int L_f, radius2;
        double dt, f_base, f_in, sigma;
        bool operator==(const Key& o) const {
            return L_f == o.L_f && radius2 == o.radius2 && dt == o.dt && f_base == o.f_base && f_in == o.f_in &&
                   sigma == o.sigma;
        }
    };
    static thread_local Key last{-1, 0, 0, 0, 0, 0};
    static thread_local TopoIn cached;
    static thread_local bool ok = false;
    const Key key{p->L_f, p->radius2, p->dt, p->f_base, p->f_in, p->sigma_stim};
    if (!(key == last)) {
        const int max_d2 = 2 * (p->L_f / 2) * (p->L_f / 2);
        cached.n = max_d2 + 1 < TOPO_IN_TAB ? max_d2 + 1 : TOPO_IN_TAB;
        for (int d2 = 0; d2 < cached.n; ++d2) cached.thr[d2] = input_threshold(p, d2);
        ok = true;
        for (int d2 = cached.n; d2 <= max_d2 && ok; ++d2) ok = input_threshold(p, d2) == cached.thr[cached.n - 1];
        last = key;
    }
    SNN_REQUIRE(ok, "topo: the input profile is not flat beyond squared distance %d (sigma_stim too wide for L_f)",
                TOPO_IN_TAB - 1);
    in = cached;
    return SNN_OK;
}

// ---- per-step arithmetic shared by the per-call kernels and the fused step loop

// Stimulus focus of step t (the same for every source channel).
__device__ __forceinline__ void topo_focus(const TopoK& k, uint64_t seed, long long t, int& fx, int& fy) {
    const u64x4 f = philox(seed, PH_TOPO_FOCUS, (uint64_t)(t / k.t_stim), 0, 0, 0);
    fx = (int)mulhi_index(f.x, (uint64_t)k.L_f);
    fy = (int)mulhi_index(f.y, (uint64_t)k.L_f);
}

// Source channels 4g .. 4g+3 of step t (one Philox block): spike bits as a nibble;
// xs[q] is channel 4g+q's trace, updated in place.
__device__ __forceinline__ uint32_t topo_input_group(const TopoK& k, const uint64_t* thr, int n_thr, uint64_t seed,
                                                     long long t, int g, int fx, int fy, float (&xs)[4]) {
    uint32_t nib = 0;
    const u64x4 u = philox(seed, PH_TOPO_INPUT, (uint64_t)t, (uint64_t)g, 0, 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = 4 * g + q;
        if (c < k.N) {
            int dx = abs((c % k.L) % k.L_f - fx);
            int dy = abs((c / k.L) % k.L_f - fy);
            dx = min(dx, k.L_f - dx);
            dy = min(dy, k.L_f - dy);
            const bool s = u[q] < thr[min(dx * dx + dy * dy, n_thr - 1)];
            if (s) nib |= 1u << q;
            xs[q] = xs[q] * k.dplus + (s ? 1.0f : 0.0f);
        }
    }
    return nib;
}

// One conductance-LIF neuron step: g decays and takes the summed input I, then either a
// refractory hold or exponential Euler with g held over the step; traces y (ydec = its
// decayed value before the spike) and x.  Returns the spike.
__device__ __forceinline__ bool topo_neuron(const TopoK& k, float I, float& gs, float& V, int& ref, float& y,
                                            float& ydec, float& x) {
    bool z = false;
    const float g = gs * k.ds + I;
    gs = g;
    float v = V;
    if (ref > 0) {
        v = k.V_reset;
        ref = ref - 1;
    } else {
        const float geff = g / k.g_leak;
        const float vinf = (k.V_rest + geff * k.E_exc) / (1.0f + geff);
        v = vinf + (v - vinf) * expf(-k.dt_over_tau_m * (1.0f + geff));
        if (v >= k.V_theta) {
            z = true;
            v = k.V_reset;
            ref = k.n_ref;
        }
    }
    V = v;
    ydec = y * k.dminus;
    y = ydec + (z ? 1.0f : 0.0f);
    x = x * k.dplus + (z ? 1.0f : 0.0f);
    return z;
}

// STDP on one synapse: depression by the postsynaptic trace if the row's neuron spiked,
// then potentiation by the presynaptic trace if the target spiked; clamped to [0, g_max].
__device__ __forceinline__ float stdp_slot(float g, bool pre, bool post, float yd, float xp, float A_plus,
                                           float A_minus, float g_max) {
    if (pre) g = fmaxf(0.0f, g - A_minus * yd);
    if (post) g = fminf(g_max, g + A_plus * xp);
    return g;
}

// Thread = 4 source channels (one Philox block); nibbles of 8 lanes form one word.
__global__ void k_topo_input(TopoK k, const __grid_constant__ TopoIn in, uint64_t seed, long long t,
                             uint32_t* __restrict__ bits, float* __restrict__ x_src) {
    __shared__ int focus[2];
    __shared__ uint64_t s_thr[TOPO_IN_TAB];
    if (threadIdx.x == 0) topo_focus(k, seed, t, focus[0], focus[1]);
    for (int d = threadIdx.x; d < in.n; d += blockDim.x) s_thr[d] = in.thr[d];
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_groups = (k.N + 3) >> 2;
    uint32_t nib = 0;
    if (g < n_groups) {
        float xs[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) xs[q] = 4 * g + q < k.N ? x_src[4 * g + q] : 0.0f;
        nib = topo_input_group(k, s_thr, in.n, seed, t, g, focus[0], focus[1], xs);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < k.N) x_src[4 * g + q] = xs[q];
    }
    uint32_t word = nib << (4 * (g & 7));
    word |= __shfl_xor_sync(0xffffffffu, word, 1);
    word |= __shfl_xor_sync(0xffffffffu, word, 2);
    word |= __shfl_xor_sync(0xffffffffu, word, 4);
    if ((g & 7) == 0 && (g >> 3) < k.Nw) bits[g >> 3] = word;
}

__global__ void k_topo_neurons(TopoK k, float* __restrict__ V, float* __restrict__ gs, int32_t* __restrict__ ref,
                               float* __restrict__ x_tgt, float* __restrict__ y, float* __restrict__ ydec,
                               long long* __restrict__ acc, uint32_t* __restrict__ bits) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool z = false;
    if (j < k.N) {
        const float I = from_fixed<float>(acc[j]);
        acc[j] = 0;
        float g = gs[j], v = V[j], yy = y[j], yd, x = x_tgt[j];
        int r = ref[j];
        z = topo_neuron(k, I, g, v, r, yy, yd, x);
        gs[j] = g;
        V[j] = v;
        ref[j] = r;
        y[j] = yy;
        ydec[j] = yd;
        x_tgt[j] = x;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, z);
    if ((threadIdx.x & 31) == 0 && (j >> 5) < k.Nw) bits[j >> 5] = m;
}

// Warp per row: depression if the row's neuron spiked, potentiation of slots whose
// target spiked; per synapse depression comes first, then potentiation.
__global__ void k_stdp(const int32_t* __restrict__ len, const int32_t* __restrict__ ind, float* __restrict__ w,
                       int P, int C, const uint32_t* __restrict__ pre_bits, const uint32_t* __restrict__ post_bits,
                       const float* __restrict__ x_pre, const float* __restrict__ ydec, float A_plus, float A_minus,
                       float g_max) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= P) return;
    const bool pre = (pre_bits[i >> 5] >> (i & 31)) & 1u;
    const int n = len[i];
    const float xp = x_pre[i];
    for (int s = lane_id(); s < n; s += 32) {
        const size_t o = (size_t)i * C + s;
        const int j = ind[o];
        const bool post = (post_bits[j >> 5] >> (j & 31)) & 1u;
        if (!pre && !post) continue;
        w[o] = stdp_slot(w[o], pre, post, pre ? ydec[j] : 0.0f, xp, A_plus, A_minus, g_max);
    }
}

struct RewireK {
    int P, Q, C, Qw, L, n_att;
    float g_theta, g_new;
    uint64_t thr_dep, thr_pot;
    uint64_t seed, rewire;
    unsigned long long *elim_d2, *form_d2;   // optional event histograms by squared distance
};

__device__ __forceinline__ int torus_d2(int i, int j, int L) {
    int dx = abs(i % L - j % L), dy = abs(i / L - j / L);
    dx = min(dx, L - dx);
    dy = min(dy, L - dy);
    return dx * dx + dy * dy;
}

// One warp: the rewiring of row i with a attempts (Sec. 2.1.3): candidate selection
// without replacement in the warp's shared-memory bitfield cand [Qw] (zero on entry and
// on exit), stable elimination by ballot compaction, and formation of the remaining
// candidates in ascending target order.  Counts are added to the lanes' registers.
__device__ __forceinline__ void topo_rewire_row(const RewireK& k, const int i, const int a, int32_t* __restrict__ len,
                                                int32_t* __restrict__ ind, float* __restrict__ w,
                                                const uint64_t* __restrict__ thr_form, int32_t* status,
                                                uint32_t* cand, long long& removed, long long& formed,
                                                long long& overflow) {
    const int lane = threadIdx.x & 31;
    const uint32_t tail_mask = (k.Q & 31) ? ~((1u << (k.Q & 31)) - 1u) : 0u;
    for (int wi = lane; wi < k.Qw; wi += 32) cand[wi] = 0u;
    __syncwarp();
    // candidates without replacement: the kk-th is the m-th unselected target
    for (int kk = 0; kk < a; ++kk) {
        const u64x4 u = philox(k.seed, PH_TOPO_CAND, k.rewire, (uint64_t)i, (uint64_t)kk, 0);
        const int mth = (int)mulhi_index(u.x, (uint64_t)(k.Q - kk));
        int seen = 0, target = -1;
        for (int wb = 0; wb < k.Qw && target < 0; wb += 32) {
            const int wi = wb + lane;
            uint32_t word = 0xffffffffu;
            if (wi < k.Qw) {
                word = cand[wi];
                if (wi == k.Qw - 1) word |= tail_mask;
            }
            const int zeros = __popc(~word);
            const int incl = warp_incl_scan(zeros);
            const int excl = incl - zeros;
            const uint32_t hm = __ballot_sync(0xffffffffu, mth >= seen + excl && mth < seen + incl);
            if (hm) {
                const int src = __ffs(hm) - 1;
                int tg = -1;
                if (lane == src) tg = wi * 32 + nth_set_bit(~word, mth - seen - excl);
                target = __shfl_sync(0xffffffffu, tg, src);
            }
            seen += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0 && target >= 0) cand[target >> 5] |= 1u << (target & 31);
        if (target < 0 && lane == 0) atomicOr(status, ST_STATE);
        __syncwarp();
    }
    // elimination of existing synapses on candidates
    const int n = __ldcg(len + i);
    const size_t row = (size_t)i * k.C;
    int wp = 0;
    for (int base = 0; base < n; base += 32) {
        const int s = base + lane;
        const bool valid = s < n;
        int j = 0;
        float g = 0.0f;
        bool is_c = false, rm = false;
        if (valid) {
            j = __ldcg(ind + row + s);
            g = __ldcg(w + row + s);
            is_c = (cand[j >> 5] >> (j & 31)) & 1u;
            if (is_c) {
                const u64x4 u = philox(k.seed, PH_TOPO_DRAW, k.rewire, (uint64_t)i, (uint64_t)j, 0);
                rm = u.x < (g < k.g_theta ? k.thr_dep : k.thr_pot);
            }
        }
        const bool keep = valid && !rm;
        const uint32_t mask = __ballot_sync(0xffffffffu, keep);
        removed += rm ? 1 : 0;
        if (rm && k.elim_d2) atomicAdd(&k.elim_d2[torus_d2(i, j, k.L)], 1ull);
        __syncwarp();
        if (is_c) atomicAnd(&cand[j >> 5], ~(1u << (j & 31)));
        if (keep) {
            const int pos = wp + __popc(mask & lanemask_lt());
            ind[row + pos] = j;
            w[row + pos] = g;
        }
        wp += __popc(mask);
        __syncwarp();
    }
    // formation of the remaining candidates, ascending target order
    for (int wb = 0; wb < k.Qw; wb += 32) {
        const int wi = wb + lane;
        uint32_t word = (wi < k.Qw) ? cand[wi] : 0u;
        uint32_t pass = 0;
        for (uint32_t rest = word; rest; rest &= rest - 1u) {
            const int bpos = __ffs(rest) - 1;
            const int j = wi * 32 + bpos;
            const u64x4 u = philox(k.seed, PH_TOPO_DRAW, k.rewire, (uint64_t)i, (uint64_t)j, 0);
            if (u.x < thr_form[torus_d2(i, j, k.L)]) pass |= 1u << bpos;
        }
        const int cnt = __popc(pass);
        const int incl = warp_incl_scan(cnt);
        int rank = incl - cnt;
        for (uint32_t rest = pass; rest; rest &= rest - 1u, ++rank) {
            const int j = wi * 32 + __ffs(rest) - 1;
            const int slot = wp + rank;
            if (slot < k.C) {
                ind[row + slot] = j;
                w[row + slot] = k.g_new;
                ++formed;
                if (k.form_d2) atomicAdd(&k.form_d2[torus_d2(i, j, k.L)], 1ull);
            } else {
                ++overflow;
            }
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        wp = min(wp + total, k.C);
        if (wi < k.Qw) cand[wi] = 0u;
        __syncwarp();
    }
    if (lane == 0) len[i] = wp;
}

// Warp totals of the rewiring counts added to stats (lane 0 of every warp).
__device__ __forceinline__ void topo_flush_counts(snn_rewire_stats* stats, long long removed, long long formed,
                                                  long long overflow, long long attempts, int lane) {
    removed = warp_sum(removed);
    formed = warp_sum(formed);
    overflow = warp_sum(overflow);
    attempts = lane == 0 ? attempts : 0;
    attempts = warp_sum(attempts);
    if (lane == 0 && stats && (removed | formed | overflow | attempts)) {
        atomicAdd((unsigned long long*)&stats->removed, (unsigned long long)removed);
        atomicAdd((unsigned long long*)&stats->formed, (unsigned long long)formed);
        atomicAdd((unsigned long long*)&stats->overflow, (unsigned long long)overflow);
        atomicAdd((unsigned long long*)&stats->attempts, (unsigned long long)attempts);
    }
}

// One CTA.  Histogram of attempt rows, then one warp per row with attempts
// (topo_rewire_row).  Row data are read through L2 (ld.global.cg): inside the fused step
// loop other CTAs of the cluster write them between calls.
__device__ void topo_rewire_cta(const RewireK& k, int32_t* __restrict__ len, int32_t* __restrict__ ind,
                                float* __restrict__ w, const uint64_t* __restrict__ thr_form, int32_t* status,
                                snn_rewire_stats* stats, unsigned char* smem) {
    int* att = (int*)smem;                       // [P]
    int* list = att + k.P;                       // [n_att]
    int* n_rows = list + k.n_att;                // [1]
    uint32_t* cand_all = (uint32_t*)(n_rows + 1);   // [warps][Qw]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = tid; i < k.P; i += blockDim.x) att[i] = 0;
    if (tid == 0) *n_rows = 0;
    __syncthreads();
    for (int g = tid; g < (k.n_att + 3) / 4; g += blockDim.x) {
        const u64x4 u = philox(k.seed, PH_TOPO_ATT, k.rewire, (uint64_t)g, 0, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < k.n_att) atomicAdd(&att[(int)mulhi_index(u[q], (uint64_t)k.P)], 1);
    }
    __syncthreads();
    for (int i = tid; i < k.P; i += blockDim.x)
        if (att[i] > 0) list[atomicAdd(n_rows, 1)] = i;
    __syncthreads();
    const int nr = *n_rows;
    uint32_t* cand = cand_all + (size_t)warp * k.Qw;
    long long removed = 0, formed = 0, overflow = 0, attempts = 0;
    for (int li = warp; li < nr; li += nwarps) {
        const int i = list[li];
        const int a = min(att[i], k.Q);
        attempts += a;
        topo_rewire_row(k, i, a, len, ind, w, thr_form, status, cand, removed, formed, overflow);
    }
    topo_flush_counts(stats, removed, formed, overflow, attempts, lane);
}

__global__ void __launch_bounds__(1024)
    k_topo_rewire(RewireK k, int32_t* __restrict__ len, int32_t* __restrict__ ind, float* __restrict__ w,
                  const uint64_t* __restrict__ thr_form, int32_t* status, snn_rewire_stats* stats) {
    extern __shared__ __align__(16) unsigned char smem[];
    topo_rewire_cta(k, len, ind, w, thr_form, status, stats, smem);
}

// Many CTAs (maps too large for one CTA's shared memory, or many attempts): the attempt
// histogram and the list of rows with attempts go to the handle's scratch in global
// memory, then every warp of the grid takes rows from the list.  A row's rewiring does not
// depend on which warp takes it or when, so the results equal the one-CTA path's.
__global__ void k_topo_att(RewireK k, int32_t* __restrict__ att) {
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < (k.n_att + 3) / 4;
         g += (long long)gridDim.x * blockDim.x) {
        const u64x4 u = philox(k.seed, PH_TOPO_ATT, k.rewire, (uint64_t)g, 0, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < k.n_att) atomicAdd(&att[(int)mulhi_index(u[q], (uint64_t)k.P)], 1);
    }
}

__global__ void k_topo_list(RewireK k, const int32_t* __restrict__ att, int32_t* __restrict__ list,
                            int32_t* __restrict__ n_rows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.P; i += gridDim.x * blockDim.x)
        if (att[i] > 0) list[atomicAdd(n_rows, 1)] = i;
}

constexpr int TOPO_ROW_THREADS = 256;

__global__ void __launch_bounds__(TOPO_ROW_THREADS)
    k_topo_rewire_rows(RewireK k, const int32_t* __restrict__ att, const int32_t* __restrict__ list,
                       const int32_t* __restrict__ n_rows, int32_t* __restrict__ len, int32_t* __restrict__ ind,
                       float* __restrict__ w, const uint64_t* __restrict__ thr_form, int32_t* status,
                       snn_rewire_stats* stats) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* cand = (uint32_t*)smem + (size_t)warp * k.Qw;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int nr = *n_rows;
    long long removed = 0, formed = 0, overflow = 0, attempts = 0;
    for (int li = blockIdx.x * (blockDim.x >> 5) + warp; li < nr; li += nw) {
        const int i = list[li];
        const int a = min(att[i], k.Q);
        attempts += a;
        topo_rewire_row(k, i, a, len, ind, w, thr_form, status, cand, removed, formed, overflow);
    }
    topo_flush_counts(stats, removed, formed, overflow, attempts, lane);
}

static size_t rewire_smem(int P, int n_att, int Qw, int threads) {
    return (size_t)(P + n_att + 1) * 4 + (size_t)(threads / 32) * Qw * 4;
}

static snn_status check_topo(const snn_topo_params* p) {
    SNN_REQUIRE(p, "topo: NULL parameters");
    SNN_REQUIRE(p->L > 0 && p->L_f > 0 && p->L % p->L_f == 0, "topo: need L > 0 and L a multiple of L_f");
    SNN_REQUIRE(p->t_stim > 0 && p->tau_ref >= 0 && p->dt > 0 && p->tau_m > 0 && p->tau_s > 0 && p->g_leak > 0 &&
                    p->tau_plus > 0 && p->tau_minus > 0,
                "topo: bad time constants");
    SNN_REQUIRE(p->tau_ref / p->dt < 1e9, "topo: tau_ref / dt too large");
    SNN_REQUIRE(p->g_max >= 0 && p->A_plus_rel >= 0 && p->B >= 0, "topo: g_max, A_plus_rel and B must be >= 0");
    SNN_REQUIRE(p->sigma_stim >= 0.0, "topo: sigma_stim must be >= 0");
    return SNN_OK;
}

// Validates one projection's rewiring parameters, refreshes its formation-threshold
// table when they changed and fills the kernel constants (rewire index left at 0).
static snn_status rewire_prepare(snn_ragged* r, const snn_topo_rewire* p, RewireK& k, cudaStream_t s) {
    const snn_ragged_desc& d = r->d;
    SNN_REQUIRE(d.dtype == SNN_F32, "snn_rewire_topo: F32 ragged matrices only");
    SNN_REQUIRE(p->L > 0 && (long long)p->L * p->L == d.Q && d.P == d.Q,
                "snn_rewire_topo: the matrix must be L*L x L*L (got P=%d Q=%d L=%d)", d.P, d.Q, p->L);
    SNN_REQUIRE(p->n_att >= 0 && p->n_att <= 65536, "snn_rewire_topo: n_att must be in [0, 65536]");
    SNN_REQUIRE(p->sigma > 0, "snn_rewire_topo: sigma must be > 0");
    const int max_d2 = 2 * (p->L / 2) * (p->L / 2);
    SNN_REQUIRE(max_d2 + 1 <= r->thr_cap, "snn_rewire_topo: distance table does not fit");
    if (r->thr_L != p->L || r->thr_p != p->p_form || r->thr_sigma != p->sigma) {
        // formation thresholds by squared distance, computed once per parameter set on
        // the host in double precision (the first call with new parameters copies them)
        std::vector<uint64_t> tab(max_d2 + 1);
        for (int d2 = 0; d2 <= max_d2; ++d2)
            tab[d2] = prob_threshold(p->p_form * std::exp(-(double)d2 / (2.0 * p->sigma * p->sigma)));
        SNN_CUDA(cudaMemcpyAsync(r->thr_form, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        SNN_CUDA(cudaStreamSynchronize(s));
        r->thr_L = p->L;
        r->thr_p = p->p_form;
        r->thr_sigma = p->sigma;
    }
    k.P = d.P;
    k.Q = d.Q;
    k.C = d.C;
    k.Qw = r->Qw;
    k.L = p->L;
    k.n_att = p->n_att;
    SNN_REQUIRE(p->g_max >= 0, "snn_rewire_topo: g_max must be >= 0");
    k.g_theta = (float)(0.5 * p->g_max);      // Tab. 2G: g_theta = g_max / 2
    k.g_new = (float)p->g_max;                // a new synapse starts at g_max
    k.thr_dep = prob_threshold(p->p_elim_dep);
    k.thr_pot = prob_threshold(p->p_elim_pot);
    k.seed = d.seed;
    k.rewire = 0;
    k.elim_d2 = (unsigned long long*)p->elim_d2;
    k.form_d2 = (unsigned long long*)p->form_d2;
    SNN_REQUIRE((size_t)(TOPO_ROW_THREADS / 32) * k.Qw * 4 <= 227 * 1024, "snn_rewire_topo: Q = %d too large",
                k.Q);
    return SNN_OK;
}

// The one-CTA form serves maps whose attempt histogram fits one CTA's shared memory and
// few attempts (one launch, the paper's sizes); others spread the rows over the grid.
static bool rewire_one_cta(const RewireK& k) {
    return rewire_smem(k.P, k.n_att, k.Qw, 1024) <= 227 * 1024 && k.n_att <= 4096;
}

static snn_status rewire_launch(snn_ragged* r, const snn_topo_rewire* p, int64_t rewire_idx, snn_rewire_stats* stats,
                                cudaStream_t s) {
    RewireK k;
    const snn_status e = rewire_prepare(r, p, k, s);
    if (e != SNN_OK) return e;
    k.rewire = (uint64_t)rewire_idx;
    const snn_ragged_desc& d = r->d;
    if (rewire_one_cta(k)) {
        const int threads = 1024;
        const size_t smem = rewire_smem(k.P, k.n_att, k.Qw, threads);
        if (smem > 48 * 1024)
            SNN_CUDA(cudaFuncSetAttribute(k_topo_rewire, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_topo_rewire<<<1, threads, smem, s>>>(k, d.row_len, d.ind, (float*)d.w, r->thr_form, r->status, stats);
        SNN_LAUNCH_CHECK();
        return SNN_OK;
    }
    int32_t* att = r->cnt;            // handle scratch [P] (also DEEP R's; calls on a handle are ordered)
    int32_t* list = r->taken;         // [P]
    int32_t* n_rows = r->scal;        // one word
    SNN_CUDA(cudaMemsetAsync(att, 0, (size_t)k.P * sizeof(int32_t), s));
    SNN_CUDA(cudaMemsetAsync(n_rows, 0, sizeof(int32_t), s));
    k_topo_att<<<std::max(1, std::min(ceil_div((k.n_att + 3) / 4, 256), 4 * sm_count())), 256, 0, s>>>(k, att);
    SNN_LAUNCH_CHECK();
    k_topo_list<<<std::max(1, std::min(ceil_div(k.P, 256), 4 * sm_count())), 256, 0, s>>>(k, att, list, n_rows);
    SNN_LAUNCH_CHECK();
    const size_t smem = (size_t)(TOPO_ROW_THREADS / 32) * k.Qw * sizeof(uint32_t);
    if (smem > 48 * 1024)
        SNN_CUDA(cudaFuncSetAttribute(k_topo_rewire_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = std::max(1, std::min(ceil_div(std::min(k.n_att, k.P), TOPO_ROW_THREADS / 32), 4 * sm_count()));
    k_topo_rewire_rows<<<grid, TOPO_ROW_THREADS, smem, s>>>(k, att, list, n_rows, d.row_len, d.ind, (float*)d.w,
                                                             r->thr_form, r->status, stats);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

// Connectivity profile: one warp per row; every synapse adds to its torus displacement's
// count and weight sum and to its target's in-degree (global atomics; an analysis pass,
// called once per time bin, not per step).
__global__ void k_topo_profile(const int32_t* __restrict__ len, const int32_t* __restrict__ ind,
                               const float* __restrict__ w, int P, int C, int L,
                               unsigned long long* __restrict__ count, double* __restrict__ wsum,
                               int32_t* __restrict__ indeg) {
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= P) return;
    const int n = len[i], ix = i % L, iy = i / L;
    const size_t row = (size_t)i * C;
    for (int s = lane_id(); s < n; s += 32) {
        const int j = ind[row + s];
        int dx = j % L - ix, dy = j / L - iy;
        dx += dx < 0 ? L : 0;
        dy += dy < 0 ? L : 0;
        const int bin = dy * L + dx;
        if (count) atomicAdd(&count[bin], 1ull);
        if (wsum) atomicAdd(&wsum[bin], (double)w[row + s]);
        if (indeg) atomicAdd(&indeg[j], 1);
    }
}

// ---- fused step loop: the whole network in one thread-block cluster
//
// One cluster of CS CTAs x FUSED_THREADS threads runs many steps in one launch.  Global
// thread j owns target neuron j (and j + CS*FUSED_THREADS ...) with V, g, refractory count and y in
// registers; thread g < ceil(N/4) owns source channels 4g..4g+3 and their traces.  Per
// step, separated by cluster barriers (release/acquire; cross-CTA data are read through
// L2 with ld.global.cg):
//   A. input of step t; propagation of step t-1's source and target spikes (warp per
//      bit word, exact int64 fixed-point atomics into acc)
//   B. neurons of step t (acc consumed), spike words, traces x_tgt, ydec
//   C. STDP on both projections (warp per row, the step's spike words staged in shared
//      memory); after steps with (t+1) % every == 0, CTA 0 rewires ff and CTA 1 lateral.
// The arithmetic is the per-call kernels' (shared device functions), so results are
// identical to the sequence of per-call launches.
struct TopoRun {
    TopoK k;
    TopoIn in;
    int32_t* len[2];      // ff, lateral
    int32_t* ind[2];
    float* w[2];
    int C[2];
    float *V, *gs, *x_src, *x_tgt, *y, *ydec;
    int32_t* ref;
    unsigned long long* acc;
    uint32_t *src_bits, *tgt_bits;
    uint64_t in_seed;
    long long t0;
    int n_steps, rewire_every;
    RewireK rk[2];
    const uint64_t* thr[2];
    int32_t* status[2];
    snn_rewire_stats* stats[2];
};

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

constexpr int FUSED_THREADS = 512;
constexpr int TOPO_FUSED_MAX_NPT = 4;   // neurons per thread the fused loop accepts (1, 2 or 4)

template <int NPT>
__global__ void __launch_bounds__(FUSED_THREADS, 1) k_topo_fused(const __grid_constant__ TopoRun r) {
    extern __shared__ __align__(16) unsigned char smem[];
    const TopoK& k = r.k;
    const int N = k.N, Nw = k.Nw;
    const int TT = gridDim.x * blockDim.x;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = gt >> 5, nwarps = TT >> 5;
    uint32_t* sb_src = (uint32_t*)smem;           // [Nw] spike words of the step (STDP)
    uint32_t* sb_tgt = sb_src + Nw;               // [Nw]
    __shared__ uint64_t s_thr[TOPO_IN_TAB];       // input thresholds by squared focus distance
    for (int d = threadIdx.x; d < r.in.n; d += blockDim.x) s_thr[d] = r.in.thr[d];
    __syncthreads();
    float V[NPT], gs[NPT], y[NPT], xt[NPT];
    int ref[NPT];
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const int j = gt + q * TT;
        const bool ok = j < N;
        V[q] = ok ? r.V[j] : 0.0f;
        gs[q] = ok ? r.gs[j] : 0.0f;
        y[q] = ok ? r.y[j] : 0.0f;
        xt[q] = ok ? r.x_tgt[j] : 0.0f;
        ref[q] = ok ? r.ref[j] : 0;
    }
    const int Ng = (N + 3) >> 2;
    const bool has_group = gt < Ng;
    float xs[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xs[q] = (has_group && 4 * gt + q < N) ? r.x_src[4 * gt + q] : 0.0f;
    long long fper = -1;
    int fx = 0, fy = 0;
    for (long long t = r.t0; t < r.t0 + r.n_steps; ++t) {
        const int cur = (int)(t & 1), prv = cur ^ 1;
        // ---------------- A: input of step t, propagation of step t-1
        {
            uint32_t nib = 0;
            if (has_group) {
                if (t / k.t_stim != fper) {
                    fper = t / k.t_stim;
                    topo_focus(k, r.in_seed, t, fx, fy);
                }
                nib = topo_input_group(k, s_thr, r.in.n, r.in_seed, t, gt, fx, fy, xs);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * gt + q < N) r.x_src[4 * gt + q] = xs[q];
            }
            uint32_t word = nib << (4 * (gt & 7));
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            word |= __shfl_xor_sync(0xffffffffu, word, 4);
            if ((gt & 7) == 0 && (gt >> 3) < Nw) r.src_bits[cur * Nw + (gt >> 3)] = word;
        }
        for (int wd = gwarp; wd < 2 * Nw; wd += nwarps) {
            const int m = wd < Nw ? 0 : 1;            // 0: ff rows (source spikes), 1: lateral
            const int wi = wd - m * Nw;
            uint32_t bits = __ldcg((m == 0 ? r.src_bits : r.tgt_bits) + prv * Nw + wi);
            const int32_t* ind = r.ind[m];
            const float* wt = r.w[m];
            const int C = r.C[m];
            // lengths of all spiking rows of the word in one round trip
            const int n_l = ((bits >> lane) & 1u) ? __ldcg(r.len[m] + wi * 32 + lane) : 0;
            while (bits) {
                const int b = __ffs(bits) - 1;
                const int i = wi * 32 + b;
                bits &= bits - 1u;
                const int n = __shfl_sync(0xffffffffu, n_l, b);
                for (int s = lane; s < n; s += 32) {
                    const size_t o = (size_t)i * C + s;
                    atomicAdd(r.acc + __ldcg(ind + o), (unsigned long long)to_fixed(__ldcg(wt + o)));
                }
            }
        }
        cluster_barrier();
        // ---------------- B: neurons of step t
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int j = gt + q * TT;
            bool z = false;
            if (j < N) {
                const float I = from_fixed<float>((long long)__ldcg(r.acc + j));
                r.acc[j] = 0ull;
                float yd;
                z = topo_neuron(k, I, gs[q], V[q], ref[q], y[q], yd, xt[q]);
                r.ydec[j] = yd;
                r.x_tgt[j] = xt[q];
            }
            const uint32_t zm = __ballot_sync(0xffffffffu, z);
            const int j0 = j - lane;                  // the warp's first neuron
            if (lane == 0 && (j0 >> 5) < Nw) r.tgt_bits[cur * Nw + (j0 >> 5)] = zm;
        }
        cluster_barrier();
        // ---------------- C: STDP of step t, then rewiring
        for (int wi = threadIdx.x; wi < Nw; wi += blockDim.x) {
            sb_src[wi] = __ldcg(r.src_bits + cur * Nw + wi);
            sb_tgt[wi] = __ldcg(r.tgt_bits + cur * Nw + wi);
        }
        __syncthreads();
        // warp = batches of 8 rows whose loads are issued together (3 L2 round trips per
        // 32-slot chunk of the batch instead of per row)
        for (int rb = gwarp * 8; rb < 2 * N; rb += nwarps * 8) {
            int n_l = 0;
            float xp_l = 0.0f;
            bool pre_l = false;
            if (lane < 8 && rb + lane < 2 * N) {
                const int row = rb + lane, m = row < N ? 0 : 1, i = row - m * N;
                n_l = __ldcg(r.len[m] + i);
                xp_l = __ldcg((m == 0 ? r.x_src : r.x_tgt) + i);
                pre_l = ((m == 0 ? sb_src : sb_tgt)[i >> 5] >> (i & 31)) & 1u;
            }
            int nq[8], nmax = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                nq[q] = __shfl_sync(0xffffffffu, n_l, q);
                nmax = max(nmax, nq[q]);
            }
            for (int s0 = 0; s0 < nmax; s0 += 32) {
                int j[8];
                size_t o[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int row = rb + q, m = row < N ? 0 : 1, i = row - m * N;
                    o[q] = (size_t)i * r.C[m] + s0 + lane;
                    j[q] = s0 + lane < nq[q] ? __ldcg(r.ind[m] + o[q]) : -1;
                }
                float g[8], yd[8];
                bool pre[8], post[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int row = rb + q, m = row < N ? 0 : 1;
                    pre[q] = __shfl_sync(0xffffffffu, pre_l, q);
                    post[q] = j[q] >= 0 && ((sb_tgt[j[q] >> 5] >> (j[q] & 31)) & 1u);
                    const bool upd = j[q] >= 0 && (pre[q] || post[q]);
                    g[q] = upd ? __ldcg(r.w[m] + o[q]) : 0.0f;
                    yd[q] = (upd && pre[q]) ? __ldcg(r.ydec + j[q]) : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int row = rb + q, m = row < N ? 0 : 1;
                    const float xp = __shfl_sync(0xffffffffu, xp_l, q);
                    if (j[q] >= 0 && (pre[q] || post[q]))
                        r.w[m][o[q]] = stdp_slot(g[q], pre[q], post[q], yd[q], xp, k.A_plus, k.A_minus, k.g_max);
                }
            }
        }
        if ((t + 1) % r.rewire_every == 0) {
            cluster_barrier();
            if (blockIdx.x < 2) {
                const int m = blockIdx.x;
                RewireK rk = r.rk[m];
                rk.rewire = (uint64_t)((t + 1) / r.rewire_every - 1);
                topo_rewire_cta(rk, r.len[m], r.ind[m], r.w[m], r.thr[m], r.status[m], r.stats[m], smem);
            }
        }
        cluster_barrier();
    }
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const int j = gt + q * TT;
        if (j < N) {
            r.V[j] = V[q];
            r.gs[j] = gs[q];
            r.y[j] = y[q];
            r.ref[j] = ref[q];
        }
    }
}

// Cluster size for the fused loop: the largest of 16 / 8 / 4 / 2 CTAs that can be
// resident (0 if none).
template <int NPT>
static int fused_cluster_size(size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_topo_fused<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    cudaFuncSetAttribute(k_topo_fused<NPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cs = 16; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(FUSED_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_topo_fused<NPT>, &cfg) == cudaSuccess && n >= 1) return cs;
    }
    cudaGetLastError();
    return 0;
}

template <int NPT>
static snn_status launch_fused(const TopoRun& run, int cs, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(FUSED_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SNN_CUDA(cudaLaunchKernelEx(&cfg, k_topo_fused<NPT>, run));
    return SNN_OK;
}

}  // namespace snn

using namespace snn;

extern "C" {

snn_status snn_topo_input(const snn_topo_params* p, const snn_topo_state* st, uint64_t seed, int64_t t,
                          snn_stream stream) {
    clear_error();
    snn_status e = check_topo(p);
    if (e != SNN_OK) return e;
    SNN_REQUIRE(st && st->src_bits && st->x_src && t >= 0, "snn_topo_input: bad argument");
    TopoK k = topo_consts(p);
    static thread_local TopoIn in;
    if ((e = topo_input_table(p, in)) != SNN_OK) return e;
    const int groups = (k.N + 3) / 4;
    k_topo_input<<<ceil_div(groups, 256), 256, 0, (cudaStream_t)stream>>>(k, in, seed, t,
                                                                          st->src_bits + (t & 1) * k.Nw, st->x_src);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_topo_neurons(const snn_topo_params* p, const snn_topo_state* st, int64_t t, snn_stream stream) {
    clear_error();
    snn_status e = check_topo(p);
    if (e != SNN_OK) return e;
    SNN_REQUIRE(st && st->V && st->gs && st->ref && st->x_tgt && st->y && st->ydec && st->acc && st->tgt_bits && t >= 0,
                "snn_topo_neurons: bad argument");
    TopoK k = topo_consts(p);
    k_topo_neurons<<<ceil_div(k.N, 256), 256, 0, (cudaStream_t)stream>>>(k, st->V, st->gs, st->ref, st->x_tgt, st->y,
                                                                        st->ydec, (long long*)st->acc,
                                                                        st->tgt_bits + (t & 1) * k.Nw);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_topo_derive(const snn_topo_params* p, snn_topo_derived* out) {
    clear_error();
    SNN_REQUIRE(out, "snn_topo_derive: NULL output");
    snn_status st = check_topo(p);
    if (st != SNN_OK) return st;
    *out = topo_derived(p);
    return SNN_OK;
}

snn_status snn_stdp_update(snn_ragged* r, const snn_topo_params* p, const uint32_t* pre_bits, const uint32_t* post_bits,
                           const float* x_pre, const float* ydec, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && p && pre_bits && post_bits && x_pre && ydec, "snn_stdp_update: NULL argument");
    SNN_REQUIRE(r->d.dtype == SNN_F32, "snn_stdp_update: F32 only");
    snn_status st = check_topo(p);
    if (st != SNN_OK) return st;
    const snn_topo_derived dv = topo_derived(p);
    const snn_ragged_desc& d = r->d;
    k_stdp<<<ceil_div((long long)d.P * 32, 256), 256, 0, (cudaStream_t)stream>>>(
        d.row_len, d.ind, (float*)d.w, d.P, d.C, pre_bits, post_bits, x_pre, ydec, (float)dv.A_plus,
        (float)dv.A_minus, (float)p->g_max);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_rewire_topo(snn_ragged* r, const snn_topo_rewire* p, int64_t rewire_idx, snn_rewire_stats* stats,
                           snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && p && rewire_idx >= 0, "snn_rewire_topo: bad argument");
    return rewire_launch(r, p, rewire_idx, stats, (cudaStream_t)stream);
}

snn_status snn_topo_connectivity(const snn_ragged* r, int32_t L, int64_t* disp_count, double* disp_wsum,
                                 int32_t* in_degree, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r, "snn_topo_connectivity: NULL handle");
    const snn_ragged_desc& d = r->d;
    SNN_REQUIRE(d.dtype == SNN_F32, "snn_topo_connectivity: F32 ragged matrices only");
    SNN_REQUIRE(L > 0 && (long long)L * L == d.Q && d.P == d.Q,
                "snn_topo_connectivity: the matrix must be L*L x L*L (got P=%d Q=%d L=%d)", d.P, d.Q, L);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)L * L;
    if (disp_count) SNN_CUDA(cudaMemsetAsync(disp_count, 0, N * sizeof(int64_t), s));
    if (disp_wsum) SNN_CUDA(cudaMemsetAsync(disp_wsum, 0, N * sizeof(double), s));
    if (in_degree) SNN_CUDA(cudaMemsetAsync(in_degree, 0, N * sizeof(int32_t), s));
    if (!disp_count && !disp_wsum && !in_degree) return SNN_OK;
    const int threads = 256;
    k_topo_profile<<<ceil_div((long long)d.P * 32, threads), threads, 0, s>>>(
        d.row_len, d.ind, (const float*)d.w, d.P, d.C, L, (unsigned long long*)disp_count, disp_wsum, in_degree);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_topo_run(const snn_topo_params* p, const snn_topo_state* st, snn_ragged* ff, snn_ragged* lat,
                        const snn_topo_rewire* rw_ff, const snn_topo_rewire* rw_lat, uint64_t input_seed,
                        int32_t rewire_every, int64_t t0, int32_t n_steps, snn_rewire_stats* stats_ff,
                        snn_rewire_stats* stats_lat, snn_stream stream) {
    clear_error();
    snn_status e = check_topo(p);
    if (e != SNN_OK) return e;
    SNN_REQUIRE(st && ff && lat && rw_ff && rw_lat && rewire_every > 0 && t0 >= 0 && n_steps >= 0,
                "snn_topo_run: bad argument");
    const int N = p->L * p->L, Nw = (N + 31) / 32;
    SNN_REQUIRE(ff->d.P == N && ff->d.Q == N && lat->d.P == N && lat->d.Q == N,
                "snn_topo_run: projections must be N x N with N = L*L");
    if (n_steps == 0) return SNN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // fused path: one cluster launch per (up to) 1000 steps
    if (ff->d.dtype == SNN_F32 && lat->d.dtype == SNN_F32 && st->V && st->gs && st->ref && st->x_src && st->x_tgt &&
        st->y && st->ydec && st->acc && st->src_bits && st->tgt_bits) {
        TopoRun run;
        if ((e = rewire_prepare(ff, rw_ff, run.rk[0], s)) != SNN_OK) return e;
        if ((e = rewire_prepare(lat, rw_lat, run.rk[1], s)) != SNN_OK) return e;
        const int max_att = rw_ff->n_att > rw_lat->n_att ? rw_ff->n_att : rw_lat->n_att;
        size_t smem = rewire_smem(N, max_att, ff->Qw > lat->Qw ? ff->Qw : lat->Qw, FUSED_THREADS);
        if (smem < (size_t)2 * Nw * 4) smem = (size_t)2 * Nw * 4;
        // one neuron per thread: beyond one cluster's threads the per-step launches spread
        // STDP over the whole GPU and win
        // neurons per thread: one while the cluster has a thread per neuron, else up to
        // TOPO_FUSED_MAX_NPT (beyond that the per-step launches spread STDP wider)
        int cs = smem <= 227 * 1024 ? fused_cluster_size<1>(smem, s) : 0;
        const int npt = cs >= 2 ? (N + cs * FUSED_THREADS - 1) / (cs * FUSED_THREADS) : 0;
        // the chosen instantiation gets its own launch attributes and cluster size
        if (npt == 2) cs = fused_cluster_size<2>(smem, s);
        if (npt > 2 && npt <= 4) cs = fused_cluster_size<4>(smem, s);
        if (cs >= 2 && npt <= TOPO_FUSED_MAX_NPT && N <= (npt > 2 ? 4 : npt) * cs * FUSED_THREADS) {
            run.k = topo_consts(p);
            if ((e = topo_input_table(p, run.in)) != SNN_OK) return e;
            for (int m = 0; m < 2; ++m) {
                snn_ragged* r = m == 0 ? ff : lat;
                run.len[m] = r->d.row_len;
                run.ind[m] = r->d.ind;
                run.w[m] = (float*)r->d.w;
                run.C[m] = r->d.C;
                run.thr[m] = r->thr_form;
                run.status[m] = r->status;
            }
            run.stats[0] = stats_ff;
            run.stats[1] = stats_lat;
            run.V = st->V;
            run.gs = st->gs;
            run.ref = st->ref;
            run.x_src = st->x_src;
            run.x_tgt = st->x_tgt;
            run.y = st->y;
            run.ydec = st->ydec;
            run.acc = (unsigned long long*)st->acc;
            run.src_bits = st->src_bits;
            run.tgt_bits = st->tgt_bits;
            run.in_seed = input_seed;
            run.rewire_every = rewire_every;
            for (int64_t t = t0; t < t0 + n_steps; t += 1000) {
                run.t0 = t;
                run.n_steps = (int)(t0 + n_steps - t < 1000 ? t0 + n_steps - t : 1000);
                e = npt == 1 ? launch_fused<1>(run, cs, smem, s)
                             : npt == 2 ? launch_fused<2>(run, cs, smem, s) : launch_fused<4>(run, cs, smem, s);
                if (e != SNN_OK) return e;
            }
            return SNN_OK;
        }
    }
    for (int64_t t = t0; t < t0 + n_steps; ++t) {
        const int cur = (int)(t & 1), prv = cur ^ 1;
        if ((e = snn_topo_input(p, st, input_seed, t, stream)) != SNN_OK) return e;
        if ((e = snn_propagate(ff, st->src_bits + prv * Nw, 1, st->acc, stream)) != SNN_OK) return e;
        if ((e = snn_propagate(lat, st->tgt_bits + prv * Nw, 1, st->acc, stream)) != SNN_OK) return e;
        if ((e = snn_topo_neurons(p, st, t, stream)) != SNN_OK) return e;
        if ((e = snn_stdp_update(ff, p, st->src_bits + cur * Nw, st->tgt_bits + cur * Nw, st->x_src, st->ydec,
                                 stream)) != SNN_OK)
            return e;
        if ((e = snn_stdp_update(lat, p, st->tgt_bits + cur * Nw, st->tgt_bits + cur * Nw, st->x_tgt, st->ydec,
                                 stream)) != SNN_OK)
            return e;
        if ((t + 1) % rewire_every == 0) {
            const int64_t ridx = (t + 1) / rewire_every - 1;
            if ((e = snn_rewire_topo(ff, rw_ff, ridx, stats_ff, stream)) != SNN_OK) return e;
            if ((e = snn_rewire_topo(lat, rw_lat, ridx, stats_lat, stream)) != SNN_OK) return e;
        }
    }
    return SNN_OK;
}

}  // extern "C"
