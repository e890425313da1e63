// DEEP R rewiring on the ragged matrix with sign and connectivity bitfields
// (Sec. 2.1.2, Fig. 2B-C of the paper).
//
//  k_deepr_eliminate  : one warp per row, two 32-slot chunks per memory round trip; a
//                       synapse is dormant when its weight's sign is strictly opposite to
//                       its fixed sign bit (read from the slot's sign tag when the tag's
//                       target matches, else from the bitfield); survivors are compacted
//                       stably with a warp ballot + prefix count (w, m, v move along),
//                       connectivity bits of removed synapses are cleared; the dormant
//                       total D is summed on the device.
//  k_deepr_round0     : the whole grid draws round 0 of the redistribution (D rows)
//                       into a per-row histogram with integer atomics.
//  k_deepr_accept0    : the whole grid accepts round 0 up to each row's room.
//  k_deepr_distribute : one CTA; runs the remaining rounds on the leftovers
//                       (order-independent counts).
//  k_deepr_form       : one warp per row with activations; per-chunk free counts (chunks
//                       of 1024 targets, kept in shared memory); a row with up to 32
//                       activations resolves them side by side (one lane each), a row
//                       with more one after another; either way a scan over the chunk
//                       counts finds the chunk and a 32-word scan finds the bit.
//  k_deepr_form_guided: distance-guided variant (a guide attached to the handle).
#include "deepr_dev.cuh"

#include <cmath>
#include <mutex>
#include <vector>

namespace snn {

constexpr int DEEPR_THREADS = 256;

template <typename real>
__global__ void __launch_bounds__(DEEPR_THREADS)
    k_deepr_eliminate(int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w,
                      real* __restrict__ m, real* __restrict__ v, const uint32_t* __restrict__ sign,
                      uint32_t* __restrict__ conn, uint32_t* __restrict__ tag, int32_t* __restrict__ dormant,
                      int32_t* __restrict__ cnt, unsigned long long* __restrict__ dsum, int P, int C, int Qw) {
    __shared__ int removed_w[DEEPR_THREADS / 32];
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (i < P) eliminate_row(len, ind, w, m, v, sign, conn, tag, dormant, cnt, i, C, Qw);
    if (lane == 0) removed_w[threadIdx.x >> 5] = i < P ? dormant[i] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += removed_w[k];
        if (t) atomicAdd(dsum, (unsigned long long)t);
    }
}

// Round 0 of the redistribution over the whole grid: activation k draws row mulhi(u, P)
// with u = Philox(DEEPR_DIST; (rewire, 0, k/4, 0)) word k%4.
__global__ void k_deepr_round0(const unsigned long long* __restrict__ dsum, int32_t* __restrict__ cnt, int P,
                               uint64_t seed, uint64_t rewire, const long long* ridx_dev) {
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    const long long D = (long long)*dsum;
    const long long groups = (D + 3) >> 2;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const u64x4 u = philox(seed, PH_DEEPR_DIST, rewire, 0, (uint64_t)g, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < D) atomicAdd(&cnt[(int)mulhi_index(u[q], (uint64_t)P)], 1);
    }
}

// Round 0 accepted over the whole grid: each row's room is min(C - len, free targets);
// it takes min(cnt, room) activations, the rest are rejections (summed on the device).
__global__ void k_deepr_accept0(const int32_t* __restrict__ len, const int32_t* __restrict__ cnt,
                                int32_t* __restrict__ room, int32_t* __restrict__ taken,
                                unsigned long long* __restrict__ rejected, int P, int C, int Q, int no_autapse) {
    __shared__ long long red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    long long rej = 0;
    if (i < P) {
        const int forb = (no_autapse && i < Q) ? 1 : 0;
        const int l = len[i];
        const int r1 = C - l, r2 = Q - forb - l;
        const int rm = r1 < r2 ? r1 : r2;
        const int c = cnt[i];
        const int acc = c < rm ? c : rm;
        room[i] = rm;
        taken[i] = acc;
        rej = c - acc;
    }
    const long long t = block_sum_ll(rej, red);
    if (threadIdx.x == 0 && t) atomicAdd(rejected, (unsigned long long)t);
}

// Rounds 1..63 on the activations round 0 rejected (usually none: the CTA then only
// records the counts).  One CTA; per round it draws the remaining activations' rows
// with integer atomics and accepts them up to each row's remaining room.
__global__ void __launch_bounds__(1024)
    k_deepr_distribute(const int32_t* __restrict__ room, int32_t* __restrict__ taken, int32_t* __restrict__ cnt,
                       const unsigned long long* __restrict__ dsum, const unsigned long long* __restrict__ rejected,
                       int P, uint64_t seed, uint64_t rewire, const long long* ridx_dev, int32_t* status,
                       snn_rewire_stats* stats) {
    __shared__ long long red[32];
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    const long long D = (long long)*dsum;
    long long remaining = (long long)*rejected;
    for (int r = 1; r < 64 && remaining > 0; ++r) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const long long groups = (remaining + 3) >> 2;
        for (long long g = threadIdx.x; g < groups; g += blockDim.x) {
            const u64x4 u = philox(seed, PH_DEEPR_DIST, rewire, (uint64_t)r, (uint64_t)g, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (4 * g + q < remaining) atomicAdd(&cnt[(int)mulhi_index(u[q], (uint64_t)P)], 1);
            }
        }
        __syncthreads();
        long long rej = 0;
#pragma unroll 8
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int c = cnt[i];
            if (c) {
                const int free_ = room[i] - taken[i];
                const int acc = c < free_ ? c : free_;
                taken[i] += acc;
                rej += c - acc;
            }
        }
        remaining = block_sum_ll(rej, red);
    }
    if (threadIdx.x == 0) {
        if (remaining > 0) atomicOr(status, ST_CAPACITY);
        if (stats) {
            atomicAdd((unsigned long long*)&stats->removed, (unsigned long long)D);
            atomicAdd((unsigned long long*)&stats->overflow, (unsigned long long)remaining);
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(DEEPR_THREADS)
    k_deepr_form(int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w, real* __restrict__ m,
                 real* __restrict__ v, uint32_t* __restrict__ conn, const int32_t* __restrict__ taken, int P, int C,
                 int Q, int Qw, int no_autapse, uint64_t seed, uint64_t rewire, const long long* ridx_dev,
                 int32_t* status, snn_rewire_stats* stats) {
    extern __shared__ int32_t form_smem[];           // per warp: free counts of its row's chunks
    const int NC = (Qw + 31) >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    if (i >= P) return;
    form_row_warp<real>(len, ind, w, m, v, conn, taken, i, C, Q, Qw, no_autapse, seed, rewire, status, stats,
                        form_smem + (size_t)(threadIdx.x >> 5) * (NC + 1));
}

// ---- distance-guided formation
struct GuideK {
    const int32_t* pre_site;
    const int32_t* post_site;
    const uint32_t* q;           // weight by squared torus distance of the two sites
    int L;
};

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t guide_weight(const GuideK& g, int sx, int sy, int j) {
    const int t = g.post_site[j];
    int dx = abs(t % g.L - sx), dy = abs(t / g.L - sy);
    dx = min(dx, g.L - dx);
    dy = min(dy, g.L - dy);
    return g.q[dx * dx + dy * dy];
}

// Weight of the free targets in one bitfield word (free: its zero bits, inverted).
__device__ __forceinline__ unsigned long long word_weight(const GuideK& g, int sx, int sy, uint32_t free_bits,
                                                          int wi) {
    unsigned long long s = 0;
    for (uint32_t rest = free_bits; rest; rest &= rest - 1u) s += guide_weight(g, sx, sy, wi * 32 + __ffs(rest) - 1);
    return s;
}

// One warp per row with activations; activation k draws u as the uniform rule does and
// picks the free target where the running weight sum (ascending targets) first exceeds
// r = mulhi(u, S), S the weight total; with S = 0 every free target weighs 1 (the
// uniform rule).  Two passes over the row's bitfield per activation: the total, then
// the word holding r, whose owner lane walks its free bits.
template <typename real>
__global__ void __launch_bounds__(DEEPR_THREADS)
    k_deepr_form_guided(int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w,
                        real* __restrict__ m, real* __restrict__ v, uint32_t* __restrict__ conn,
                        const int32_t* __restrict__ taken, int P, int C, int Q, int Qw, int no_autapse, uint64_t seed,
                        uint64_t rewire, const long long* ridx_dev, int32_t* status, snn_rewire_stats* stats,
                        GuideK g) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    if (i >= P) return;
    const int nt = taken[i];
    if (nt == 0) return;
    const int lane = lane_id();
    const int forb = (no_autapse && i < Q) ? 1 : 0;
    const uint32_t tail_mask = (Q & 31) ? ~((1u << (Q & 31)) - 1u) : 0u;
    uint32_t* crow = conn + (size_t)i * Qw;
    const size_t row = (size_t)i * C;
    const int si = g.pre_site[i];
    const int sx = si % g.L, sy = si / g.L;
    int n = len[i];
    int formed = 0;
    uint64_t u_l = 0;
    for (int k = 0; k < nt; ++k) {
        const int n_free = Q - forb - n;
        if (n_free <= 0 || n >= C) {
            if (lane == 0) atomicOr(status, ST_STATE);
            break;
        }
        if ((k & 31) == 0 && k + lane < nt) u_l = philox(seed, PH_DEEPR_FORM, rewire, (uint64_t)i, (uint64_t)(k + lane), 0).x;
        const uint64_t u = __shfl_sync(0xffffffffu, u_l, k & 31);
        unsigned long long S = 0;
        for (int wb = 0; wb < Qw; wb += 32) {
            const int wi = wb + lane;
            S += word_weight(g, sx, sy, ~conn_word(crow, wi, Qw, i, forb, tail_mask), wi);
        }
        S = warp_sum(S);
        const bool flat = S == 0;
        const unsigned long long r = mulhi_index(u, flat ? (uint64_t)n_free : (uint64_t)S);
        unsigned long long seen = 0;
        int target = -1;
        for (int wb = 0; wb < Qw && target < 0; wb += 32) {
            const int wi = wb + lane;
            const uint32_t fb = ~conn_word(crow, wi, Qw, i, forb, tail_mask);
            const unsigned long long ww = flat ? (unsigned long long)__popc(fb) : word_weight(g, sx, sy, fb, wi);
            const unsigned long long incl = warp_incl_scan_u64(ww);
            const unsigned long long excl = incl - ww;
            const uint32_t hm = __ballot_sync(0xffffffffu, r >= seen + excl && r < seen + incl);
            if (hm) {
                const int src = __ffs(hm) - 1;
                int tg = -1;
                if (lane == src) {
                    unsigned long long acc = seen + excl;
                    for (uint32_t rest = fb; rest; rest &= rest - 1u) {
                        const int j = wi * 32 + __ffs(rest) - 1;
                        acc += flat ? 1ull : guide_weight(g, sx, sy, j);
                        if (acc > r) {
                            tg = j;
                            break;
                        }
                    }
                }
                target = __shfl_sync(0xffffffffu, tg, src);
            }
            seen += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (target < 0) {
            if (lane == 0) atomicOr(status, ST_STATE);
            break;
        }
        if (lane == 0) {
            ind[row + n] = target;
            w[row + n] = real(0);
            m[row + n] = real(0);
            v[row + n] = real(0);
            crow[target >> 5] |= 1u << (target & 31);
        }
        __syncwarp();
        ++n;
        ++formed;
    }
    if (lane == 0) {
        len[i] = n;
        if (stats) atomicAdd((unsigned long long*)&stats->formed, (unsigned long long)formed);
    }
}

__global__ void k_check_sites(const int32_t* __restrict__ site, int n, int lim, int32_t* status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && (site[k] < 0 || site[k] >= lim)) atomicOr(status, ST_STATE);
}

// Launch sequence of one rewiring.  dsum: device uint64[2] scratch (dormant total,
// round-0 rejections), zeroed here.
template <typename real>
static snn_status rewire_launch_all(const snn_ragged_desc& d, int Qw, int32_t* dormant, int32_t* taken,
                                    int32_t* room, int32_t* cnt, unsigned long long* dsum, int32_t* status,
                                    uint64_t rewire, const long long* ridx_dev, snn_rewire_stats* stats,
                                    cudaStream_t s, const GuideK* guide = nullptr, uint32_t* tag = nullptr) {
    const int blocks = ceil_div((long long)d.P * 32, DEEPR_THREADS);
    // every size check before the first launch: a refused call leaves the matrix untouched
    const size_t smem = (size_t)(DEEPR_THREADS / 32) * ((Qw + 31) / 32 + 1) * sizeof(int32_t);
    SNN_REQUIRE(guide || smem <= 48 * 1024, "snn_rewire_deepr: Q = %d too large for the formation chunk table",
                d.Q);
    SNN_CUDA(cudaMemsetAsync(dsum, 0, 2 * sizeof(unsigned long long), s));
    k_deepr_eliminate<real><<<blocks, DEEPR_THREADS, 0, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v,
                                                              d.sign_bits, d.conn_bits, tag, dormant, cnt, dsum, d.P,
                                                              d.C, Qw);
    SNN_LAUNCH_CHECK();
    k_deepr_round0<<<2 * sm_count(), 256, 0, s>>>(dsum, cnt, d.P, d.seed, rewire, ridx_dev);
    SNN_LAUNCH_CHECK();
    k_deepr_accept0<<<ceil_div(d.P, 256), 256, 0, s>>>(d.row_len, cnt, room, taken, dsum + 1, d.P, d.C, d.Q,
                                                       d.no_autapse);
    SNN_LAUNCH_CHECK();
    k_deepr_distribute<<<1, 1024, 0, s>>>(room, taken, cnt, dsum, dsum + 1, d.P, d.seed, rewire, ridx_dev, status,
                                          stats);
    SNN_LAUNCH_CHECK();
    if (guide) {
        k_deepr_form_guided<real><<<blocks, DEEPR_THREADS, 0, s>>>(
            d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v, d.conn_bits, taken, d.P, d.C, d.Q, Qw, d.no_autapse,
            d.seed, rewire, ridx_dev, status, stats, *guide);
        SNN_LAUNCH_CHECK();
        return SNN_OK;
    }
    k_deepr_form<real><<<blocks, DEEPR_THREADS, smem, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v,
                                                            d.conn_bits, taken, d.P, d.C, d.Q, Qw, d.no_autapse,
                                                            d.seed, rewire, ridx_dev, status, stats);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

template <typename real>
static snn_status rewire_impl(snn_ragged* r, uint64_t rewire, const long long* ridx_dev, snn_rewire_stats* stats,
                              cudaStream_t s) {
    GuideK g;
    if (r->guide_on) {
        g.pre_site = r->guide_pre;
        g.post_site = r->guide_post;
        g.q = r->guide_q;
        g.L = r->guide_L;
    }
    return rewire_launch_all<real>(r->d, r->Qw, r->dormant, r->taken, r->room, r->cnt,
                                   (unsigned long long*)r->scal, r->status, rewire, ridx_dev, stats, s,
                                   r->guide_on ? &g : nullptr, r->stag);
}

// ------------------------------------------------------------------ no-allocation variant
// Fixed scratch for snn_rewire_deepr_noalloc: four int32 arrays of NOALLOC_MAX_ROWS rows
// (dormant counts, taken, room, per-round histogram), one status word and (at words
// 8-11 of the tail) the uint64 dormant total and round-0 rejections.  It lives in
// every device that loads the library until the process exits.
constexpr int NOALLOC_MAX_ROWS = 16384;
static __device__ __align__(256) int32_t g_noalloc_scratch[4 * NOALLOC_MAX_ROWS + 32];

static int32_t* g_noalloc_ptr[256];
static std::mutex g_noalloc_mu;

// Device address of the static scratch for the current device.  The first call on a
// device looks it up with cudaGetSymbolAddress (the host-side symbol is only a stand-in
// for it) and caches it.
static snn_status noalloc_scratch(int32_t** out) {
    int dev = -1;
    SNN_CUDA(cudaGetDevice(&dev));
    SNN_REQUIRE(dev >= 0 && dev < 256, "snn_rewire_deepr_noalloc: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("snn_rewire_deepr_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SNN_ECUDA;
        }
        g_noalloc_ptr[dev] = (int32_t*)p;
    }
    *out = g_noalloc_ptr[dev];
    return SNN_OK;
}

template <typename real>
static snn_status rewire_noalloc_impl(const snn_ragged_desc& d, int32_t* scratch, int32_t* status, uint64_t rewire,
                                      snn_rewire_stats* stats, cudaStream_t s) {
    const int Qw = (d.Q + 31) / 32;
    int32_t* dormant = scratch;
    int32_t* taken = scratch + NOALLOC_MAX_ROWS;
    int32_t* room = scratch + 2 * NOALLOC_MAX_ROWS;
    int32_t* cnt = scratch + 3 * NOALLOC_MAX_ROWS;
    unsigned long long* dsum = (unsigned long long*)(scratch + 4 * NOALLOC_MAX_ROWS + 8);
    if (!status) status = scratch + 4 * NOALLOC_MAX_ROWS;
    return rewire_launch_all<real>(d, Qw, dormant, taken, room, cnt, dsum, status, rewire, nullptr, stats, s);
}

}  // namespace snn

using namespace snn;

extern "C" snn_status snn_rewire_deepr_noalloc(const snn_ragged_desc* d, int64_t rewire_idx, snn_rewire_stats* stats,
                                               int32_t* status, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(d, "snn_rewire_deepr_noalloc: NULL descriptor");
    SNN_REQUIRE(rewire_idx >= 0, "snn_rewire_deepr_noalloc: rewire_idx must be >= 0");
    SNN_REQUIRE(d->P > 0 && d->Q > 0 && d->C > 0, "snn_rewire_deepr_noalloc: P, Q, C must be > 0");
    SNN_REQUIRE(d->P <= NOALLOC_MAX_ROWS,
                "snn_rewire_deepr_noalloc: P = %d rows exceeds the fixed scratch of %d rows "
                "(use snn_create_ragged + snn_rewire_deepr for larger matrices)",
                d->P, NOALLOC_MAX_ROWS);
    SNN_REQUIRE((long long)d->P * d->C < (1ll << 31), "snn_rewire_deepr_noalloc: P*C must be < 2^31");
    SNN_REQUIRE(d->dtype == SNN_F32 || d->dtype == SNN_F64, "snn_rewire_deepr_noalloc: bad dtype");
    SNN_REQUIRE(d->reserved == 0, "snn_rewire_deepr_noalloc: reserved must be 0");
    SNN_REQUIRE(d->row_len && d->ind && d->w && d->m && d->v && d->sign_bits && d->conn_bits,
                "snn_rewire_deepr_noalloc: needs row_len, ind, w, m, v, sign_bits and conn_bits");
    int32_t* scratch = nullptr;
    snn_status st = noalloc_scratch(&scratch);
    if (st != SNN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return d->dtype == SNN_F32 ? rewire_noalloc_impl<float>(*d, scratch, status, (uint64_t)rewire_idx, stats, s)
                               : rewire_noalloc_impl<double>(*d, scratch, status, (uint64_t)rewire_idx, stats, s);
}

extern "C" snn_status snn_rewire_deepr(snn_ragged* r, int64_t rewire_idx, snn_rewire_stats* stats, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r, "snn_rewire_deepr: NULL handle");
    SNN_REQUIRE(rewire_idx >= 0, "snn_rewire_deepr: rewire_idx must be >= 0");
    const snn_ragged_desc& d = r->d;
    SNN_REQUIRE(d.m && d.v && d.sign_bits && d.conn_bits,
                "snn_rewire_deepr: needs Adam moments m, v and the sign / connectivity bitfields");
    cudaStream_t s = (cudaStream_t)stream;
    return d.dtype == SNN_F32 ? rewire_impl<float>(r, (uint64_t)rewire_idx, nullptr, stats, s)
                              : rewire_impl<double>(r, (uint64_t)rewire_idx, nullptr, stats, s);
}

extern "C" snn_status snn_rewire_deepr_dev(snn_ragged* r, const int64_t* rewire_idx_dev, snn_rewire_stats* stats,
                                           snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && rewire_idx_dev, "snn_rewire_deepr_dev: NULL argument");
    const snn_ragged_desc& d = r->d;
    SNN_REQUIRE(d.m && d.v && d.sign_bits && d.conn_bits,
                "snn_rewire_deepr_dev: needs Adam moments m, v and the sign / connectivity bitfields");
    cudaStream_t s = (cudaStream_t)stream;
    const long long* ridx = (const long long*)rewire_idx_dev;
    return d.dtype == SNN_F32 ? rewire_impl<float>(r, 0, ridx, stats, s) : rewire_impl<double>(r, 0, ridx, stats, s);
}

extern "C" snn_status snn_ragged_set_deepr_guide(snn_ragged* r, const snn_deepr_guide* g, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r, "snn_ragged_set_deepr_guide: NULL handle");
    if (!g) {
        r->guide_on = 0;
        return SNN_OK;
    }
    SNN_REQUIRE(g->reserved == 0, "snn_ragged_set_deepr_guide: reserved must be 0");
    SNN_REQUIRE(g->L > 0 && (long long)g->L * g->L < (1ll << 31), "snn_ragged_set_deepr_guide: bad L = %d", g->L);
    SNN_REQUIRE(g->sigma > 0.0, "snn_ragged_set_deepr_guide: sigma must be > 0");
    SNN_REQUIRE(g->pre_site && g->post_site, "snn_ragged_set_deepr_guide: pre_site and post_site are required");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = 2 * (g->L / 2) * (g->L / 2) + 1;
    // weights by squared distance, floor(2^24 exp(-d2 / (2 sigma^2))), on the host in double
    std::vector<uint32_t> q(n);
    for (int d2 = 0; d2 < n; ++d2)
        q[d2] = (uint32_t)(std::exp(-(double)d2 / (2.0 * g->sigma * g->sigma)) * 16777216.0);
    // table plus one word for the site check
    if (r->guide_qcap < n + 1) {
        cudaFree(r->guide_q);
        r->guide_q = nullptr;
        r->guide_qcap = 0;
        if (cudaMalloc(&r->guide_q, (size_t)(n + 1) * sizeof(uint32_t)) != cudaSuccess) {
            set_error("snn_ragged_set_deepr_guide: cudaMalloc failed");
            return SNN_ENOMEM;
        }
        r->guide_qcap = n + 1;
    }
    r->guide_on = 0;
    SNN_CUDA(cudaMemcpyAsync(r->guide_q, q.data(), (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    int32_t* flag = (int32_t*)(r->guide_q + n);
    SNN_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    const int lim = g->L * g->L;
    k_check_sites<<<ceil_div(r->d.P, 256), 256, 0, s>>>(g->pre_site, r->d.P, lim, flag);
    SNN_LAUNCH_CHECK();
    k_check_sites<<<ceil_div(r->d.Q, 256), 256, 0, s>>>(g->post_site, r->d.Q, lim, flag);
    SNN_LAUNCH_CHECK();
    int32_t st = 0;
    SNN_CUDA(cudaMemcpyAsync(&st, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (st != 0) {
        r->guide_on = 0;
        set_error("snn_ragged_set_deepr_guide: a site is outside [0, L*L)");
        return SNN_ESTATE;
    }
    r->guide_on = 1;
    r->guide_L = g->L;
    r->guide_pre = g->pre_site;
    r->guide_post = g->post_site;
    return SNN_OK;
}
