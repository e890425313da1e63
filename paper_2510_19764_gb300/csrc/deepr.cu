// DEEP R rewiring on the ragged matrix with sign and connectivity bitfields
// (Sec. 2.1.2, Fig. 2B-C of the paper).
//
//  k_deepr_eliminate  : one warp per row; a synapse is dormant when its weight's sign is
//                       strictly opposite to its fixed sign bit; survivors are compacted
//                       stably with a warp ballot + prefix count (w, m, v move along),
//                       connectivity bits of removed synapses are cleared.
//  k_deepr_distribute : one CTA; sums the dormant counts on the device and spreads them
//                       over rows in rounds (per-round histogram with integer atomics,
//                       so the result does not depend on thread order).
//  k_deepr_form       : one warp per row with activations; each activation appends the
//                       m-th free target found with a warp popcount scan over the row's
//                       connectivity bitfield.
#include "common.cuh"

#include <mutex>

namespace snn {

template <typename real>
__global__ void k_deepr_eliminate(int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w,
                                  real* __restrict__ m, real* __restrict__ v, const uint32_t* __restrict__ sign,
                                  uint32_t* __restrict__ conn, int32_t* __restrict__ dormant, int P, int C, int Qw) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= P) return;
    const int lane = lane_id();
    const int n = len[i];
    const size_t row = (size_t)i * C;
    int wp = 0;
    for (int base = 0; base < n; base += 32) {
        const int s = base + lane;
        const bool valid = s < n;
        int j = 0;
        real ww = 0, mm = 0, vv = 0;
        bool keep = false;
        if (valid) {
            j = ind[row + s];
            ww = w[row + s];
            mm = m[row + s];
            vv = v[row + s];
            const bool pos = (sign[(size_t)i * Qw + (j >> 5)] >> (j & 31)) & 1u;
            const bool opposite = pos ? (ww < real(0)) : (ww > real(0));
            keep = !opposite;
            if (opposite) atomicAnd(&conn[(size_t)i * Qw + (j >> 5)], ~(1u << (j & 31)));
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
            const int pos = wp + __popc(mask & lanemask_lt());
            ind[row + pos] = j;
            w[row + pos] = ww;
            m[row + pos] = mm;
            v[row + pos] = vv;
        }
        wp += __popc(mask);
        __syncwarp();
    }
    if (lane == 0) {
        len[i] = wp;
        dormant[i] = n - wp;
    }
}

__device__ __forceinline__ long long block_sum_ll(long long x, long long* red) {
    x = warp_sum(x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = x;
    __syncthreads();
    long long s = 0;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(1024)
    k_deepr_distribute(const int32_t* __restrict__ len, const int32_t* __restrict__ dormant, int32_t* __restrict__ room,
                       int32_t* __restrict__ taken, int32_t* __restrict__ cnt, int P, int C, int Q, int no_autapse,
                       uint64_t seed, uint64_t rewire, const long long* ridx_dev, int32_t* status,
                       snn_rewire_stats* stats) {
    __shared__ long long red[32];
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    long long dsum = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int forb = (no_autapse && i < Q) ? 1 : 0;
        const int l = len[i];
        const int r1 = C - l, r2 = Q - forb - l;
        room[i] = r1 < r2 ? r1 : r2;
        taken[i] = 0;
        dsum += dormant[i];
    }
    const long long D = block_sum_ll(dsum, red);
    long long remaining = D;
    for (int r = 0; r < 64 && remaining > 0; ++r) {
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
__global__ void k_deepr_form(int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w,
                             real* __restrict__ m, real* __restrict__ v, uint32_t* __restrict__ conn,
                             const int32_t* __restrict__ taken, int P, int C, int Q, int Qw, int no_autapse,
                             uint64_t seed, uint64_t rewire, const long long* ridx_dev, int32_t* status,
                             snn_rewire_stats* stats) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ridx_dev) rewire = (uint64_t)*ridx_dev;
    if (i >= P) return;
    const int nt = taken[i];
    if (nt == 0) return;
    const int lane = lane_id();
    const int forb = (no_autapse && i < Q) ? 1 : 0;
    const uint32_t tail_mask = (Q & 31) ? ~((1u << (Q & 31)) - 1u) : 0u;   // bits beyond Q in the last word
    uint32_t* crow = conn + (size_t)i * Qw;
    const size_t row = (size_t)i * C;
    int n = len[i];
    int formed = 0;
    for (int k = 0; k < nt; ++k) {
        const int n_free = Q - forb - n;
        if (n_free <= 0 || n >= C) {
            if (lane == 0) atomicOr(status, ST_STATE);
            break;
        }
        const u64x4 u = philox(seed, PH_DEEPR_FORM, rewire, (uint64_t)i, (uint64_t)k, 0);
        const int mth = (int)mulhi_index(u.x, (uint64_t)n_free);
        int target = -1, seen = 0;
        for (int wb = 0; wb < Qw && target < 0; wb += 32) {
            const int wi = wb + lane;
            uint32_t word = 0xffffffffu;
            if (wi < Qw) {
                word = crow[wi];
                if (forb && (i >> 5) == wi) word |= 1u << (i & 31);
                if (wi == Qw - 1) word |= tail_mask;
            }
            const int zeros = __popc(~word);
            const int incl = warp_incl_scan(zeros);
            const int excl = incl - zeros;
            const bool hit = mth >= seen + excl && mth < seen + incl;
            const uint32_t hm = __ballot_sync(0xffffffffu, hit);
            if (hm) {
                const int src = __ffs(hm) - 1;
                int tg = -1;
                if (lane == src) tg = wi * 32 + nth_set_bit(~word, mth - seen - excl);
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

template <typename real>
static snn_status rewire_impl(snn_ragged* r, uint64_t rewire, const long long* ridx_dev, snn_rewire_stats* stats,
                              cudaStream_t s) {
    const snn_ragged_desc& d = r->d;
    const int blocks = ceil_div((long long)d.P * 32, 256);
    k_deepr_eliminate<real><<<blocks, 256, 0, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v,
                                                    d.sign_bits, d.conn_bits, r->dormant, d.P, d.C, r->Qw);
    SNN_LAUNCH_CHECK();
    k_deepr_distribute<<<1, 1024, 0, s>>>(d.row_len, r->dormant, r->room, r->taken, r->cnt, d.P, d.C, d.Q,
                                          d.no_autapse, d.seed, rewire, ridx_dev, r->status, stats);
    SNN_LAUNCH_CHECK();
    k_deepr_form<real><<<blocks, 256, 0, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v, d.conn_bits,
                                               r->taken, d.P, d.C, d.Q, r->Qw, d.no_autapse, d.seed, rewire,
                                               ridx_dev, r->status, stats);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

// ------------------------------------------------------------------ no-allocation variant
// Fixed scratch for snn_rewire_deepr_noalloc: four int32 arrays of NOALLOC_MAX_ROWS rows
// (dormant counts, taken, room, per-round histogram) and one status word.  It lives in
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
    if (!status) status = scratch + 4 * NOALLOC_MAX_ROWS;
    const int blocks = ceil_div((long long)d.P * 32, 256);
    k_deepr_eliminate<real><<<blocks, 256, 0, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v,
                                                    d.sign_bits, d.conn_bits, dormant, d.P, d.C, Qw);
    SNN_LAUNCH_CHECK();
    k_deepr_distribute<<<1, 1024, 0, s>>>(d.row_len, dormant, room, taken, cnt, d.P, d.C, d.Q, d.no_autapse, d.seed,
                                          rewire, nullptr, status, stats);
    SNN_LAUNCH_CHECK();
    k_deepr_form<real><<<blocks, 256, 0, s>>>(d.row_len, d.ind, (real*)d.w, (real*)d.m, (real*)d.v, d.conn_bits,
                                               taken, d.P, d.C, d.Q, Qw, d.no_autapse, d.seed, rewire, nullptr, status,
                                               stats);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
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
