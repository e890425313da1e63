// Target-tiled spike propagation (Fig. 1's operation: for every spiking row, add its
// weights to its targets' inputs), regrouped so that the additions land in shared
// memory instead of global atomics.
//
// The ragged matrix is row-major and its rows are unsorted, so a projection's targets
// are scattered over the whole postsynaptic range.  The plan keeps a second copy of the
// synapses grouped by target tile (W consecutive targets): tile k holds an entry
// (i << 12 | j - kW, w_ij) for every synapse i -> j with kW <= j < (k+1)W, in row-block
// order.  A propagation CTA owns one tile and one group of up to 16 instances: it reads
// its tile's entries once for all of them (the weights are shared by the instances),
// looks up which instances spiked the entry's row in a per-row 16-bit mask, and adds the
// weight to those instances' accumulators in shared memory.  The accumulators are exact
// 64-bit integers (40 fractional bits, as snn_propagate's): the low word is added with an
// atomic that returns the old value, the high word with the high half plus the carry out
// of the low word.  Whatever the order of the additions, the low word ends as the sum of
// the low halves modulo 2^32 and the high word gains one carry per wrap of it, so the
// pair holds the sum modulo 2^64, the value global int64 atomics give.  Each CTA then
// adds its tile into post_acc once, with plain loads and stores (no other CTA touches
// those words).
//
// Building the tiles (snn_prop_plan_pack) is a counting sort by tile: per row block a
// histogram of tiles, an exclusive scan of the counts in (tile, row block) order, then
// a scatter that places each row block's synapses in its reserved range of every tile.
#include "common.cuh"

namespace snn {

constexpr int PLAN_RB = 64;          // rows per row block of the counting sort
constexpr int PLAN_IG = 16;          // instances per propagation CTA (one 16-bit mask per row)
constexpr int PLAN_LT_BITS = 12;     // local target bits of an entry key (W <= 4096)
constexpr int PLAN_THREADS = 512;
constexpr int PLAN_U = 8;            // entries a propagation thread has in flight

// A row's length, or -1 when it is outside [0, C] (the row is skipped and flagged).
__device__ __forceinline__ int plan_row_len(const int32_t* row_len, int i, int C) {
    const int n = row_len[i];
    return (n < 0 || n > C) ? -1 : n;
}

// Pass 1: tile histogram of one row block (warp per row), written as cnt[tile][rb].
__global__ void k_plan_count(const int32_t* __restrict__ row_len, const int32_t* __restrict__ ind, int P, int Q,
                             int C, int W, int ntiles, int nrb, int32_t* __restrict__ cnt, int32_t* status) {
    extern __shared__ int hist[];
    const int rb = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    bool bad = false;
    for (int i = rb * PLAN_RB + warp; i < min(P, (rb + 1) * PLAN_RB); i += nw) {
        const int n = plan_row_len(row_len, i, C);
        bad |= n < 0;
        for (int s = lane; s < n; s += 32) {
            const int j = ind[(size_t)i * C + s];
            if (j < 0 || j >= Q) {
                bad = true;
                continue;
            }
            atomicAdd(&hist[j / W], 1);
        }
    }
    if (bad) atomicOr(status, ST_STATE);
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) cnt[(size_t)t * nrb + rb] = hist[t];
}

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple of 32, <= 1024);
// returns the thread's exclusive prefix, total in *total.  ws: 32 ints of shared memory.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* ws, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const long long before = warp > 0 ? ws[warp - 1] : 0;
    *total = ws[nw - 1];
    __syncthreads();
    return before + x - v;
}

// Pass 2 (CTA per tile): the tile's row-block counts become offsets within the tile;
// the tile's total goes to tile_base[t + 1].
__global__ void k_plan_scan_tile(int32_t* __restrict__ cnt, int nrb, int32_t* __restrict__ tile_base) {
    __shared__ long long ws[32];
    int32_t* c = cnt + (size_t)blockIdx.x * nrb;
    long long carry = 0;
    for (int b0 = 0; b0 < nrb; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        const long long v = k < nrb ? c[k] : 0;
        long long total;
        const long long ex = block_excl_scan(v, ws, &total);
        if (k < nrb) c[k] = (int32_t)(carry + ex);
        carry += total;
    }
    if (threadIdx.x == 0) tile_base[blockIdx.x + 1] = (int32_t)carry;
}

// Pass 3 (one CTA): tile totals -> tile starts (exclusive scan in place, tile_base[0] = 0).
__global__ void k_plan_scan_base(int32_t* __restrict__ tile_base, int ntiles) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        const long long v = k < ntiles ? tile_base[k + 1] : 0;
        long long total;
        const long long ex = block_excl_scan(v, ws, &total);
        __syncthreads();
        if (k < ntiles) tile_base[k + 1] = (int32_t)(carry + ex + v);
        carry += total;
    }
    if (threadIdx.x == 0) tile_base[0] = 0;
}

// Pass 4: each row block places its synapses in its reserved range of every tile (the
// same skips as pass 1, so the counts match), weights converted to fixed point.
template <typename real>
__global__ void k_plan_scatter(const int32_t* __restrict__ row_len, const int32_t* __restrict__ ind,
                               const real* __restrict__ w, int P, int Q, int C, int W, int ntiles, int nrb,
                               const int32_t* __restrict__ cnt, const int32_t* __restrict__ tile_base,
                               uint32_t* __restrict__ keys, long long* __restrict__ fx) {
    extern __shared__ int pos[];
    const int rb = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) pos[t] = tile_base[t] + cnt[(size_t)t * nrb + rb];
    __syncthreads();
    for (int i = rb * PLAN_RB + warp; i < min(P, (rb + 1) * PLAN_RB); i += nw) {
        const int n = plan_row_len(row_len, i, C);
        for (int s = lane; s < n; s += 32) {
            const size_t g = (size_t)i * C + s;
            const int j = ind[g];
            if (j < 0 || j >= Q) continue;
            const int t = j / W;
            const int e = atomicAdd(&pos[t], 1);
            keys[e] = ((uint32_t)i << PLAN_LT_BITS) | (uint32_t)(j - t * W);
            fx[e] = to_fixed(w[g]);
        }
    }
}

// Per call: mask[g][i] bit q = row i spiked in instance 16 g + q.  Thread = (group, row);
// the 32 threads of a warp share each instance's spike word.
__global__ void k_plan_rowmask(const uint32_t* __restrict__ pre_bits, int B, int P, int Pw,
                               uint16_t* __restrict__ mask) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int groups = (B + PLAN_IG - 1) / PLAN_IG;
    if (k >= (long long)groups * P) return;
    const int g = (int)(k / P), i = (int)(k % P);
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < PLAN_IG; ++q) {
        const int b = g * PLAN_IG + q;
        if (b < B) v |= ((pre_bits[(size_t)b * Pw + (i >> 5)] >> (i & 31)) & 1u) << q;
    }
    mask[k] = (uint16_t)v;
}

// Exact 64-bit accumulation in shared memory from 32-bit atomics (see the file comment):
// low word at lo, high word at lo + n_acc.  The low and high words are separate arrays so
// that lanes adding to consecutive accumulators hit consecutive banks.
__device__ __forceinline__ void acc64_add(uint32_t* lo_w, int n_acc, unsigned long long x) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const uint32_t old = atomicAdd(lo_w, lo);
    atomicAdd(lo_w + n_acc, hi + (old + lo < lo ? 1u : 0u));
}

// One CTA per (tile, instance group): accumulator q * W + lt for instance q < IG of the
// group and local target lt < W.
__global__ void __launch_bounds__(PLAN_THREADS)
    k_propagate_tiled(const uint32_t* __restrict__ keys, const long long* __restrict__ fx,
                      const int32_t* __restrict__ tile_base, const uint16_t* __restrict__ mask, int P, int Q,
                      int W, int IG, int B, long long* __restrict__ post_acc) {
    extern __shared__ __align__(16) uint32_t accs[];
    const int tile = blockIdx.x, g = blockIdx.y;
    const int e0 = tile_base[tile], e1 = tile_base[tile + 1];
    if (e0 == e1) return;   // no synapse aims at this tile: nothing to add
    const int n_acc = IG * W;
    for (int k = threadIdx.x; k < 2 * n_acc; k += blockDim.x) accs[k] = 0u;
    __syncthreads();
    const uint16_t* mg = mask + (size_t)g * P;
    // PLAN_U entries per thread in flight: their keys and weights are loaded together,
    // then their masks, then the additions
    const int stride = blockDim.x * PLAN_U;
    for (int e = e0 + threadIdx.x; e < e1; e += stride) {
        uint32_t key[PLAN_U];
        long long xv[PLAN_U];
#pragma unroll
        for (int u = 0; u < PLAN_U; ++u) {
            const int eu = e + u * blockDim.x;
            key[u] = eu < e1 ? keys[eu] : 0u;
            xv[u] = eu < e1 ? fx[eu] : 0ll;
        }
        uint32_t m[PLAN_U];
#pragma unroll
        for (int u = 0; u < PLAN_U; ++u) m[u] = e + u * blockDim.x < e1 ? mg[key[u] >> PLAN_LT_BITS] : 0u;
#pragma unroll
        for (int u = 0; u < PLAN_U; ++u) {
            uint32_t* a = accs + (key[u] & ((1u << PLAN_LT_BITS) - 1u));
            for (uint32_t mm = m[u]; mm; mm &= mm - 1u)
                acc64_add(a + W * (__ffs(mm) - 1), n_acc, (unsigned long long)xv[u]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
        const int q = k / W, lt = k - q * W;
        const int b = g * PLAN_IG + q, j = tile * W + lt;
        if (b < B && j < Q) {
            const unsigned long long v = ((unsigned long long)accs[n_acc + k] << 32) | accs[k];
            if (v) post_acc[(size_t)b * Q + j] += (long long)v;
        }
    }
}

}  // namespace snn

struct snn_prop_plan {
    snn_ragged* r;
    int32_t W, ntiles, nrb, IG, max_B;
    uint32_t* keys;        // [P*C] entry keys, grouped by tile
    long long* fx;         // [P*C] entry weights, fixed point (SNN_FIXED_FRAC_BITS)
    int32_t* cnt;          // [ntiles][nrb] row-block counts, then offsets within the tile
    int32_t* tile_base;    // [ntiles + 1] first entry of each tile
    uint16_t* mask;        // [ceil(max_B / 16)][P] per-row instance masks
};

using namespace snn;

extern "C" {

snn_status snn_destroy_prop_plan(snn_prop_plan* p) {
    if (!p) return SNN_OK;
    cudaFree(p->keys);
    cudaFree(p->fx);
    cudaFree(p->cnt);
    cudaFree(p->tile_base);
    cudaFree(p->mask);
    delete p;
    return SNN_OK;
}

snn_status snn_create_prop_plan(snn_ragged* r, int32_t max_B, snn_prop_plan** out) {
    clear_error();
    SNN_REQUIRE(r && out, "snn_create_prop_plan: NULL argument");
    *out = nullptr;
    const snn_ragged_desc& d = r->d;
    SNN_REQUIRE(max_B > 0, "snn_create_prop_plan: max_B must be > 0");
    SNN_REQUIRE(d.P <= (1 << (32 - PLAN_LT_BITS)), "snn_create_prop_plan: P = %d > 2^20", d.P);
    snn_prop_plan* p = new (std::nothrow) snn_prop_plan();
    if (!p) {
        set_error("snn_create_prop_plan: out of host memory");
        return SNN_ENOMEM;
    }
    p->r = r;
    p->max_B = max_B;
    p->IG = max_B < PLAN_IG ? max_B : PLAN_IG;
    // about two tiles per SM, 32 to 1024 targets each
    int W = (int)ceil_div(d.Q, 2 * sm_count());
    W = W < 32 ? 32 : (W > 1024 ? 1024 : W);
    p->W = W;
    p->ntiles = (int)ceil_div(d.Q, W);
    p->nrb = (int)ceil_div(d.P, PLAN_RB);
    const size_t n = (size_t)d.P * d.C;
    const int groups = (int)ceil_div(max_B, PLAN_IG);
    cudaError_t e = cudaSuccess;
    e = e != cudaSuccess ? e : cudaMalloc(&p->keys, n * sizeof(uint32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&p->fx, n * sizeof(long long));
    e = e != cudaSuccess ? e : cudaMalloc(&p->cnt, (size_t)p->ntiles * p->nrb * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&p->tile_base, (size_t)(p->ntiles + 1) * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&p->mask, (size_t)groups * d.P * sizeof(uint16_t));
    // an unpacked plan holds no entries
    e = e != cudaSuccess ? e : cudaMemset(p->tile_base, 0, (size_t)(p->ntiles + 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        snn_destroy_prop_plan(p);
        set_error("snn_create_prop_plan: %s", cudaGetErrorString(e));
        return SNN_ENOMEM;
    }
    const int hist = p->ntiles * (int)sizeof(int);
    SNN_REQUIRE(hist <= 227 * 1024, "snn_create_prop_plan: %d tiles is too many", p->ntiles);
    if (hist > 48 * 1024) {
        SNN_CUDA(cudaFuncSetAttribute(k_plan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, hist));
        SNN_CUDA(cudaFuncSetAttribute(k_plan_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, hist));
        SNN_CUDA(cudaFuncSetAttribute(k_plan_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, hist));
    }
    const int accb = 8 * p->IG * W;
    if (accb > 48 * 1024) {
        SNN_CUDA(cudaFuncSetAttribute(k_propagate_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, accb));
    }
    *out = p;
    return SNN_OK;
}

snn_status snn_prop_plan_pack(snn_prop_plan* p, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(p, "snn_prop_plan_pack: NULL plan");
    const snn_ragged_desc& d = p->r->d;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t hist = (size_t)p->ntiles * sizeof(int);
    k_plan_count<<<p->nrb, 256, hist, s>>>(d.row_len, d.ind, d.P, d.Q, d.C, p->W, p->ntiles, p->nrb, p->cnt,
                                            p->r->status);
    SNN_LAUNCH_CHECK();
    k_plan_scan_tile<<<p->ntiles, 1024, 0, s>>>(p->cnt, p->nrb, p->tile_base);
    SNN_LAUNCH_CHECK();
    k_plan_scan_base<<<1, 1024, 0, s>>>(p->tile_base, p->ntiles);
    SNN_LAUNCH_CHECK();
    if (d.dtype == SNN_F32)
        k_plan_scatter<float><<<p->nrb, 256, hist, s>>>(d.row_len, d.ind, (const float*)d.w, d.P, d.Q, d.C, p->W,
                                                        p->ntiles, p->nrb, p->cnt, p->tile_base, p->keys,
                                                        p->fx);
    else
        k_plan_scatter<double><<<p->nrb, 256, hist, s>>>(d.row_len, d.ind, (const double*)d.w, d.P, d.Q, d.C, p->W,
                                                         p->ntiles, p->nrb, p->cnt, p->tile_base, p->keys,
                                                         p->fx);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_propagate_tiled(const snn_prop_plan* p, const uint32_t* pre_bits, int32_t B, int64_t* post_acc,
                               snn_stream stream) {
    clear_error();
    SNN_REQUIRE(p && pre_bits && post_acc, "snn_propagate_tiled: NULL argument");
    SNN_REQUIRE(B > 0 && B <= p->max_B, "snn_propagate_tiled: B = %d outside [1, %d]", B, p->max_B);
    const snn_ragged_desc& d = p->r->d;
    cudaStream_t s = (cudaStream_t)stream;
    const int Pw = (d.P + 31) / 32;
    const int groups = (int)ceil_div(B, PLAN_IG);
    k_plan_rowmask<<<(int)ceil_div((long long)groups * d.P, 256), 256, 0, s>>>(pre_bits, B, d.P, Pw, p->mask);
    SNN_LAUNCH_CHECK();
    const dim3 grid(p->ntiles, groups);
    const size_t accb = (size_t)8 * p->IG * p->W;
    k_propagate_tiled<<<grid, PLAN_THREADS, accb, s>>>(p->keys, p->fx, p->tile_base, p->mask, d.P, d.Q, p->W,
                                                       p->IG, B, (long long*)post_acc);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // extern "C"
