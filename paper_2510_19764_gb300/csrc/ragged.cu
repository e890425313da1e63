// Ragged sparse matrix handle (Sec. 2.1, Fig. 1), DEEP R bitfield initialisation
// (Sec. 2.1.2, Fig. 2A), spike propagation (Fig. 1) and the library's error state.
#include "common.cuh"

#include <cstdlib>
#include <cstring>

namespace snn {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }

int sm_count() {
    static int cached[256] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 152;
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

// ------------------------------------------------------------------ validation
// One warp per row: row length range, target range, self targets, duplicate targets.
__global__ void k_validate(const int32_t* __restrict__ row_len, const int32_t* __restrict__ ind, int P, int Q,
                           int C, int no_autapse, int32_t* status) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= P) return;
    int i = warp;
    int len = row_len[i];
    if (len < 0 || len > C) {
        if (lane_id() == 0) atomicOr(status, ST_STATE);
        return;
    }
    const int32_t* row = ind + (size_t)i * C;
    bool bad = false;
    for (int s = lane_id(); s < len; s += 32) {
        int j = row[s];
        if (j < 0 || j >= Q || (no_autapse && j == i)) bad = true;
        for (int s2 = 0; s2 < s; ++s2)
            if (row[s2] == j) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(status, ST_STATE);
}

__global__ void k_sign_random(uint32_t* sign, uint32_t* conn, int P, int Qw, uint64_t seed) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)P * Qw) return;
    int i = (int)(k / Qw), w = (int)(k % Qw);
    u64x4 r = philox(seed, PH_SIGN, (uint64_t)i, (uint64_t)w, 0, 0);
    sign[k] = (uint32_t)(r.x & 0xffffffffull);
    conn[k] = 0u;
}

template <typename real>
__global__ void k_sign_from_weights(const int32_t* __restrict__ row_len, const int32_t* __restrict__ ind,
                                    const real* __restrict__ w, uint32_t* sign, uint32_t* conn, int P, int C,
                                    int Qw) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= P) return;
    int i = warp;
    int len = row_len[i];
    for (int s = lane_id(); s < len; s += 32) {
        int j = ind[(size_t)i * C + s];
        real ws = w[(size_t)i * C + s];
        size_t word = (size_t)i * Qw + (j >> 5);
        uint32_t bit = 1u << (j & 31);
        atomicOr(&conn[word], bit);
        if (ws > real(0)) atomicOr(&sign[word], bit);
        else if (ws < real(0)) atomicAnd(&sign[word], ~bit);
    }
}

// ------------------------------------------------------------------ row updates
// One warp per row with an edit (targets[i] >= 0).  Add: skip a target already in the
// row (connectivity bit when the handle has bitfields, else a ballot over the row) or a
// full row, else append at slot row_len with the given weight and zero optimiser state.
// Remove: find the target's slot, move the later slots down one (every lane of a chunk
// reads before any writes), clear the bit.  Counts go to stats (formed / removed /
// overflow for skipped adds).
template <typename real>
__global__ void k_row_edit(int remove, int32_t* __restrict__ len, int32_t* __restrict__ ind, real* __restrict__ w,
                           real* __restrict__ m, real* __restrict__ v, real* __restrict__ grad,
                           uint32_t* __restrict__ conn, const int32_t* __restrict__ targets,
                           const real* __restrict__ w_new, int P, int Q, int C, int Qw, int no_autapse,
                           int32_t* status, snn_rewire_stats* stats) {
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= P) return;
    const int t = targets[i];
    if (t < 0) return;
    const int lane = lane_id();
    if (t >= Q || (no_autapse && t == i)) {
        if (lane == 0) {
            atomicOr(status, ST_STATE);
            if (stats && !remove) atomicAdd((unsigned long long*)&stats->overflow, 1ull);
        }
        return;
    }
    const int n = len[i];
    const size_t row = (size_t)i * C;
    int found = -1;                                  // slot of t in the row, or -1
    if (remove || !conn) {
        for (int b0 = 0; b0 < n && found < 0; b0 += 32) {
            const int s = b0 + lane;
            const uint32_t hm = __ballot_sync(0xffffffffu, s < n && ind[row + s] == t);
            if (hm) found = b0 + __ffs(hm) - 1;
        }
    } else {
        found = ((conn[(size_t)i * Qw + (t >> 5)] >> (t & 31)) & 1u) ? 0 : -1;
    }
    if (!remove) {
        if (lane == 0) {
            if (found >= 0 || n >= C) {
                if (stats) atomicAdd((unsigned long long*)&stats->overflow, 1ull);
            } else {
                ind[row + n] = t;
                w[row + n] = w_new ? w_new[i] : real(0);
                if (m) m[row + n] = real(0);
                if (v) v[row + n] = real(0);
                if (grad) grad[row + n] = real(0);
                if (conn) conn[(size_t)i * Qw + (t >> 5)] |= 1u << (t & 31);
                len[i] = n + 1;
                if (stats) atomicAdd((unsigned long long*)&stats->formed, 1ull);
            }
        }
        return;
    }
    if (found < 0) return;
    for (int b0 = found + 1; b0 < n; b0 += 32) {
        const int s = b0 + lane;
        const bool ok = s < n;
        int j = 0;
        real ww = 0, mm = 0, vv = 0, gg = 0;
        if (ok) {
            j = ind[row + s];
            ww = w[row + s];
            if (m) mm = m[row + s];
            if (v) vv = v[row + s];
            if (grad) gg = grad[row + s];
        }
        __syncwarp();
        if (ok) {
            ind[row + s - 1] = j;
            w[row + s - 1] = ww;
            if (m) m[row + s - 1] = mm;
            if (v) v[row + s - 1] = vv;
            if (grad) grad[row + s - 1] = gg;
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (conn) conn[(size_t)i * Qw + (t >> 5)] &= ~(1u << (t & 31));
        len[i] = n - 1;
        if (stats) atomicAdd((unsigned long long*)&stats->removed, 1ull);
    }
}

// ------------------------------------------------------------------ propagation
// Grid (word blocks, B).  A warp owns one 32-row word of the presynaptic spike bits of
// instance b and walks its set bits; lanes stride the row's slots and add the weight
// to the target's fixed-point accumulator (order-independent sums).
template <typename real>
__global__ void k_propagate(const int32_t* __restrict__ row_len, const int32_t* __restrict__ ind,
                            const real* __restrict__ w, const uint32_t* __restrict__ pre_bits, int P, int Pw,
                            int Q, int C, long long* __restrict__ acc) {
    int word = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int b = blockIdx.y;
    if (word >= Pw) return;
    uint32_t bits = pre_bits[(size_t)b * Pw + word];
    unsigned long long* a = (unsigned long long*)(acc + (size_t)b * Q);
    while (bits) {
        int i = word * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        if (i >= P) break;
        int len = row_len[i];
        const int32_t* ri = ind + (size_t)i * C;
        const real* rw = w + (size_t)i * C;
        // four 32-slot chunks per iteration: their loads are issued before the adds
        for (int s0 = 0; s0 < len; s0 += 128) {
            int j[4];
            real x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = s0 + 32 * q + lane_id();
                j[q] = s < len ? ri[s] : -1;
                x[q] = s < len ? rw[s] : real(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j[q] >= 0) atomicAdd(a + j[q], (unsigned long long)to_fixed(x[q]));
        }
    }
}

__global__ void k_philox(uint64_t seed, uint64_t purpose, const uint64_t* ctr, long long n, uint64_t* out) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    u64x4 r = philox(seed, purpose, ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2], ctr[4 * k + 3]);
    out[4 * k] = r.x;
    out[4 * k + 1] = r.y;
    out[4 * k + 2] = r.z;
    out[4 * k + 3] = r.w;
}

}  // namespace snn

using namespace snn;

extern "C" {

const char* snn_last_error(void) { return g_last_error.c_str(); }
int32_t snn_abi_version(void) { return 8; }

snn_status snn_create_ragged(const snn_ragged_desc* d, int32_t init_bits, snn_stream stream, snn_ragged** out) {
    clear_error();
    SNN_REQUIRE(d && out, "snn_create_ragged: NULL argument");
    *out = nullptr;
    SNN_REQUIRE(d->P > 0 && d->Q > 0 && d->C > 0, "snn_create_ragged: P, Q, C must be > 0 (got %d, %d, %d)", d->P,
                d->Q, d->C);
    SNN_REQUIRE((long long)d->P * d->C < (1ll << 31), "snn_create_ragged: P*C must be < 2^31");
    SNN_REQUIRE(d->dtype == SNN_F32 || d->dtype == SNN_F64, "snn_create_ragged: dtype must be SNN_F32 or SNN_F64");
    SNN_REQUIRE(d->reserved == 0, "snn_create_ragged: reserved must be 0");
    SNN_REQUIRE(d->row_len && d->ind && d->w, "snn_create_ragged: row_len, ind and w are required");
    SNN_REQUIRE(!init_bits || (d->sign_bits && d->conn_bits),
                "snn_create_ragged: init_deepr_bitfields needs sign_bits and conn_bits");
    cudaStream_t s = (cudaStream_t)stream;
    snn_ragged* r = (snn_ragged*)calloc(1, sizeof(snn_ragged));
    if (!r) {
        set_error("snn_create_ragged: out of host memory");
        return SNN_ENOMEM;
    }
    r->d = *d;
    r->Qw = (d->Q + 31) / 32;
    r->thr_cap = d->Q / 2 + 2;
    r->thr_L = -1;
    size_t P = (size_t)d->P;
    cudaError_t e = cudaSuccess;
    e = e != cudaSuccess ? e : cudaMalloc(&r->status, sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->dormant, P * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->taken, P * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->room, P * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->cnt, P * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->scal, 4 * sizeof(int32_t));
    e = e != cudaSuccess ? e : cudaMalloc(&r->thr_form, (size_t)r->thr_cap * sizeof(uint64_t));
    if (d->sign_bits) e = e != cudaSuccess ? e : cudaMalloc(&r->stag, P * (size_t)d->C * sizeof(uint32_t));
    if (e != cudaSuccess) {
        snn_destroy_ragged(r);
        set_error("snn_create_ragged: cudaMalloc failed: %s", cudaGetErrorString(e));
        return SNN_ENOMEM;
    }
    SNN_CUDA(cudaMemsetAsync(r->status, 0, sizeof(int32_t), s));
    if (r->stag) SNN_CUDA(cudaMemsetAsync(r->stag, 0xFF, P * (size_t)d->C * sizeof(uint32_t), s));   // no tags yet
    int threads = 256;
    int blocks = ceil_div((long long)d->P * 32, threads);
    k_validate<<<blocks, threads, 0, s>>>(d->row_len, d->ind, d->P, d->Q, d->C, d->no_autapse, r->status);
    SNN_LAUNCH_CHECK();
    if (init_bits) {
        long long nw = (long long)d->P * r->Qw;
        k_sign_random<<<ceil_div(nw, 256), 256, 0, s>>>(d->sign_bits, d->conn_bits, d->P, r->Qw, d->seed);
        SNN_LAUNCH_CHECK();
        if (d->dtype == SNN_F32)
            k_sign_from_weights<float><<<blocks, threads, 0, s>>>(d->row_len, d->ind, (const float*)d->w,
                                                                  d->sign_bits, d->conn_bits, d->P, d->C, r->Qw);
        else
            k_sign_from_weights<double><<<blocks, threads, 0, s>>>(d->row_len, d->ind, (const double*)d->w,
                                                                   d->sign_bits, d->conn_bits, d->P, d->C, r->Qw);
        SNN_LAUNCH_CHECK();
    }
    int32_t st = 0;
    SNN_CUDA(cudaMemcpyAsync(&st, r->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (st != 0) {
        snn_destroy_ragged(r);
        set_error("snn_create_ragged: invalid contents (row_len > C, target out of range, duplicate or self target)");
        return SNN_ESTATE;
    }
    *out = r;
    return SNN_OK;
}

snn_status snn_destroy_ragged(snn_ragged* r) {
    if (!r) return SNN_OK;
    cudaFree(r->guide_q);
    cudaFree(r->stag);
    cudaFree(r->status);
    cudaFree(r->dormant);
    cudaFree(r->taken);
    cudaFree(r->room);
    cudaFree(r->cnt);
    cudaFree(r->scal);
    cudaFree(r->thr_form);
    free(r);
    return SNN_OK;
}

snn_status snn_ragged_status(snn_ragged* r, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r, "snn_ragged_status: NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t st = 0;
    SNN_CUDA(cudaMemcpyAsync(&st, r->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemsetAsync(r->status, 0, sizeof(int32_t), s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (st & ST_STATE) {
        set_error("device reported an invariant violation (bad index or row)");
        return SNN_ESTATE;
    }
    if (st & ST_TIMEOUT) {
        set_error("a bounded device-side wait gave up");
        return SNN_ETIMEOUT;
    }
    if (st & ST_CAPACITY) {
        set_error("a row ran out of capacity or activations were left over");
        return SNN_ECAPACITY;
    }
    return SNN_OK;
}

static snn_status row_edit(snn_ragged* r, int remove, const int32_t* targets, const void* w_new,
                           snn_rewire_stats* stats, snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && targets, "snn_ragged_%s_row: NULL argument", remove ? "remove" : "add");
    const snn_ragged_desc& d = r->d;
    const int threads = 256;
    const int blocks = ceil_div((long long)d.P * 32, threads);
    cudaStream_t s = (cudaStream_t)stream;
    if (d.dtype == SNN_F32)
        k_row_edit<float><<<blocks, threads, 0, s>>>(remove, d.row_len, d.ind, (float*)d.w, (float*)d.m, (float*)d.v,
                                                     (float*)d.grad, d.conn_bits, targets, (const float*)w_new, d.P,
                                                     d.Q, d.C, r->Qw, d.no_autapse, r->status, stats);
    else
        k_row_edit<double><<<blocks, threads, 0, s>>>(remove, d.row_len, d.ind, (double*)d.w, (double*)d.m,
                                                      (double*)d.v, (double*)d.grad, d.conn_bits, targets,
                                                      (const double*)w_new, d.P, d.Q, d.C, r->Qw, d.no_autapse,
                                                      r->status, stats);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_ragged_add_row(snn_ragged* r, const int32_t* targets, const void* w_new, snn_rewire_stats* stats,
                              snn_stream stream) {
    return row_edit(r, 0, targets, w_new, stats, stream);
}

snn_status snn_ragged_remove_row(snn_ragged* r, const int32_t* targets, snn_rewire_stats* stats, snn_stream stream) {
    return row_edit(r, 1, targets, nullptr, stats, stream);
}

snn_status snn_propagate(const snn_ragged* r, const uint32_t* pre_bits, int32_t B, int64_t* post_acc,
                         snn_stream stream) {
    clear_error();
    SNN_REQUIRE(r && pre_bits && post_acc, "snn_propagate: NULL argument");
    SNN_REQUIRE(B > 0, "snn_propagate: B must be > 0");
    const snn_ragged_desc& d = r->d;
    int Pw = (d.P + 31) / 32;
    int warps = 8;
    dim3 grid(ceil_div(Pw, warps), B);
    cudaStream_t s = (cudaStream_t)stream;
    if (d.dtype == SNN_F32)
        k_propagate<float><<<grid, warps * 32, 0, s>>>(d.row_len, d.ind, (const float*)d.w, pre_bits, d.P, Pw, d.Q,
                                                        d.C, (long long*)post_acc);
    else
        k_propagate<double><<<grid, warps * 32, 0, s>>>(d.row_len, d.ind, (const double*)d.w, pre_bits, d.P, Pw,
                                                         d.Q, d.C, (long long*)post_acc);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

snn_status snn_philox(uint64_t seed, uint64_t purpose, const uint64_t* ctr, int64_t n, uint64_t* out,
                      snn_stream stream) {
    clear_error();
    SNN_REQUIRE(ctr && out && n >= 0, "snn_philox: bad argument");
    if (n == 0) return SNN_OK;
    k_philox<<<ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(seed, purpose, ctr, n, out);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // extern "C"
