// Shared definitions of the CUDA library: error handling, Philox4x64-10, fixed-point
// accumulators, warp helpers and the library-owned handle structs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/snnsp.h"

namespace snn {

// ------------------------------------------------------------------ error reporting
void set_error(const char* fmt, ...);
void clear_error();

#define SNN_REQUIRE(cond, ...)                                   \
    do {                                                         \
        if (!(cond)) {                                           \
            ::snn::set_error(__VA_ARGS__);                       \
            return SNN_EINVAL;                                   \
        }                                                        \
    } while (0)

#define SNN_CUDA(call)                                                             \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::snn::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                  \
            return SNN_ECUDA;                                                      \
        }                                                                          \
    } while (0)

#define SNN_LAUNCH_CHECK() SNN_CUDA(cudaGetLastError())

// device status word flags (OR-ed by kernels, read by snn_ragged_status)
enum : int32_t {
    ST_CAPACITY = 1,
    ST_STATE = 2,
    ST_TIMEOUT = 4,
};

// ------------------------------------------------------------------ Philox4x64-10
// Salmon et al., SC'11: 10 rounds; each multiplies counter words 0 and 2 by two odd
// constants into 128-bit products, mixes the halves with words 1 and 3 and the key,
// and bumps the key by two Weyl constants.
enum : uint64_t {
    PH_INPUT = 1, PH_SIGN = 2, PH_DEEPR_DIST = 3, PH_DEEPR_FORM = 4, PH_TOPO_ATT = 5,
    PH_TOPO_CAND = 6, PH_TOPO_DRAW = 7, PH_TOPO_FOCUS = 8, PH_TOPO_INPUT = 9, PH_DEEPR_NOISE = 10,
};

struct u64x4 {
    uint64_t x, y, z, w;
    __host__ __device__ uint64_t operator[](int i) const { return i == 0 ? x : i == 1 ? y : i == 2 ? z : w; }
};

__host__ __device__ __forceinline__ void mulhilo64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    lo = (uint64_t)p;
    hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ __forceinline__ u64x4 philox(uint64_t seed, uint64_t purpose, uint64_t c0, uint64_t c1,
                                                 uint64_t c2, uint64_t c3) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t k0 = seed, k1 = purpose;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, hi0, lo0);
        mulhilo64(M1, c2, hi1, lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return {c0, c1, c2, c3};
}

// uniform integer in [0, n): high 64 bits of u * n
__host__ __device__ __forceinline__ uint64_t mulhi_index(uint64_t u, uint64_t n) {
#ifdef __CUDA_ARCH__
    return __umul64hi(u, n);
#else
    return (uint64_t)(((unsigned __int128)u * n) >> 64);
#endif
}

// Bernoulli threshold: word < thr fires.  p * 2^64 scales a double exactly.
inline uint64_t prob_threshold(double p) {
    if (!(p > 0.0)) return 0ull;
    if (p >= 1.0) return ~0ull;
    return (uint64_t)(p * 18446744073709551616.0);
}

// ------------------------------------------------------------------ fixed point
constexpr double FIX_SCALE = 1099511627776.0;       // 2^40
constexpr double FIX_INV = 1.0 / 1099511627776.0;

// float -> int64 with 40 fractional bits using 32-bit integer operations only (GB300's
// FP64 pipe is narrow, so the FP32 path avoids 64-bit float and 64-bit conversions).
// Exact for |w| >= 2^-17; smaller magnitudes round half up; |w| must be < 2^23.
__device__ __forceinline__ long long to_fixed(float w) {
    const unsigned u = __float_as_uint(w);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned m = (u & 0x7fffffu) | 0x800000u;
    const int sh = e - 110;                 // w * 2^40 = m * 2^(e - 110)
    unsigned long long r = 0;
    if (e != 0) {
        if (sh >= 0) r = (unsigned long long)m << (sh < 39 ? sh : 39);
        else if (sh > -25) r = ((unsigned long long)m + (1ull << (-sh - 1))) >> (-sh);
    }
    return (u >> 31) ? -(long long)r : (long long)r;
}
__device__ __forceinline__ long long to_fixed(double w) { return __double2ll_rn(w * FIX_SCALE); }
template <typename real>
__device__ __forceinline__ real from_fixed(long long a);
template <>
__device__ __forceinline__ double from_fixed<double>(long long a) {
    return (double)a * FIX_INV;
}
// int64 (40 fractional bits) -> float from its two 32-bit halves, FP32 operations only
template <>
__device__ __forceinline__ float from_fixed<float>(long long a) {
    const int hi = (int)(a >> 32);
    const unsigned lo = (unsigned)(a & 0xffffffffll);
    return __fmaf_rn((float)hi, 0.00390625f, (float)lo * 9.094947017729282e-13f);
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}
__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    return v;
}

// position (0-based) of the n-th (0-based) set bit of x; x must have > n set bits.  A
// binary search by population counts: keep the low half of the window if it holds the
// bit, else move to the high half; five fixed steps, no data-dependent loop.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t low = x & ((1u << w) - 1u);
        const int c = __popc(low);
        const bool up = n >= c;
        n -= up ? c : 0;
        pos += up ? w : 0;
        x = up ? x >> w : low;
    }
    return pos;
}

__host__ __device__ __forceinline__ int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }

// Multiprocessor count of the current device (cached per device ordinal; 152 on GB300).
int sm_count();

// Adam's beta1^t, beta2^t as running products (beta^t = beta^(t-1) beta from beta^0 = 1),
// advanced from (t0, b1, b2) to t; stops early once both products have underflowed to 0
// (they stay 0).  Host and device run the same multiplications, so the values agree.
struct AdamBias {
    double b1t, b2t, beta1, beta2;
    long long t;
    long long pad;
};
__host__ __device__ __forceinline__ void adam_bias_advance(double beta1, double beta2, long long t0, double& b1,
                                                           double& b2, long long t, long long max_iter) {
    for (long long k = t0, it = 0; k < t && (b1 != 0.0 || b2 != 0.0) && it < max_iter; ++k, ++it) {
        b1 *= beta1;
        b2 *= beta2;
    }
}

}  // namespace snn

// ------------------------------------------------------------------ handles
struct snn_ragged {
    snn_ragged_desc d;
    int32_t Qw;              // words per bitfield row
    int32_t* status;         // device status word (OR of ST_* flags)
    // DEEP R scratch, [P] each
    int32_t* dormant;
    int32_t* taken;
    int32_t* room;
    int32_t* cnt;
    int32_t* scal;           // [4] device scalars: uint64 dormant total, uint64 round-0 rejections
    // topographic rewiring: formation threshold table by squared distance
    uint64_t* thr_form;      // [thr_cap]
    int32_t thr_cap;
    double thr_p, thr_sigma; // parameters the table was built for
    int32_t thr_L;
    // DEEP R sign tags [P*C]: (target | sign bit << 31) per slot, 0xFFFFFFFF = none;
    // only handles with sign bits
    uint32_t* stag;
    // distance-guided DEEP R formation (snn_ragged_set_deepr_guide)
    int32_t guide_on;
    int32_t guide_L;
    const int32_t* guide_pre;    // caller's site arrays
    const int32_t* guide_post;
    uint32_t* guide_q;           // [guide_qcap] weights by squared distance
    int32_t guide_qcap;
};

struct snn_classifier {
    snn_classifier_desc d;
    int32_t fwd_threads;     // row schedule of the forward: threads sharing one trial
    int32_t row_sched;       // SNN_ROWS_PAIRS / SNN_ROWS_PER_WARP / SNN_ROWS_PER_BLOCK
    double alpha, rho;
    int32_t KS;              // K-splits of the e-prop gather
    void* part_in;           // [KS][P_in*C_in] partial gradients
    void* part_rec;          // [KS][N*C_rec]
    void* part_out;          // [KS][N][K]
    void* pk;                // [(n_in + N) * Cf] packed forward rows (refreshed per forward call)
    int32_t* gkeys;          // [P_in*C_in + N*C_rec] gather order: (target << 11) | slot, ascending per row
    int32_t Cf;              // slots per packed row: max(C_in, C_rec + K) rounded up to 32
    unsigned long long* colsum;  // [N + 64] sum of |weight| (fixed point) aimed at each accumulator
    // Adam bias corrections: running products beta^t.  Host copy for calls that pass the
    // step count by value, device copy (snn::AdamBias) for calls that pass it in device
    // memory; each remembers the t and betas it was formed for.
    double h_b1t, h_b2t, h_beta1, h_beta2;
    long long h_t;
    void* adam_dev;
};
