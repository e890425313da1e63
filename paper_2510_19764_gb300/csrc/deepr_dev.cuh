// Device code of DEEP R rewiring (Sec. 2.1.2, Fig. 2B-C of the paper) shared by the
// per-call kernels (deepr.cu) and the persistent multi-instance kernel (multi.cu).
#pragma once

#include "common.cuh"

namespace snn {

// Sign tags: tag[slot] = (target | sign bit << 31) cached for the target the slot held
// when the tag was written.  A tag whose target differs from the slot's current target
// is stale and the sign bitfield is read instead; since a potential connection's sign
// bit never changes, a tag with the right target is always right.  0xFFFFFFFF never
// matches (targets are < 2^31 - 1).  With tags the elimination reads 20 bytes per slot
// in one round trip instead of a bitfield sector per synapse in a second one.
//
// One warp per row, ELIM_CH chunks of 32 slots at a time: every load of the batch is
// issued together, then the sign words of tag misses, then the stable compaction.
constexpr int ELIM_CH = 2;

template <typename real>
__device__ __forceinline__ void eliminate_row(int32_t* __restrict__ len, int32_t* __restrict__ ind,
                                              real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                                              const uint32_t* __restrict__ sign, uint32_t* __restrict__ conn,
                                              uint32_t* __restrict__ tag, int32_t* __restrict__ dormant,
                                              int32_t* __restrict__ cnt, int i, int C, int Qw) {
    const int lane = lane_id();
    const int n = len[i];
    const size_t row = (size_t)i * C;
    int wp = 0;
    for (int b0 = 0; b0 < n; b0 += 32 * ELIM_CH) {
        int j[ELIM_CH];
        real ww[ELIM_CH], mm[ELIM_CH], vv[ELIM_CH];
        uint32_t tg[ELIM_CH];
#pragma unroll
        for (int c = 0; c < ELIM_CH; ++c) {
            const int s = b0 + 32 * c + lane;
            j[c] = -1;
            ww[c] = mm[c] = vv[c] = real(0);
            tg[c] = 0xFFFFFFFFu;
            if (s < n) {
                j[c] = ind[row + s];
                ww[c] = w[row + s];
                mm[c] = m[row + s];
                vv[c] = v[row + s];
                if (tag) tg[c] = tag[row + s];
            }
        }
        bool pos[ELIM_CH], hit[ELIM_CH];
#pragma unroll
        for (int c = 0; c < ELIM_CH; ++c) {
            const int jc = j[c];
            hit[c] = jc >= 0 && (int)(tg[c] & 0x7FFFFFFFu) == jc;
            pos[c] = hit[c] ? (tg[c] >> 31) != 0u
                            : (jc >= 0 && ((sign[(size_t)i * Qw + (jc >> 5)] >> (jc & 31)) & 1u) != 0u);
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < ELIM_CH; ++c) {
            const int s = b0 + 32 * c + lane;
            const bool valid = j[c] >= 0;
            const bool opposite = valid && (pos[c] ? (ww[c] < real(0)) : (ww[c] > real(0)));
            const bool keep = valid && !opposite;
            if (opposite) atomicAnd(&conn[(size_t)i * Qw + (j[c] >> 5)], ~(1u << (j[c] & 31)));
            const uint32_t mask = __ballot_sync(0xffffffffu, keep);
            const int dst = wp + __popc(mask & lanemask_lt());
            if (keep && dst != s) {
                ind[row + dst] = j[c];
                w[row + dst] = ww[c];
                m[row + dst] = mm[c];
                v[row + dst] = vv[c];
            }
            if (tag && keep && (dst != s || !hit[c])) tag[row + dst] = (uint32_t)j[c] | (pos[c] ? 0x80000000u : 0u);
            wp += __popc(mask);
        }
        __syncwarp();
    }
    if (lane == 0) {
        len[i] = wp;
        dormant[i] = n - wp;
        cnt[i] = 0;
    }
    __syncwarp();
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

// The whole redistribution of D dormant synapses over the rows in one CTA (any size):
// the same rounds, draws and acceptances as k_deepr_round0 + k_deepr_accept0 +
// k_deepr_distribute (the per-round counts do not depend on the order of the atomic
// additions, so the result is the same).  cnt must be zero on entry (the elimination
// zeroes it); red: 32 long longs of shared memory.
__device__ __forceinline__ void redistribute_block(const int32_t* __restrict__ len, int32_t* __restrict__ cnt,
                                                   int32_t* __restrict__ room, int32_t* __restrict__ taken,
                                                   long long D, int P, int C, int Q, int no_autapse, uint64_t seed,
                                                   uint64_t rewire, int32_t* status, snn_rewire_stats* stats,
                                                   long long* red) {
    const long long groups0 = (D + 3) >> 2;
    for (long long g = threadIdx.x; g < groups0; g += blockDim.x) {
        const u64x4 u = philox(seed, PH_DEEPR_DIST, rewire, 0, (uint64_t)g, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < D) atomicAdd(&cnt[(int)mulhi_index(u[q], (uint64_t)P)], 1);
    }
    __syncthreads();
    long long rej = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int forb = (no_autapse && i < Q) ? 1 : 0;
        const int l = len[i];
        const int r1 = C - l, r2 = Q - forb - l;
        const int rm = r1 < r2 ? r1 : r2;
        const int c = cnt[i];
        const int acc = c < rm ? c : rm;
        room[i] = rm;
        taken[i] = acc;
        rej += c - acc;
    }
    long long remaining = block_sum_ll(rej, red);
    for (int r = 1; r < 64 && remaining > 0; ++r) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const long long groups = (remaining + 3) >> 2;
        for (long long g = threadIdx.x; g < groups; g += blockDim.x) {
            const u64x4 u = philox(seed, PH_DEEPR_DIST, rewire, (uint64_t)r, (uint64_t)g, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * g + q < remaining) atomicAdd(&cnt[(int)mulhi_index(u[q], (uint64_t)P)], 1);
        }
        __syncthreads();
        long long rj = 0;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int c = cnt[i];
            if (c) {
                const int free_ = room[i] - taken[i];
                const int acc = c < free_ ? c : free_;
                taken[i] += acc;
                rj += c - acc;
            }
        }
        remaining = block_sum_ll(rj, red);
    }
    if (threadIdx.x == 0) {
        if (remaining > 0) atomicOr(status, ST_CAPACITY);
        if (stats) {
            atomicAdd((unsigned long long*)&stats->removed, (unsigned long long)D);
            atomicAdd((unsigned long long*)&stats->overflow, (unsigned long long)remaining);
        }
    }
    __syncthreads();
}

// Free-target counts per chunk of 32 bitfield words of a row (the self target of a
// recurrent projection and the bits beyond Q count as taken).
__device__ __forceinline__ uint32_t conn_word(const uint32_t* crow, int wi, int Qw, int i, int forb,
                                              uint32_t tail_mask) {
    uint32_t word = 0xffffffffu;
    if (wi < Qw) {
        word = crow[wi];
        if (forb && (i >> 5) == wi) word |= 1u << (i & 31);
        if (wi == Qw - 1) word |= tail_mask;
    }
    return word;
}

constexpr int FORM_BATCH = 8;   // activations whose chunk words a warp loads together

// One warp: the activations of row i (taken[i] of them); F: NC + 1 ints of shared memory
// for the row's chunk counts, NC = ceil(Qw / 32).
template <typename real>
__device__ __forceinline__ void form_row_warp(int32_t* __restrict__ len, int32_t* __restrict__ ind,
                                              real* __restrict__ w, real* __restrict__ m, real* __restrict__ v,
                                              uint32_t* __restrict__ conn, const int32_t* __restrict__ taken,
                                              const int i, int C, int Q, int Qw, int no_autapse, uint64_t seed,
                                              uint64_t rewire, int32_t* status, snn_rewire_stats* stats,
                                              int32_t* F) {
    const int NC = (Qw + 31) >> 5;                   // chunks of 32 words (1024 targets)
    const int nt = taken[i];
    if (nt == 0) return;
    const int lane = lane_id();
    const int forb = (no_autapse && i < Q) ? 1 : 0;
    const uint32_t tail_mask = (Q & 31) ? ~((1u << (Q & 31)) - 1u) : 0u;   // bits beyond Q in the last word
    uint32_t* crow = conn + (size_t)i * Qw;
    const size_t row = (size_t)i * C;
    // chunk c is counted by lane c % 32: its 32 words as eight 16-byte loads (a row's
    // bitfield starts 16-byte aligned when Qw is a multiple of 4)
    const bool vec = (Qw & 3) == 0;
    for (int c = lane; c < NC; c += 32) {
        int z = 0;
        if (vec && c * 32 + 32 <= Qw) {
            const uint4* p4 = (const uint4*)(crow + c * 32);
            uint4 q[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) q[h] = p4[h];
#pragma unroll
            for (int h = 0; h < 8; ++h) z += __popc(~q[h].x) + __popc(~q[h].y) + __popc(~q[h].z) + __popc(~q[h].w);
            // self target and the bits beyond Q fall in this chunk only if its words hold them
            if (forb && (i >> 10) == c) z -= ((crow[i >> 5] >> (i & 31)) & 1u) ? 0 : 1;
            if (tail_mask && (Qw - 1) >> 5 == c) z -= __popc(~crow[Qw - 1] & tail_mask);
        } else {
            for (int h = 0; h < 32; ++h) z += __popc(~conn_word(crow, c * 32 + h, Qw, i, forb, tail_mask));
        }
        F[c] = z;
    }
    __syncwarp();
    const int n0 = len[i];
    const int n_free0 = Q - forb - n0;
    if (nt <= 32 && nt <= n_free0 && n0 + nt <= C) {
        // All activations of the row at once, the same choices as the sequential loop
        // below.  Activation k takes the m_k-th free target left by the earlier ones,
        // m_k = mulhi(u_k, n_free0 - k); among the free targets before this call that is
        // index x_k, the fixed point of x = m_k + |{x_j : j < k, x_j <= x}| (found in
        // activation order by warp votes); lane k then resolves x_k to its target by a
        // search of the chunk prefix sums and a scan of one chunk's words, so the
        // activations of a row resolve side by side instead of one after another.
        int carry = 0;
        for (int cb = 0; cb < NC; cb += 32) {        // exclusive prefix of the counts in place
            const int c = cb + lane;
            const int f = c < NC ? F[c] : 0;
            const int incl = warp_incl_scan(f);
            if (c < NC) F[c] = carry + incl - f;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        int mk = 0, xk = 0;
        if (lane < nt) {
            const uint64_t u = philox(seed, PH_DEEPR_FORM, rewire, (uint64_t)i, (uint64_t)lane, 0).x;
            mk = (int)mulhi_index(u, (uint64_t)(n_free0 - lane));
        }
        for (int k = 0; k < nt; ++k) {
            const int mkk = __shfl_sync(0xffffffffu, mk, k);
            int x = mkk;
            for (int it = 0; it <= k; ++it) {            // x grows by at most k
                const int xn = mkk + __popc(__ballot_sync(0xffffffffu, lane < k && xk <= x));
                if (xn == x) break;
                x = xn;
            }
            if (lane == k) xk = x;
        }
        // lane k: the chunk holding x_k and x_k's rank among that chunk's free targets
        int lo = 0, rem = 0;
        const bool valid = lane < nt && xk < carry;
        if (valid) {
            int hi = NC - 1;                             // last chunk whose prefix is <= x_k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (F[mid] <= xk) lo = mid;
                else hi = mid - 1;
            }
            rem = xk - F[lo];
        }
        // the whole warp resolves activation k in its chunk (lane h holds word h), the
        // chunk words of up to FORM_BATCH activations loaded together
        int target = -1;
        for (int k0 = 0; k0 < nt; k0 += FORM_BATCH) {
            uint32_t wv[FORM_BATCH];
#pragma unroll
            for (int u = 0; u < FORM_BATCH; ++u) {
                const int ck = __shfl_sync(0xffffffffu, lo, (k0 + u) & 31);
                wv[u] = k0 + u < nt ? conn_word(crow, ck * 32 + lane, Qw, i, forb, tail_mask) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < FORM_BATCH; ++u) {
                const int k = k0 + u;
                if (k >= nt) break;                      // warp-uniform
                const int ck = __shfl_sync(0xffffffffu, lo, k);
                const int rk = __shfl_sync(0xffffffffu, rem, k);
                const bool vk = __shfl_sync(0xffffffffu, valid ? 1 : 0, k) != 0;
                const uint32_t fr = ~wv[u];
                const int pc = __popc(fr);
                const int incl = warp_incl_scan(pc);
                const uint32_t hm = __ballot_sync(0xffffffffu, vk && rk >= incl - pc && rk < incl);
                int tg = -1;
                if (hm && lane == __ffs(hm) - 1) tg = (ck * 32 + lane) * 32 + nth_set_bit(fr, rk - (incl - pc));
                tg = __shfl_sync(0xffffffffu, tg, hm ? __ffs(hm) - 1 : 0);
                if (lane == k && hm) target = tg;
            }
        }
        const bool bad = __any_sync(0xffffffffu, lane < nt && target < 0);
        if (!bad && lane < nt) {
            ind[row + n0 + lane] = target;
            w[row + n0 + lane] = real(0);
            m[row + n0 + lane] = real(0);
            v[row + n0 + lane] = real(0);
            atomicOr(&crow[target >> 5], 1u << (target & 31));
        }
        if (lane == 0) {
            len[i] = bad ? n0 : n0 + nt;
            if (bad) atomicOr(status, ST_STATE);
            else if (stats) atomicAdd((unsigned long long*)&stats->formed, (unsigned long long)nt);
        }
        return;
    }
    int n = n0;
    int formed = 0;
    uint64_t u_l = 0;                                // lane k % 32's draw for activation k
    for (int k = 0; k < nt; ++k) {
        const int n_free = Q - forb - n;
        if (n_free <= 0 || n >= C) {
            if (lane == 0) atomicOr(status, ST_STATE);
            break;
        }
        // the draws depend only on (rewire, i, k): 32 activations' draws at once
        if ((k & 31) == 0 && k + lane < nt) u_l = philox(seed, PH_DEEPR_FORM, rewire, (uint64_t)i, (uint64_t)(k + lane), 0).x;
        const uint64_t u = __shfl_sync(0xffffffffu, u_l, k & 31);
        const int mth = (int)mulhi_index(u, (uint64_t)n_free);
        // chunk holding the mth free target (ascending), then its word and bit
        int chunk = -1, before = 0, seen = 0;
        for (int cb = 0; cb < NC && chunk < 0; cb += 32) {
            const int c = cb + lane;
            const int f = c < NC ? F[c] : 0;
            const int incl = warp_incl_scan(f);
            const int excl = incl - f;
            const uint32_t hm = __ballot_sync(0xffffffffu, c < NC && mth >= seen + excl && mth < seen + incl);
            if (hm) {
                const int src = __ffs(hm) - 1;
                chunk = cb + src;
                before = seen + __shfl_sync(0xffffffffu, excl, src);
            }
            seen += __shfl_sync(0xffffffffu, incl, 31);
        }
        int target = -1;
        if (chunk >= 0) {
            const int wi = chunk * 32 + lane;
            const uint32_t word = conn_word(crow, wi, Qw, i, forb, tail_mask);
            const int zeros = __popc(~word);
            const int incl = warp_incl_scan(zeros);
            const int excl = incl - zeros;
            const int want = mth - before;
            const uint32_t hm = __ballot_sync(0xffffffffu, want >= excl && want < incl);
            if (hm) {
                const int src = __ffs(hm) - 1;
                int tg = -1;
                if (lane == src) tg = wi * 32 + nth_set_bit(~word, want - excl);
                target = __shfl_sync(0xffffffffu, tg, src);
            }
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
            F[chunk] -= 1;
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

}  // namespace snn
