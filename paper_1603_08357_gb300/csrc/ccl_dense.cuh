// Step (i) on the dense strided nearest-neighbour list of Section 3: the list
// has W = (largest number of neighbours of any site) slots per site, and
// neighbour slot k of site i is nn[i + k*N]. A slot holding -1 is empty (the
// site has fewer than W neighbours); every other slot must hold a site in
// [0, N). Slot e = i + k*N has its open bit at bit e of the bit words (word
// e >> 5, bit e & 31), or draws it on the device like the CSR path.
//
// As in the CSR kernel, only the slots of row i with j < i are read (the bond
// {i, j} is decided in the row of its larger site), label[i] becomes the
// smallest open lower neighbour (or i), and the others are appended to the
// residual queue as pairs (i, j). The queue has the CSR path's band layout:
// CTA b owns the slots [N_b * W, N_b' * W) of its sites [N_b, N_b'), packs its
// pairs from the start of that range and records their count in band[b], so
// steps (ii)-(iv) run unchanged.
//
// Layout: for one k the 32 lanes of a warp (32 consecutive sites) read 32
// consecutive ints of nn and at most two bit words, so every load is a
// coalesced 128-byte line; no shared-memory staging is needed.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "ccl_device.cuh"

namespace ccl {

#ifndef CCL_DENSE_THREADS
#define CCL_DENSE_THREADS 256
#endif
#ifndef CCL_DENSE_CHUNKS
#define CCL_DENSE_CHUNKS 2
#endif
constexpr int kDenseThreads = CCL_DENSE_THREADS;
constexpr int kDenseChunks = CCL_DENSE_CHUNKS;               // chunks a warp scans at once
constexpr int kDenseSpan = kDenseThreads * kDenseChunks;     // sites per CTA step

template <bool kGen>
__device__ __forceinline__ bool dense_open(const Params &P, int64_t e, int32_t i, int32_t j) {
    if (kGen) return gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i);
    return (__ldg(P.one.bits + (e >> 5)) >> (e & 31)) & 1u;
}

// Label of site i with smallest open lower neighbour m (cnt of them): the
// sites of this CTA's band before the current step [vis_lo, vis_hi) hold
// their step-(i) labels and are visible after the step barrier, so a site
// whose m lies there takes label[m] (an ancestor of m) instead of m.
__device__ __forceinline__ int32_t dense_label(const Params &P, int32_t i, int32_t m, int32_t cnt,
                                               int64_t vis_lo, int64_t vis_hi) {
    if (!cnt) return i;
    if (m >= vis_lo && m < vis_hi) return __ldcg(P.one.labels + m);
    return m;
}

// Appends the warp's residual pairs (r of them at this lane) to the band's
// part of the queue: returns this lane's first slot.
__device__ __forceinline__ int64_t dense_emit_slot(int64_t qband, unsigned long long *band_cnt, int lane,
                                                   int r, unsigned long long &my_pairs) {
    const int incl = warp_incl_scan(r, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (total) {
        if (lane == 0) base = atomicAdd(band_cnt, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 0);
        if (lane == 0) my_pairs += (unsigned long long)total;
    }
    return qband + (int64_t)base + (incl - r);
}

template <bool kGen>
__global__ void __launch_bounds__(kDenseThreads) k_init_dense(Params P) {
    __shared__ unsigned long long band_cnt;
    int64_t band_lo, band_hi;
    cta_band(P.n_tiles, band_lo, band_hi);
    const int64_t n = P.one.n;
    const int W = (int)P.nn_width;
    const int64_t n_words = ((int64_t)W * n + 31) >> 5;
    const int64_t s_lo = min(band_lo * kTileSites, n), s_hi = min(band_hi * kTileSites, n);
    const int64_t qband = s_lo * W;
    if (threadIdx.x == 0) {
        band_cnt = 0;
        P.band[blockIdx.x].qbase = qband;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned long long my_pairs = 0;
    bool bad = false;
    for (int64_t t0 = s_lo; t0 < s_hi; t0 += kDenseSpan) {
        if (W <= kRowRegs) {
            // Every load of the step is issued before any is used: lane i's
            // slots, and the chunk's bit words. Chunk c0 (a multiple of 32)
            // has the bits of slot k in the 64 bits from word (c0 + k*n) >> 5
            // on: lane k holds that word, lane 8 + k the next one.
            int32_t jr[kDenseChunks][kRowRegs];
            uint32_t wl[kDenseChunks];
#pragma unroll
            for (int c = 0; c < kDenseChunks; ++c) {
                const int64_t c0 = t0 + (int64_t)(warp * kDenseChunks + c) * kChunk;
                const int64_t i64 = c0 + lane;
                const bool live = i64 < s_hi;
#pragma unroll
                for (int k = 0; k < kRowRegs; ++k)
                    jr[c][k] = (live && k < W) ? __ldcs(P.nn + i64 + k * n) : -1;
                wl[c] = 0;
                if (!kGen) {
                    const int kk = lane & 7;
                    const int64_t w = ((c0 + (int64_t)kk * n) >> 5) + (lane >> 3);
                    if (lane < 16 && kk < W && c0 < s_hi && w < n_words) wl[c] = __ldg(P.one.bits + w);
                }
            }
#pragma unroll
            for (int c = 0; c < kDenseChunks; ++c) {
                const int64_t c0 = t0 + (int64_t)(warp * kDenseChunks + c) * kChunk;
                if (c0 >= s_hi) break;
                const int64_t i64 = c0 + lane;
                const int32_t i = (int32_t)i64;
                int32_t m = INT32_MAX, mk = 0;
                uint32_t lowmask = 0;
#pragma unroll
                for (int k = 0; k < kRowRegs; ++k) {
                    bool open;
                    const int32_t j = jr[c][k];
                    if (kGen) {
                        open = j >= 0 && j < i && gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i);
                    } else {
                        const uint32_t lo = __shfl_sync(kFull, wl[c], k);
                        const uint32_t hi = __shfl_sync(kFull, wl[c], 8 + k);
                        const uint32_t win = __funnelshift_r(lo, hi, (uint32_t)((c0 + (int64_t)k * n) & 31));
                        open = j >= 0 && j < i && ((win >> lane) & 1u);
                    }
                    bad |= j < -1 || (int64_t)j >= n;
                    if (open) {
                        lowmask |= 1u << k;
                        if (j < m) { m = j; mk = k; }
                    }
                }
                const int cnt = __popc(lowmask);
                if (i64 < s_hi) P.one.labels[i] = dense_label(P, i, m, cnt, s_lo, t0);
                const int r = cnt > 1 ? cnt - 1 : 0;
                int64_t slot = dense_emit_slot(qband, &band_cnt, lane, r, my_pairs);
                if (r > 0) {
                    const uint32_t rm = lowmask & ~(1u << mk);
#pragma unroll
                    for (int k = 0; k < kRowRegs; ++k)
                        if ((rm >> k) & 1u) P.q[slot++] = make_int2(i, jr[c][k]);
                }
            }
        } else {
            for (int c = 0; c < kDenseChunks; ++c) {
                const int64_t c0 = t0 + (int64_t)(warp * kDenseChunks + c) * kChunk;
                if (c0 >= s_hi) break;
                const int64_t i64 = c0 + lane;
                const bool live = i64 < s_hi;
                const int32_t i = (int32_t)i64;
                int32_t m = INT32_MAX, mk = -1, cnt = 0;
                if (live) {
                    for (int k = 0; k < W; ++k) {
                        const int64_t e = i64 + (int64_t)k * n;
                        const int32_t j = __ldg(P.nn + e);
                        bad |= j < -1 || (int64_t)j >= n;
                        if (j >= 0 && j < i && dense_open<kGen>(P, e, i, j)) {
                            ++cnt;
                            if (j < m) { m = j; mk = k; }
                        }
                    }
                    P.one.labels[i] = dense_label(P, i, m, cnt, s_lo, t0);
                }
                const int r = cnt > 1 ? cnt - 1 : 0;
                int64_t slot = dense_emit_slot(qband, &band_cnt, lane, r, my_pairs);
                if (r > 0) {
                    for (int k = 0; k < W; ++k) {
                        const int64_t e = i64 + (int64_t)k * n;
                        const int32_t j = __ldg(P.nn + e);
                        if (k != mk && j >= 0 && j < i && dense_open<kGen>(P, e, i, j)) P.q[slot++] = make_int2(i, j);
                    }
                }
            }
        }
        __syncthreads();        // this step's labels become visible to the CTA's next steps
    }
    if (bad) raise_err(P.err, kErrIndex);
    if (lane == 0 && my_pairs) {
        atomicAdd(P.counters, my_pairs);
        atomicAdd(&P.band[blockIdx.x].cnt, my_pairs);
    }
}

}  // namespace ccl
