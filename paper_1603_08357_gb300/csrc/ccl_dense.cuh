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
    cta_band(P, band_lo, band_hi);
    const int64_t n = P.one.n;
    const int W = (int)P.nn_width;
    const int64_t n_words = ((int64_t)W * n + 31) >> 5;
    const int64_t s_lo = min(band_lo * kTileSites, n), s_hi = min(band_hi * kTileSites, n);
    const int64_t qband = s_lo * W;
    if (threadIdx.x == 0) {
        band_cnt = 0;
        P.band[P.band_off + blockIdx.x].qbase = qband;
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
        atomicAdd(&P.band[P.band_off + blockIdx.x].cnt, my_pairs);
    }
}

// ---------------------------------------------------------------------------
// Dense list through the step-(i) pipeline of k_init: for lists of at most
// kRowRegs slots, a producer lane streams each 1024-site tile's W slot slabs
// (slot k: the tile's sites' entries nn[s0 + k*N ...], contiguous) and their
// bit words into a 3-stage shared-memory ring with bulk asynchronous copies;
// 16 consumer warps scan two 32-site chunks each, store labels after both are
// scanned (the band shortcut's load overlaps the second scan) and append the
// residual pairs of both through one prefix sum.

constexpr int kDenseSlab = kTileSites + 8;        // a slot's slab, + 16-byte rounding
constexpr int kDenseWords = kTileSites / 32 + 8;  // its bit words, + rounding

struct __align__(16) DenseStageHdr {
    int2 off[kRowRegs];        // staged tiles: slab[k] index and bw[k] bit index of site s0
    int64_t nn_lo[kRowRegs];   // element of nn held at slab[k][0]
    int64_t w_lo[kRowRegs];    // word of the bit array held at bw[k][0]
    int32_t nn_cnt[kRowRegs];  // elements held
    int32_t w_cnt[kRowRegs];   // words held
    int64_t qband;             // first queue slot of the CTA's band
    int32_t s0, ts;            // first site and sites of the tile
    int32_t staged;            // 1: every slab and its bits are held whole
    int32_t pad_;
};

struct __align__(16) DenseStage {
    DenseStageHdr h;
    int32_t nn[kRowRegs][kDenseSlab];
    uint32_t bw[kRowRegs][kDenseWords];
};

constexpr size_t kDenseSmem = 64 + sizeof(DenseStage) * kStages;

template <bool kGen>
__device__ __forceinline__ void dense_produce(const Params &P, DenseStage *st, uint64_t *full, uint64_t *empty) {
    int64_t band_lo, band_hi;
    cta_band(P, band_lo, band_hi);
    const int64_t n = P.one.n;
    const int W = (int)P.nn_width;
    const int64_t n_words = ((int64_t)W * n + 31) >> 5;
    const int32_t *nn_end = P.nn + (int64_t)W * n;
    const uint32_t *bits_end = kGen ? nullptr : P.one.bits + n_words;
    const int64_t qband = min(band_lo * kTileSites, n) * W;
    if (band_lo < band_hi) P.band[P.band_off + blockIdx.x].qbase = qband;
    int64_t t_local = 0;
    for (int64_t tile = band_lo; tile < band_hi; ++tile, ++t_local) {
        const int s = (int)(t_local % kStages);
        const int64_t use = t_local / kStages;
        if (use > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((use - 1) & 1))) {
            raise_err(P.err, kErrNonconv);
            break;
        }
        DenseStageHdr &h = st[s].h;
        const int64_t s0 = tile * kTileSites;
        const int64_t ts = min((int64_t)kTileSites, n - s0);
        h.s0 = (int32_t)s0;
        h.ts = (int32_t)ts;
        h.qband = qband;
        uint32_t bytes = 0;
        int staged = 1;
        for (int k = 0; k < W; ++k) {
            const int64_t e0 = s0 + (int64_t)k * n, e1 = e0 + ts;
            int64_t lo, hi;
            copy_window(P.nn, e0, e1, P.nn, nn_end, kDenseSlab, lo, hi);
            h.nn_lo[k] = lo;
            h.nn_cnt[k] = (int32_t)(hi - lo);
            staged &= lo <= e0 && hi >= e1;
            bytes += 4u * (uint32_t)(hi - lo);
            if (!kGen) {
                const int64_t w0 = e0 >> 5, w1 = ((e1 - 1) >> 5) + 1;
                copy_window(P.one.bits, w0, w1, P.one.bits, bits_end, kDenseWords, lo, hi);
                h.w_lo[k] = lo;
                h.w_cnt[k] = (int32_t)(hi - lo);
                staged &= lo <= w0 && hi >= w1;
                bytes += 4u * (uint32_t)(hi - lo);
            }
        }
        h.staged = staged;
        if (staged)
            for (int k = 0; k < W; ++k) {
                const int64_t e0 = s0 + (int64_t)k * n;
                h.off[k] = make_int2((int32_t)(e0 - h.nn_lo[k]), kGen ? 0 : (int32_t)(e0 - 32 * h.w_lo[k]));
            }
        mbar_arrive_expect_tx(&full[s], bytes);
        for (int k = 0; k < W; ++k) {
            if (h.nn_cnt[k]) bulk_g2s(st[s].nn[k], P.nn + h.nn_lo[k], 4u * (uint32_t)h.nn_cnt[k], &full[s]);
            if (!kGen && h.w_cnt[k])
                bulk_g2s(st[s].bw[k], P.one.bits + h.w_lo[k], 4u * (uint32_t)h.w_cnt[k], &full[s]);
        }
    }
    drain_armed(full, t_local, P.err);
}

// one lane's site of a staged chunk: slot k's neighbour and its open bit
template <bool kGen>
__device__ __forceinline__ void dense_slot(const Params &P, const DenseStage &S, int k, int64_t e, int32_t i,
                                           int32_t &j, bool &open) {
    const DenseStageHdr &h = S.h;
    const int64_t r = e - h.nn_lo[k];
    j = (r >= 0 && r < h.nn_cnt[k]) ? S.nn[k][r] : __ldg(P.nn + e);
    if (kGen) {
        open = j >= 0 && j < i && gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i);
    } else {
        const int64_t w = (e >> 5) - h.w_lo[k];
        const uint32_t word = (w >= 0 && w < h.w_cnt[k]) ? S.bw[k][w] : __ldg(P.one.bits + (e >> 5));
        open = (word >> (e & 31)) & 1u;
    }
}

struct DenseChunk {
    int32_t i, lab, m;
    uint32_t lowmask;       // open lower slots
    int32_t mk, r;
};

template <bool kGen>
__device__ __forceinline__ void dense_scan_chunk(const Params &P, const DenseStage &S, int cc, int lane,
                                                 const TileCtx &tc, DenseChunk &c) {
    const DenseStageHdr &h = S.h;
    const int64_t n = P.one.n;
    const int W = (int)P.nn_width;
    const int32_t loc = cc * kChunk + lane;
    const int32_t i = h.s0 + loc;
    const bool live = loc < h.ts;
    int32_t m = INT32_MAX, mk = 0;
    uint32_t lowmask = 0;
    bool bad = false;
    if (tc.staged) {
#pragma unroll
        for (int k = 0; k < kRowRegs; ++k) {
            if (k >= W) break;
            const int2 off = h.off[k];
            const int32_t j = live ? S.nn[k][off.x + loc] : -1;
            bool open;
            if (kGen) {
                open = (uint32_t)j < (uint32_t)i &&
                       gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i);
            } else {
                const int32_t b = off.y + loc;
                open = (S.bw[k][b >> 5] >> (b & 31)) & 1u;
            }
            bad |= (uint32_t)(j + 1) > (uint32_t)n;        // j < -1 or j >= n
            if (open && (uint32_t)j < (uint32_t)i) {         // 0 <= j < i
                lowmask |= 1u << k;
                if (j < m) { m = j; mk = k; }
            }
        }
    } else {
        for (int k = 0; k < W; ++k) {
            int32_t j = -1;
            bool open = false;
            if (live) dense_slot<kGen>(P, S, k, (int64_t)i + (int64_t)k * n, i, j, open);
            bad |= j < -1 || (int64_t)j >= n;
            if (j >= 0 && j < i && open) {
                lowmask |= 1u << k;
                if (j < m) { m = j; mk = k; }
            }
        }
    }
    if (bad) raise_err(P.err, kErrIndex);
    const int cnt = __popc(lowmask);
    int32_t lab = cnt ? m : i;
    if (cnt) {
        const int32_t mt = (int32_t)((uint32_t)m / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab = __ldcg(P.one.labels + m);
    }
    c.i = i;
    c.lab = lab;
    c.m = m;
    c.mk = mk;
    c.lowmask = cnt ? (lowmask & ~(1u << mk)) : 0u;
    c.r = cnt > 1 ? cnt - 1 : 0;
}

// Both chunks of a consumer warp at once on a staged tile whose two chunks
// are full: each slot's header offsets are read once and the two chunks'
// loads interleave. Returns false (having done nothing) otherwise.
template <bool kGen>
__device__ __forceinline__ bool dense_scan_pair(const Params &P, const DenseStage &S, int cc0, int lane,
                                                const TileCtx &tc, DenseChunk &c0, DenseChunk &c1) {
    const DenseStageHdr &h = S.h;
    const int64_t n = P.one.n;
    const int W = (int)P.nn_width;
    const int32_t loc0 = cc0 * kChunk + lane, loc1 = loc0 + kChunk;
    if (!tc.staged || (cc0 + 2) * kChunk > h.ts) return false;
    const int32_t i0 = h.s0 + loc0, i1 = i0 + kChunk;
    int32_t m0 = INT32_MAX, m1 = INT32_MAX, k0 = 0, k1 = 0;
    uint32_t l0 = 0, l1 = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kRowRegs; ++k) {
        if (k >= W) break;
        const int2 off = h.off[k];
        const int32_t j0 = S.nn[k][off.x + loc0], j1 = S.nn[k][off.x + loc1];
        bool o0, o1;
        if (kGen) {
            o0 = (uint32_t)j0 < (uint32_t)i0 && gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j0, (uint32_t)i0);
            o1 = (uint32_t)j1 < (uint32_t)i1 && gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j1, (uint32_t)i1);
        } else {
            const int32_t b0 = off.y + loc0, b1 = b0 + kChunk;
            o0 = (S.bw[k][b0 >> 5] >> (b0 & 31)) & 1u;
            o1 = (S.bw[k][b1 >> 5] >> (b1 & 31)) & 1u;
        }
        bad |= (uint32_t)(j0 + 1) > (uint32_t)n || (uint32_t)(j1 + 1) > (uint32_t)n;
        if (o0 && (uint32_t)j0 < (uint32_t)i0) {
            l0 |= 1u << k;
            if (j0 < m0) { m0 = j0; k0 = k; }
        }
        if (o1 && (uint32_t)j1 < (uint32_t)i1) {
            l1 |= 1u << k;
            if (j1 < m1) { m1 = j1; k1 = k; }
        }
    }
    if (bad) raise_err(P.err, kErrIndex);
    const int n0 = __popc(l0), n1 = __popc(l1);
    int32_t lab0 = n0 ? m0 : i0, lab1 = n1 ? m1 : i1;
    if (n0) {
        const int32_t mt = (int32_t)((uint32_t)m0 / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab0 = __ldcg(P.one.labels + m0);
    }
    if (n1) {
        const int32_t mt = (int32_t)((uint32_t)m1 / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab1 = __ldcg(P.one.labels + m1);
    }
    c0.i = i0; c0.lab = lab0; c0.m = m0; c0.mk = k0;
    c0.lowmask = n0 ? (l0 & ~(1u << k0)) : 0u; c0.r = n0 > 1 ? n0 - 1 : 0;
    c1.i = i1; c1.lab = lab1; c1.m = m1; c1.mk = k1;
    c1.lowmask = n1 ? (l1 & ~(1u << k1)) : 0u; c1.r = n1 > 1 ? n1 - 1 : 0;
    return true;
}

template <bool kGen>
__device__ __forceinline__ void dense_emit_chunk(const Params &P, const DenseStage &S, const DenseChunk &c,
                                                 bool staged, int64_t slot) {
    const int64_t n = P.one.n;
    const int32_t loc = c.i - S.h.s0;
    uint32_t rm = c.lowmask;
    while (rm) {
        const int k = __ffs(rm) - 1;
        rm &= rm - 1;
        int32_t j;
        if (staged) {
            j = S.nn[k][S.h.off[k].x + loc];
        } else {
            bool open;
            dense_slot<kGen>(P, S, k, (int64_t)c.i + (int64_t)k * n, c.i, j, open);
        }
        P.q[slot++] = make_int2(c.lab, j);      // (parent of i, j): see init_emit_chunk
    }
}

template <bool kGen>
__global__ void __launch_bounds__(kInitThreads, 2) k_init_dense_tma(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kStages;
    DenseStage *st = reinterpret_cast<DenseStage *>(smem_raw + 64);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kInitConsumers);
        }
        mbar_fence_init();
    }
    __shared__ unsigned long long band_cnt;
    if (threadIdx.x == 0) band_cnt = 0;
    __syncthreads();
    if (warp == kInitConsumers) {
        if (lane == 0) dense_produce<kGen>(P, st, full, empty);
        return;
    }
    unsigned long long my_pairs = 0;
    int64_t band_lo, band_hi;
    cta_band(P, band_lo, band_hi);
    int64_t t_local = 0;
    for (int64_t tile = band_lo; tile < band_hi; ++tile, ++t_local) {
        const int s = (int)(t_local % kStages);
        if (!mbar_wait_bounded(&full[s], (uint32_t)((t_local / kStages) & 1))) {
            raise_err(P.err, kErrNonconv);
            break;
        }
        const DenseStage &S = st[s];
        TileCtx tc;
        tc.rb0 = 0;
        tc.nbits = 0;
        tc.staged = S.h.staged != 0;
        {
            const int64_t hi = tile - kStages;
            tc.vis_lo = (int32_t)band_lo;
            tc.vis_hi = hi < band_lo ? -1 : (int32_t)hi;
        }
        const int cc0 = warp * 2, cc1 = warp * 2 + 1;
        DenseChunk c0, c1;
        c0.r = c1.r = 0;
        const bool has0 = cc0 * kChunk < S.h.ts, has1 = cc1 * kChunk < S.h.ts;
        if (!(has1 && dense_scan_pair<kGen>(P, S, cc0, lane, tc, c0, c1))) {
            if (has0) dense_scan_chunk<kGen>(P, S, cc0, lane, tc, c0);
            if (has1) dense_scan_chunk<kGen>(P, S, cc1, lane, tc, c1);
        }
        if (has0 && c0.i < P.one.n) P.one.labels[c0.i] = c0.lab;
        if (has1 && c1.i < P.one.n) P.one.labels[c1.i] = c1.lab;
        const int rr = c0.r + c1.r;
        const int incl = warp_incl_scan(rr, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        if (total > 0) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&band_cnt, (unsigned long long)total);
            base = __shfl_sync(kFull, base, 0);
            if (lane == 0) my_pairs += (unsigned long long)total;
            const int64_t slot = S.h.qband + (int64_t)base + (incl - rr);
            if (c0.r > 0) dense_emit_chunk<kGen>(P, S, c0, tc.staged, slot);
            if (c1.r > 0) dense_emit_chunk<kGen>(P, S, c1, tc.staged, slot + c0.r);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (lane == 0 && my_pairs) {
        atomicAdd(P.counters, my_pairs);
        atomicAdd(&P.band[P.band_off + blockIdx.x].cnt, my_pairs);
    }
}

}  // namespace ccl
