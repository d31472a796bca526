// Device side of the labelling library: the four steps of Section 3 of
// Komura, "A generalized GPU-based connected component labeling algorithm",
// as sm_103a kernels over one or many instances.
//
// Sites are grouped in chunks of 32 consecutive sites of one instance and
// chunks in tiles of kTileSites sites.
//  * Step (i) streams the CSR input: per CTA one producer warp moves each
//    tile's row pointers, column indices and bit words into shared memory with
//    bulk asynchronous copies (cp.async.bulk, completion on mbarriers, a ring
//    of kStages stages); kInitConsumers consumer warps scan the rows (two
//    chunks per warp and tile, interleaved), write the labels and append the
//    residual pairs to their CTA's part of the queue through one prefix sum
//    per warp and tile. Each CTA owns a contiguous band of tiles; a site whose
//    smallest lower neighbour lies in a band tile finished kStages tiles
//    earlier takes that neighbour's label (most of step (ii) on lattices).
//  * Step (iii) runs Algorithm 1 over the queue: each warp drains a window of
//    pairs with kRedSlots (six) pairs per lane in lockstep rounds (one load
//    or atomicMin per live pair per round, next state from a small table).
//  * Steps (ii)/(iv) chase every site's chain to its root, two chains per
//    lane at once (four in a batch), each warp over a contiguous range of
//    sites (or interleaved, for inputs without locality).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "ccl_types.cuh"

namespace ccl {

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ void raise_err(unsigned *err, unsigned bit) {
    if ((*(volatile unsigned *)err & bit) == 0) atomicOr(err, bit);
}

// Bond state drawn on the device. SplitMix64 (Steele, Lea & Flood 2014) in
// counter form: output number `key` of the generator started from state `seed`
// is mix(seed + (key + 1) * 0x9E3779B97F4A7C15); the bond {lo, hi} (lo < hi)
// has key lo * 2^32 + hi and is open iff (output >> 11) < thr, i.e. iff
// (output >> 11) * 2^-53 < p for thr = ceil(p * 2^53).
__device__ __forceinline__ bool gen_bond_open(uint64_t seed, uint64_t thr, uint32_t lo, uint32_t hi) {
    const uint64_t key = ((uint64_t)lo << 32) | hi;
    uint64_t z = seed + (key + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (z >> 11) < thr;
}

// largest k with insts[k].chunk_begin <= c (instances ordered)
__device__ __forceinline__ int find_inst(const Params &P, int64_t c) {
    int lo = 0, hi = P.K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.insts[mid].chunk_begin) <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_inst_tile(const Params &P, int64_t t) {
    int lo = 0, hi = P.K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.insts[mid].tile_begin) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool kBatched>
__device__ __forceinline__ Inst inst_of(const Params &P, int k) {
    if (!kBatched) return P.one;
    return P.insts[k];
}

// The instance of a staged tile as the step (i) consumers use it: from the
// kernel parameters for one instance, else from the stage header (shared
// memory) that the producer filled from the instance table.
template <bool kBatched>
__device__ __forceinline__ Inst stage_inst(const Params &P, const StageHdr &h) {
    if (!kBatched) return P.one;
    Inst I;
    I.row_ptr = h.i_rp;
    I.col_idx = h.i_ci;
    I.bits = h.i_bits;
    I.labels = h.i_lab;
    I.bit_off = h.i_bit_off;
    I.tile_begin = h.i_tile_begin;
    I.n = h.i_n;
    I.nnz = h.i_nnz;
    I.rp_lo = I.rp_hi = I.ci_lo = I.ci_hi = I.bits_lo = I.bits_hi = nullptr;   // not used by consumers
    I.q_off = I.chunk_begin = 0;
    return I;
}

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (inline PTX)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete; gives up after a bounded
// number of polls (each poll itself suspends for a hardware-bounded time).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Called by the producer lane before it returns: waits (bounded) until the
// copies of the last kStages tiles it armed (tiles 0 .. n_armed-1 of its
// band, stage t % kStages) have landed. Copies of earlier tiles have landed
// already: their stages were released by consumers that waited for them. So
// the CTA never exits with bulk copies still writing into its shared memory,
// also when a bounded wait expired and a loop was left early.
__device__ __forceinline__ void drain_armed(uint64_t *full, int64_t n_armed, unsigned *err) {
    for (int64_t t = n_armed > kStages ? n_armed - kStages : 0; t < n_armed; ++t)
        if (!mbar_wait_bounded(&full[t % kStages], (uint32_t)((t / kStages) & 1))) raise_err(err, kErrNonconv);
}

// 1-D bulk copy global -> shared, completing `bytes` on the mbarrier.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// The 16-byte aligned span covering elements [lo, hi) of the 4-byte array
// `arr`, clipped to the readable memory [mlo, mhi). Returns the element range
// [c_lo, c_hi) it covers (relative to arr; may extend past [lo, hi)), or an
// empty range if nothing can be copied or it exceeds `cap` elements.
__device__ __forceinline__ void copy_window(const void *arr, int64_t lo, int64_t hi, const void *mlo,
                                            const void *mhi, int cap, int64_t &c_lo, int64_t &c_hi) {
    const uintptr_t base = (uintptr_t)arr;
    uintptr_t a = (base + 4 * (uintptr_t)lo) & ~(uintptr_t)15;
    uintptr_t b = (base + 4 * (uintptr_t)hi + 15) & ~(uintptr_t)15;
    const uintptr_t l = ((uintptr_t)mlo + 15) & ~(uintptr_t)15;
    const uintptr_t h = (uintptr_t)mhi & ~(uintptr_t)15;
    if (a < l) a = l;
    if (b > h) b = h;
    if (hi <= lo || b <= a || (b - a) / 4 > (uintptr_t)cap) { c_lo = c_hi = lo; return; }
    c_lo = ((intptr_t)a - (intptr_t)base) / 4;
    c_hi = ((intptr_t)b - (intptr_t)base) / 4;
}

// ---------------------------------------------------------------------------
// Step (i): initialisation. For site i: lower = open entries j < i of row i;
// label[i] = min(lower) or i; every other entry of `lower` (one occurrence of
// the minimum removed) is a residual pair (i, j).

// tiles of CTA b: the contiguous band [band_lo, band_hi) of the launch's
// P.n_tiles tiles, which start at tile P.tile_off (0 unless step (i) runs in
// parts); its band record is P.band[P.band_off + b]
__device__ __forceinline__ void cta_band(const Params &P, int64_t &band_lo, int64_t &band_hi) {
    const int64_t per = (P.n_tiles + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min((int64_t)blockIdx.x * per, P.n_tiles);
    band_lo = P.tile_off + lo;
    band_hi = P.tile_off + min(lo + per, P.n_tiles);
}

template <bool kBatched, bool kGen = false>
__device__ __forceinline__ void init_produce(const Params &P, Stage *st, uint64_t *full,
                                             uint64_t *empty) {
    int64_t band_lo, band_hi;
    cta_band(P, band_lo, band_hi);
    int64_t t_local = 0;
    int64_t qband = 0;
    int kc = 0;                              // cached instance and its tile range
    int64_t kc_lo = 0, kc_hi = kBatched ? 0 : P.n_tiles;
    for (int64_t tile = band_lo; tile < band_hi; ++tile, ++t_local) {
        const int s = (int)(t_local % kStages);
        const int64_t use = t_local / kStages;
        if (use > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((use - 1) & 1))) {
            raise_err(P.err, kErrNonconv);
            break;
        }
        if (kBatched && (tile < kc_lo || tile >= kc_hi)) {
            kc = find_inst_tile(P, tile);
            kc_lo = P.insts[kc].tile_begin;
            kc_hi = kc + 1 < P.K ? P.insts[kc + 1].tile_begin : P.n_tiles;
        }
        const int k = kc;
        const Inst I = inst_of<kBatched>(P, k);
        StageHdr h;
        h.k = k;
        h.s0 = (int32_t)((tile - I.tile_begin) * kTileSites);
        h.ts = min(kTileSites, I.n - h.s0);
        h.e0 = __ldcs(I.row_ptr + h.s0);
        h.e1 = __ldcs(I.row_ptr + h.s0 + h.ts);
        h.status = (h.e0 < 0 || h.e1 < h.e0 || h.e1 > I.nnz) ? 1 : 0;
        // row_ptr[0] == 0 and row_ptr[n] == nnz, once per instance
        if (h.s0 == 0 && h.e0 != 0) raise_err(P.err, kErrShape);
        if (h.s0 + h.ts == I.n && h.e1 != I.nnz) raise_err(P.err, kErrShape);
        h.i_rp = I.row_ptr;
        h.i_ci = I.col_idx;
        h.i_bits = I.bits;
        h.i_lab = I.labels;
        h.i_bit_off = I.bit_off;
        h.i_tile_begin = I.tile_begin;
        h.i_n = I.n;
        h.i_nnz = I.nnz;
        if (t_local == 0) {
            qband = I.q_off + (h.status ? 0 : h.e0);
            P.band[P.band_off + blockIdx.x].qbase = qband;
        }
        h.qband = qband;
        int64_t lo, hi;
        copy_window(I.row_ptr, h.s0, (int64_t)h.s0 + h.ts + 1, I.rp_lo, I.rp_hi, kRpBuf, lo, hi);
        h.rp_lo = (int32_t)lo;
        h.rp_hi = (int32_t)hi;
        if (h.status == 0) {
            copy_window(I.col_idx, h.e0, h.e1, I.ci_lo, I.ci_hi, kColBuf, lo, hi);
            h.ci_lo = (int32_t)lo;
            h.ci_hi = (int32_t)hi;
            const int64_t w0 = (I.bit_off + h.e0) >> 5;
            const int64_t w1 = (h.e1 > h.e0 && !kGen) ? ((I.bit_off + h.e1 - 1) >> 5) + 1 : w0;
            copy_window(I.bits, w0, w1, I.bits_lo, I.bits_hi, kBitBuf, h.w_lo, h.w_hi);
        } else {
            h.ci_lo = h.ci_hi = 0;
            h.w_lo = h.w_hi = 0;
        }
        h.t_rb0 = (int32_t)(I.bit_off - (h.w_lo << 5));
        h.t_nbits = (int32_t)(32 * (h.w_hi - h.w_lo));
        h.t_staged = h.status == 0 && h.e0 >= h.ci_lo && h.e1 <= h.ci_hi &&
                     (kGen || (h.t_rb0 + h.e0 >= 0 && h.t_rb0 + h.e1 <= h.t_nbits));
        {
            // tiles of this band finished at least kStages tiles ago
            const int64_t lo = max(band_lo, I.tile_begin) - I.tile_begin;
            const int64_t hi = tile - kStages - I.tile_begin;
            h.t_vis_lo = (int32_t)lo;
            h.t_vis_hi = hi < lo ? -1 : (int32_t)hi;
        }
        st[s].h = h;
        const uint32_t b_rp = 4u * (uint32_t)(h.rp_hi - h.rp_lo);
        const uint32_t b_ci = 4u * (uint32_t)(h.ci_hi - h.ci_lo);
        const uint32_t b_bw = 4u * (uint32_t)(h.w_hi - h.w_lo);
        mbar_arrive_expect_tx(&full[s], b_rp + b_ci + b_bw);
        if (b_rp) bulk_g2s(st[s].rp, I.row_ptr + h.rp_lo, b_rp, &full[s]);
        if (b_ci) bulk_g2s(st[s].ci, I.col_idx + h.ci_lo, b_ci, &full[s]);
        if (b_bw) bulk_g2s(st[s].bw, I.bits + h.w_lo, b_bw, &full[s]);
    }
    drain_armed(full, t_local, P.err);
}

// General scan of one lane's row (rows longer than kRowRegs, or parts of the
// input outside the shared-memory copy): per-entry bounds-checked reads.
// the open bit of local entry e of instance I (row i, column j < i)
template <bool kGen>
__device__ __forceinline__ bool entry_open(const Params &P, const Stage &S, const Inst &I, int32_t e,
                                           int32_t i, int32_t j) {
    if (kGen) return gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i);
    const StageHdr &h = S.h;
    const int64_t ge = I.bit_off + e;
    const int64_t we = ge >> 5;
    const uint32_t w = (we >= h.w_lo && we < h.w_hi) ? S.bw[we - h.w_lo] : __ldg(I.bits + we);
    return (w >> (ge & 31)) & 1u;
}

template <bool kGen>
__device__ __forceinline__ void scan_row_general(const Params &P, const Stage &S, const Inst &I, int32_t a,
                                                 int32_t a_next, int32_t i, int32_t &m, int32_t &mk,
                                                 int32_t &cnt, bool &bad) {
    const StageHdr &h = S.h;
    for (int32_t e = a; e < a_next; ++e) {
        const int32_t j = (e >= h.ci_lo && e < h.ci_hi) ? S.ci[e - h.ci_lo] : __ldg(I.col_idx + e);
        bad |= (uint32_t)j >= (uint32_t)I.n;
        if ((uint32_t)j < (uint32_t)i && entry_open<kGen>(P, S, I, e, i, j)) {
            ++cnt;
            if (j < m) { m = j; mk = e; }
        }
    }
}

// Per-tile values a consumer warp computes once: the stage-relative bit
// offset of entry 0 and the number of copied bits (32-bit), and the range of
// the instance's tiles whose labels are final and visible here.
struct TileCtx {
    int32_t rb0;        // stage-relative bit index of local entry 0
    int32_t nbits;      // bits present in the stage
    int32_t vis_lo;     // instance-local tiles [vis_lo, vis_hi] are visible
    int32_t vis_hi;
    bool staged;        // the stage holds the columns and bits of the tile's whole entry range
};

// The stage header words the register path reads, copied to registers once
// per tile with 16-byte shared-memory loads.
struct TileHdr {
    int32_t k, s0, ts, e0, e1, rp_lo, rp_hi, ci_lo;
};

__device__ __forceinline__ void load_tile_hdr(const StageHdr &h, TileHdr &th, TileCtx &tc) {
    const int4 a = *reinterpret_cast<const int4 *>(&h.k);
    const int4 b = *reinterpret_cast<const int4 *>(&h.e1);
    const int4 c = *reinterpret_cast<const int4 *>(&h.t_rb0);
    th.k = a.x; th.s0 = a.y; th.ts = a.z; th.e0 = a.w;
    th.e1 = b.x; th.rp_lo = b.y; th.rp_hi = b.z; th.ci_lo = b.w;
    tc.rb0 = c.x; tc.nbits = c.y; tc.staged = c.z != 0; tc.vis_lo = c.w;
    tc.vis_hi = h.t_vis_hi;
}

// One chunk of 32 sites. The tiles of this CTA's band that were finished at
// least kStages tiles ago are visible (their labels were released through the
// stage barriers): a site whose smallest open lower neighbour m lies in such
// a tile takes label[m] (the root of m's tree after steps (i)/(ii)) instead of
// m, which shortcuts the chain step (ii) would walk.
// What the emission of a scanned chunk needs (per lane).
struct ChunkRes {
    int32_t i, a, a_next, mk;
    int32_t lab;        // label[i] to store (may be a load still in flight)
    uint32_t resmask;
    int32_t r;          // residual pairs of the lane's site
    bool fast;          // warp-uniform: the register path scanned the chunk
};

template <bool kBatched, bool kGen = false>
__device__ __forceinline__ void init_scan_chunk(const Params &P, const Stage &S, const Inst &I,
                                                int cc, int lane, const TileCtx &tc, ChunkRes &cr) {
    const StageHdr &h = S.h;
    const int32_t n = I.n;
    const int32_t s0 = h.s0 + cc * kChunk;
    const int32_t i = s0 + lane;
    const int32_t slast = min(s0 + kChunk, n);
    int32_t a, a_next;
    if (s0 >= h.rp_lo && slast < h.rp_hi) {
        a = S.rp[min(i, slast) - h.rp_lo];
        a_next = S.rp[min(i + 1, slast) - h.rp_lo];
    } else {
        a = __ldcs(I.row_ptr + min(i, slast));
        a_next = __ldcs(I.row_ptr + min(i + 1, slast));
    }
    // A row outside the tile's entry range, or running backwards, is read as
    // empty and flagged; the rows of a valid input always pass.
    if (!(a >= h.e0 && a <= a_next && a_next <= h.e1 && h.status == 0)) {
        raise_err(P.err, kErrIndex);
        a = a_next = h.e0 > 0 ? h.e0 : 0;
    }
    // rows now lie inside [e0, e1]; tc.staged says whether the stage holds
    // all of that range (columns and bits)
    const int32_t deg = a_next - a;
    const int32_t dmax = __reduce_max_sync(kFull, (uint32_t)deg);
    const bool all_fast = dmax <= kRowRegs && tc.staged;
    int32_t m = INT32_MAX, cnt = 0;
    int32_t mk = -1;
    uint32_t resmask = 0;
    bool bad = false;
    if (all_fast) {
        const int32_t *col = S.ci + (a - h.ci_lo);
        uint32_t win = 0;
        if (!kGen && deg > 0) {
            const int32_t rel = tc.rb0 + a;
            win = __funnelshift_r(S.bw[rel >> 5], S.bw[(rel + deg - 1) >> 5], (uint32_t)rel & 31u);
        }
        uint32_t lowmask = 0, jmax = 0;
#pragma unroll
        for (int t = 0; t < kRowRegs; ++t) {
            if (t >= dmax) break;
            if (t < deg) {
                const int32_t j = col[t];
                jmax = max(jmax, (uint32_t)j);
                const bool open = kGen ? ((uint32_t)j < (uint32_t)i &&
                                          gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i))
                                       : ((win >> t) & 1u) != 0;
                if (open && (uint32_t)j < (uint32_t)i) {
                    lowmask |= 1u << t;
                    if (j < m) { m = j; mk = t; }
                }
            }
        }
        bad = jmax >= (uint32_t)n;
        cnt = __popc(lowmask);
        resmask = cnt ? (lowmask & ~(1u << mk)) : 0u;
    } else {
        scan_row_general<kGen>(P, S, I, a, a_next, i, m, mk, cnt, bad);
    }
    if (bad) raise_err(P.err, kErrIndex);
    // the label; the caller stores it after scanning its other chunk, so the
    // shortcut's load below has that scan's time to arrive
    int32_t lab = cnt ? m : i;
    if (cnt) {
        const int32_t mt = (int32_t)((uint32_t)m / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab = __ldcg(I.labels + m);
    }
    cr.lab = lab;
    cr.i = i;
    cr.a = a;
    cr.a_next = a_next;
    cr.mk = mk;
    cr.resmask = resmask;
    cr.fast = all_fast;
    cr.r = cnt > 1 ? cnt - 1 : 0;
}

// Both chunks of a consumer warp at once, when every row of both is short and
// staged (the common case): the two rows of a lane are scanned in one loop,
// so their shared-memory loads and dependent arithmetic interleave. Returns
// false (having done nothing) otherwise.
template <bool kBatched, bool kGen = false>
__device__ __forceinline__ bool init_scan_pair(const Params &P, const Stage &S, const Inst &I, int cc0,
                                               int lane, const TileCtx &tc, const TileHdr &h, ChunkRes &c0,
                                               ChunkRes &c1) {
    const int32_t n = I.n;
    const int32_t s00 = h.s0 + cc0 * kChunk;
    if (!tc.staged || s00 + 2 * kChunk > n || s00 < h.rp_lo || s00 + 2 * kChunk >= h.rp_hi) return false;
    const int32_t i0 = s00 + lane, i1 = i0 + kChunk;
    const int32_t *rp = S.rp + (s00 - h.rp_lo);
    int32_t a0 = rp[lane], b0 = rp[lane + 1], a1 = rp[lane + kChunk], b1 = rp[lane + kChunk + 1];
    const bool ok0 = a0 >= h.e0 && a0 <= b0 && b0 <= h.e1, ok1 = a1 >= h.e0 && a1 <= b1 && b1 <= h.e1;
    const int32_t d0 = b0 - a0, d1 = b1 - a1;
    const int32_t dmax = __reduce_max_sync(kFull, (uint32_t)max(ok0 ? d0 : 0, ok1 ? d1 : 0));
    if (!__all_sync(kFull, ok0 && ok1) || dmax > kRowRegs) return false;
    const int32_t *col0 = S.ci + (a0 - h.ci_lo), *col1 = S.ci + (a1 - h.ci_lo);
    uint32_t w0 = 0, w1 = 0;
    if (!kGen) {
        const int32_t r0 = tc.rb0 + a0, r1 = tc.rb0 + a1;
        if (d0 > 0) w0 = __funnelshift_r(S.bw[r0 >> 5], S.bw[(r0 + d0 - 1) >> 5], (uint32_t)r0 & 31u);
        if (d1 > 0) w1 = __funnelshift_r(S.bw[r1 >> 5], S.bw[(r1 + d1 - 1) >> 5], (uint32_t)r1 & 31u);
    }
    int32_t m0 = INT32_MAX, m1 = INT32_MAX, k0 = -1, k1 = -1;
    uint32_t l0 = 0, l1 = 0, jmax = 0;
#pragma unroll
    for (int t = 0; t < kRowRegs; ++t) {
        if (t >= dmax) break;
        if (t < d0) {
            const int32_t j = col0[t];
            jmax = max(jmax, (uint32_t)j);
            const bool open = kGen ? ((uint32_t)j < (uint32_t)i0 &&
                                      gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i0))
                                   : ((w0 >> t) & 1u) != 0;
            if (open && (uint32_t)j < (uint32_t)i0) {
                l0 |= 1u << t;
                if (j < m0) { m0 = j; k0 = t; }
            }
        }
        if (t < d1) {
            const int32_t j = col1[t];
            jmax = max(jmax, (uint32_t)j);
            const bool open = kGen ? ((uint32_t)j < (uint32_t)i1 &&
                                      gen_bond_open(P.gen_seed, P.gen_thr, (uint32_t)j, (uint32_t)i1))
                                   : ((w1 >> t) & 1u) != 0;
            if (open && (uint32_t)j < (uint32_t)i1) {
                l1 |= 1u << t;
                if (j < m1) { m1 = j; k1 = t; }
            }
        }
    }
    if (jmax >= (uint32_t)n) raise_err(P.err, kErrIndex);
    const int n0 = __popc(l0), n1 = __popc(l1);
    int32_t lab0 = n0 ? m0 : i0, lab1 = n1 ? m1 : i1;
    // One pointer jump inside the warp's window of 64 sites [s00, s00 + 64):
    // a label that points to a window site takes that site's label. The value
    // taken is an ancestor of the site, so it stays a valid label, and a chain
    // along a lattice row shortens by half before step (iii) and the analysis
    // follow it. (A chunk-0 label lies below its site, so inside the window it
    // points into chunk 0; a chunk-1 label may point into either chunk.) One
    // jump measured faster end to end than jumping until the window is
    // settled: the later rounds cost step (i) more than they save afterwards.
    if (__any_sync(kFull, (uint32_t)(lab0 - s00) < 64u || (uint32_t)(lab1 - s00) < 64u)) {
        const uint32_t w0 = (uint32_t)(lab0 - s00), w1 = (uint32_t)(lab1 - s00);
        const int32_t a0v = __shfl_sync(kFull, lab0, (int)(w0 & 31u));
        const int32_t a1v = __shfl_sync(kFull, lab0, (int)(w1 & 31u));
        const int32_t b1v = __shfl_sync(kFull, lab1, (int)(w1 & 31u));
        if (w0 < 32u) lab0 = a0v;
        if (w1 < 64u) lab1 = w1 < 32u ? a1v : b1v;
    }
    // a label before the window in a tile of this band finished kStages tiles
    // ago: take that site's label (the band shortcut)
    if (lab0 < s00) {
        const int32_t mt = (int32_t)((uint32_t)lab0 / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab0 = __ldcg(I.labels + lab0);
    }
    if (lab1 < s00) {
        const int32_t mt = (int32_t)((uint32_t)lab1 / kTileSites);
        if (mt >= tc.vis_lo && mt <= tc.vis_hi) lab1 = __ldcg(I.labels + lab1);
    }
    c0.i = i0; c0.a = a0; c0.a_next = b0; c0.mk = k0; c0.lab = lab0; c0.fast = true;
    c0.resmask = n0 ? (l0 & ~(1u << k0)) : 0u; c0.r = n0 > 1 ? n0 - 1 : 0;
    c1.i = i1; c1.a = a1; c1.a_next = b1; c1.mk = k1; c1.lab = lab1; c1.fast = true;
    c1.resmask = n1 ? (l1 & ~(1u << k1)) : 0u; c1.r = n1 > 1 ? n1 - 1 : 0;
    return true;
}

// Writes the residual pairs of one scanned chunk from queue slot `slot` on.
// A pair {i, j} is stored as (label[i], j): label[i] is i's parent in the
// label forest and, i not being a root, step (iii) never rewrites it, so the
// pair joins the same two trees and its root search starts one hop higher.
template <bool kBatched, bool kGen = false>
__device__ __forceinline__ void init_emit_chunk(const Params &P, const Stage &S, const Inst &I,
                                                const ChunkRes &cr, int64_t slot) {
    const StageHdr &h = S.h;
    const int32_t i = cr.i;
    const int32_t up = cr.lab;
    if (slot + cr.r > P.q_cap) { raise_err(P.err, kErrIndex); return; }   // corrupt rows only
    if (cr.fast) {
        const int32_t *col = S.ci + (cr.a - h.ci_lo);
        uint32_t resmask = cr.resmask;
        while (resmask) {
            const int t = __ffs(resmask) - 1;
            resmask &= resmask - 1;
            P.q[slot] = make_int2(up, col[t]);
            if (kBatched) P.qk[slot] = h.k;
            ++slot;
        }
    } else {
        for (int32_t e = cr.a; e < cr.a_next; ++e) {
            const int32_t j = (e >= h.ci_lo && e < h.ci_hi) ? S.ci[e - h.ci_lo] : __ldg(I.col_idx + e);
            if ((uint32_t)j < (uint32_t)i && e != cr.mk && entry_open<kGen>(P, S, I, e, i, j)) {
                P.q[slot] = make_int2(up, j);
                if (kBatched) P.qk[slot] = h.k;
                ++slot;
            }
        }
    }
}

// Both chunks of a warp on the register path: the residual pairs of a lane's
// two sites in one loop (chunk 0's bits low, chunk 1's from bit 16), with a
// warp-uniform trip count, so the warp neither diverges nor loops twice.
// The queue order is that of init_emit_chunk on chunk 0 then chunk 1.
template <bool kBatched>
__device__ __forceinline__ void init_emit_pair(const Params &P, const Stage &S, const TileHdr &h,
                                               const ChunkRes &c0, const ChunkRes &c1, int64_t slot, int rr) {
    const int iters = (int)__reduce_max_sync(kFull, (uint32_t)rr);
    uint32_t mm = c0.resmask | (c1.resmask << 16);
    if (slot + rr > P.q_cap) {                  // corrupt rows only
        if (rr > 0) raise_err(P.err, kErrIndex);
        mm = 0;
    }
    const int32_t offA = c0.a - h.ci_lo, offB = c1.a - h.ci_lo - 16;
    int2 *qp = P.q + slot;
    int32_t *kp = kBatched ? P.qk + slot : nullptr;
    for (int it = 0; it < iters; ++it) {
        if (mm) {
            const int t = __ffs(mm) - 1;
            mm &= mm - 1;
            const bool hi = t >= 16;
            const int32_t j = S.ci[(hi ? offB : offA) + t];
            *qp++ = make_int2(hi ? c1.lab : c0.lab, j);
            if (kBatched) *kp++ = h.k;
        }
    }
}

template <bool kBatched, bool kGen = false>
__global__ void __launch_bounds__(kInitThreads, 2) k_init(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kStages;
    Stage *st = reinterpret_cast<Stage *>(smem_raw + 64);
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
    if (warp == kInitConsumers) {               // producer warp
        if (lane == 0) init_produce<kBatched, kGen>(P, st, full, empty);
        return;
    }
    unsigned long long my_pairs = 0;
    int64_t band_lo, band_hi;
    cta_band(P, band_lo, band_hi);
    // stage s = tl % kStages and phase parity (tl / kStages) & 1 of local tile
    // tl, kept incrementally in 32-bit (no 64-bit division per tile)
    int s = 0;
    uint32_t ph = 0;
    const int32_t ntl = (int32_t)(band_hi - band_lo);
    for (int32_t tl = 0; tl < ntl; ++tl, s = (s + 1 == kStages) ? 0 : s + 1, ph ^= (s == 0) ? 1u : 0u) {
        const int64_t tile = band_lo + tl;
        if (!mbar_wait_bounded(&full[s], ph)) {
            raise_err(P.err, kErrNonconv);
            break;
        }
        const Stage &S = st[s];
        const Inst I = stage_inst<kBatched>(P, S.h);
        TileCtx tc;
        TileHdr th;
        load_tile_hdr(S.h, th, tc);
        static_assert(kChunksPerConsumer == 2, "a consumer warp scans two chunks per tile");
        {
            // both chunks are scanned first; their pairs then take one range of
            // queue slots (one prefix sum and one band counter update per tile)
            const int cc0 = warp * 2, cc1 = warp * 2 + 1;
            ChunkRes c0, c1;
            c0.r = c1.r = 0;
            c0.resmask = c1.resmask = 0u;
            c0.fast = c1.fast = true;
            const bool has0 = cc0 * kChunk < th.ts, has1 = cc1 * kChunk < th.ts;
            if (!(has1 && init_scan_pair<kBatched, kGen>(P, S, I, cc0, lane, tc, th, c0, c1))) {
                if (has0) init_scan_chunk<kBatched, kGen>(P, S, I, cc0, lane, tc, c0);
                if (has1) init_scan_chunk<kBatched, kGen>(P, S, I, cc1, lane, tc, c1);
            }
            // the pair count's prefix sum and the band counter first: the
            // shortcut label loads of the scan (c0.lab, c1.lab) land meanwhile
            const int rr = c0.r + c1.r;
            const int incl = warp_incl_scan(rr, lane);
            const int total = __shfl_sync(kFull, incl, 31);
            unsigned long long base = 0;
            if (total > 0) {
                if (lane == 0) base = atomicAdd(&band_cnt, (unsigned long long)total);
                base = __shfl_sync(kFull, base, 0);
            }
            if (has0 && c0.i < I.n) I.labels[c0.i] = c0.lab;
            if (has1 && c1.i < I.n) I.labels[c1.i] = c1.lab;
            if (total > 0) {
                if (lane == 0) my_pairs += (unsigned long long)total;
                const int64_t slot = S.h.qband + (int64_t)base + (incl - rr);
                if (c0.fast && c1.fast) {
                    init_emit_pair<kBatched>(P, S, th, c0, c1, slot, rr);
                } else {
                    if (c0.r > 0) init_emit_chunk<kBatched, kGen>(P, S, I, c0, slot);
                    if (c1.r > 0) init_emit_chunk<kBatched, kGen>(P, S, I, c1, slot + c0.r);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (lane == 0 && my_pairs) {
        atomicAdd(P.counters, my_pairs);
        atomicAdd(&P.band[P.band_off + blockIdx.x].cnt, my_pairs);
    }
}

// ---------------------------------------------------------------------------
// Steps (ii) and (iv): analysis. Every site follows its label chain to the
// root and stores the root. No atomics run concurrently with this kernel and
// every value written is an ancestor of the site, so plain stores are safe.
// A warp walks kCh chunks at once (one chain per lane per chunk) so that
// their dependent loads overlap: kAnaChunks for one instance, more for a
// batch, whose labels do not fit L2 (longer latencies to cover).

// kSeq = true: warp w walks contiguous runs of chunk groups in increasing
// order, so the chains of its later sites run into roots it has already
// stored (lattices numbered row by row) and, batched, the instance of a chunk
// changes rarely. With P.ana_group = 0 each warp walks one range (the label
// array fits in L2); with P.ana_group = G > 0 the groups are cut into
// super-chunks of G groups per warp, all warps working inside one super-chunk
// at a time, so the labels in use (and the roots their chains reach, in the
// same instances) stay within L2 when the whole array does not fit.
// kSeq = false: groups are interleaved over the warps (grid stride), which
// balances inputs without locality (randomly numbered trees).
template <bool kBatched, bool kSeq, int kCh = kAnaChunks>
__global__ void __launch_bounds__(512) k_analysis(Params P) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ngroups = (P.n_chunks + kCh - 1) / kCh;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = (ngroups + nwarps - 1) / nwarps;
    // run length G and super-chunk stride: one run of `per` groups per warp,
    // or runs of ana_group groups every nwarps * ana_group groups
    const int64_t G = !kSeq ? 1 : (P.ana_group > 0 && P.ana_group < per ? (int64_t)P.ana_group : per);
    const int64_t sc_stride = kSeq ? nwarps * G : nwarps;
    // the instance of the current chunks, its chunk range and the fields used,
    // kept in registers until a chunk of another instance comes
    int64_t kc_lo = 0, kc_hi = kBatched ? 0 : P.n_chunks;
    int32_t *kc_lab = P.one.labels;
    int32_t kc_n = P.one.n;
    for (int64_t run = wid * G; run < ngroups; run += sc_stride)
    for (int64_t gidx = run; gidx < min(run + G, ngroups); ++gidx) {
        int32_t *L[kCh];
        int32_t site[kCh], x[kCh], first[kCh];
        int32_t cap = 0;
        bool act[kCh];
#pragma unroll
        for (int u = 0; u < kCh; ++u) {
            const int64_t c = gidx * kCh + u;
            act[u] = false;
            L[u] = nullptr;
            site[u] = 0;
            if (c < P.n_chunks) {
                if (kBatched && (c < kc_lo || c >= kc_hi)) {
                    const int kc = find_inst(P, c);
                    kc_lo = P.insts[kc].chunk_begin;
                    kc_hi = kc + 1 < P.K ? P.insts[kc + 1].chunk_begin : P.n_chunks;
                    kc_lab = P.insts[kc].labels;
                    kc_n = P.insts[kc].n;
                }
                site[u] = (int32_t)((c - (kBatched ? kc_lo : P.one.chunk_begin)) * kChunk) + lane;
                L[u] = kc_lab;
                cap = max(cap, kc_n);
                act[u] = site[u] < kc_n;
            }
        }
        // all loads of a round are issued before any result is used, so the
        // kCh chains of a lane are in flight together
#pragma unroll
        for (int u = 0; u < kCh; ++u) x[u] = act[u] ? L[u][site[u]] : 0;
#pragma unroll
        for (int u = 0; u < kCh; ++u) {
            first[u] = x[u];
            act[u] = act[u] && x[u] != site[u];
        }
        for (int32_t it = 0;; ++it) {
            int32_t y[kCh];
#pragma unroll
            for (int u = 0; u < kCh; ++u) y[u] = act[u] ? L[u][x[u]] : 0;
            bool any = false;
#pragma unroll
            for (int u = 0; u < kCh; ++u) {
                if (act[u]) {
                    if (y[u] == x[u]) act[u] = false;
                    else { x[u] = y[u]; any = true; }
                }
            }
            if (!any) break;
            if (it > cap || (P.iter_cap > 0 && it + 1 >= P.iter_cap)) { raise_err(P.err, kErrNonconv); break; }
        }
#pragma unroll
        for (int u = 0; u < kCh; ++u)
            if (L[u] && x[u] != first[u] && site[u] < cap) L[u][site[u]] = x[u];
    }
}

// Steps (ii)/(iv) with parking, for inputs whose chains are mostly short but
// have a long tail: every chain first gets kAnaRounds rounds in lockstep with
// its warp (coalesced first loads, as k_analysis); the chains still
// unfinished are appended to a per-warp list in shared memory and finished 32
// at a time, one per lane, so a few long chains no longer hold up the lanes
// of a whole group. Same visiting order (runs of P.ana_group groups, or one
// range per warp) and the same results as k_analysis<kBatched, true>. (The
// test option P.iter_cap is served by k_analysis alone.)
constexpr int kAnaRounds = 4;
constexpr int kParkWarps = 8;                        // warps per CTA (256 threads)
constexpr int kParkCap = 32 * kAnaChunks + 32;       // < 32 left + one group's chains
template <bool kBatched>
__global__ void __launch_bounds__(256) k_analysis_park(Params P) {
    __shared__ int s_site[8][kParkCap];
    __shared__ int s_x[8][kParkCap];
    __shared__ int s_k[kBatched ? 8 : 1][kBatched ? kParkCap : 1];
    const int lane = threadIdx.x & 31;
    const int wl = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ngroups = (P.n_chunks + kAnaChunks - 1) / kAnaChunks;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + wl;
    const int64_t per = (ngroups + nwarps - 1) / nwarps;
    const int64_t G = (P.ana_group > 0 && P.ana_group < per ? (int64_t)P.ana_group : per);
    const int64_t sc_stride = nwarps * G;
    int kc = 0;
    int64_t kc_lo = 0, kc_hi = kBatched ? 0 : P.n_chunks;
    int cnt = 0;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t capit = (int32_t)min(32 * P.n_chunks, (int64_t)INT32_MAX - 1);
    auto drain = [&](int take) {
        const int base = cnt - take;
        const bool act0 = lane < take;
        int site = 0, x = 0;
        int32_t *Lp = P.one.labels;
        if (act0) {
            site = s_site[wl][base + lane];
            x = s_x[wl][base + lane];
            if (kBatched) Lp = P.insts[s_k[wl][base + lane]].labels;
        }
        bool act = act0;
        for (int32_t it = 0;; ++it) {
            const int32_t y = act ? Lp[x] : 0;
            if (act) { if (y == x) act = false; else x = y; }
            if (!__any_sync(kFull, act)) break;
            if (it > capit || (P.iter_cap > 0 && it + 1 + kAnaRounds >= P.iter_cap)) { raise_err(P.err, kErrNonconv); break; }
        }
        if (act0) Lp[site] = x;
        cnt = base;
        __syncwarp();
    };
    for (int64_t run = wid * G; run < ngroups; run += sc_stride)
    for (int64_t gidx = run; gidx < min(run + G, ngroups); ++gidx) {
        int32_t *L[kAnaChunks];
        int32_t site[kAnaChunks], x[kAnaChunks], first[kAnaChunks];
        int kk[kAnaChunks];
        bool act[kAnaChunks];
#pragma unroll
        for (int u = 0; u < kAnaChunks; ++u) {
            const int64_t c = gidx * kAnaChunks + u;
            act[u] = false; L[u] = nullptr; site[u] = 0; kk[u] = 0;
            if (c < P.n_chunks) {
                if (kBatched && (c < kc_lo || c >= kc_hi)) {
                    kc = find_inst(P, c);
                    kc_lo = P.insts[kc].chunk_begin;
                    kc_hi = kc + 1 < P.K ? P.insts[kc + 1].chunk_begin : P.n_chunks;
                }
                const Inst I = inst_of<kBatched>(P, kc);
                site[u] = (int32_t)((c - I.chunk_begin) * kChunk) + lane;
                L[u] = I.labels; kk[u] = kc;
                act[u] = site[u] < I.n;
            }
        }
#pragma unroll
        for (int u = 0; u < kAnaChunks; ++u) x[u] = act[u] ? L[u][site[u]] : 0;
#pragma unroll
        for (int u = 0; u < kAnaChunks; ++u) { first[u] = x[u]; act[u] = act[u] && x[u] != site[u]; }
#pragma unroll
        for (int r = 0; r < kAnaRounds; ++r) {
            int32_t y[kAnaChunks];
#pragma unroll
            for (int u = 0; u < kAnaChunks; ++u) y[u] = act[u] ? L[u][x[u]] : 0;
#pragma unroll
            for (int u = 0; u < kAnaChunks; ++u)
                if (act[u]) { if (y[u] == x[u]) act[u] = false; else x[u] = y[u]; }
        }
#pragma unroll
        for (int u = 0; u < kAnaChunks; ++u) {
            if (!act[u] && L[u] && x[u] != first[u]) L[u][site[u]] = x[u];
            const unsigned pk = __ballot_sync(kFull, act[u]);
            if (pk) {
                const int pos = cnt + __popc(pk & lt);
                if (act[u]) { s_site[wl][pos] = site[u]; s_x[wl][pos] = x[u]; if (kBatched) s_k[wl][pos] = kk[u]; }
                cnt += __popc(pk);
                __syncwarp();
                if (cnt >= 32) drain(32);
            }
        }
    }
    while (cnt > 0) drain(min(cnt, 32));
}

// ---------------------------------------------------------------------------
// Step (iii): label reduction, Algorithm 1 for every residual pair (i, j).
// The pairs of all bands form one flat index space (prefix sums of the band
// counts, in shared memory). A warp drains a window of pairs (at most
// kRedWindowMax, fewer when the queue is short so every warp has one); each
// lane carries kRedSlots pairs and takes the next pair of the window as soon
// as one finishes, so a long walk holds up one slot, not the warp. Every
// round issues one load or one atomicMin per live slot before any result is
// used, so a lane's slots are in flight together.
//
// Root finding walks the larger of the two current nodes (labels decrease
// towards a root, so the larger one cannot be an ancestor of the other):
// meeting means one tree (Algorithm 1's label_1 == label_2, nothing to do);
// reaching a root at the larger node means two trees, and that root is
// linked by Algorithm 1's atomicMin loop under the other tree's root (link
// mode 0) or under the other chain's current node (link mode 1).

enum : int32_t { kTaskDone = 0, kTaskChase = 1, kTaskRoot = 2, kTaskMerge = 3 };

// Next state of a slot, 2 bits at index 4 * state + 2 * (y == a) + (y == b):
//   Done  -> Done;
//   Chase -> y == a: Root (link mode 0) or Merge (link mode 1);
//            else y == b: Done (one tree); else Chase;
//   Root  -> y == b: Merge; else Root;
//   Merge -> y == a or y == b: Done; else Merge.
constexpr uint32_t red_next_table(int link_mode) {
    uint32_t t = 0;
    for (uint32_t idx = 0; idx < 16; ++idx) {
        const uint32_t s = idx >> 2;
        const bool eq_a = (idx & 2u) != 0, eq_b = (idx & 1u) != 0;
        uint32_t nx = kTaskDone;
        if (s == kTaskChase) nx = eq_a ? (link_mode ? kTaskMerge : kTaskRoot) : (eq_b ? kTaskDone : kTaskChase);
        else if (s == kTaskRoot) nx = eq_b ? kTaskMerge : kTaskRoot;
        else if (s == kTaskMerge) nx = (eq_a || eq_b) ? kTaskDone : kTaskMerge;
        t |= nx << (2u * idx);
    }
    return t;
}
constexpr uint32_t kRedNextLink0 = red_next_table(0), kRedNextLink1 = red_next_table(1);


// Chase loads may be served from L1: a stale label is an older ancestor,
// which only lengthens a walk (labels only decrease), and every merge goes
// through an atomicMin whose returned value is current.
__device__ __forceinline__ int32_t red_load(const int32_t *p) { return __ldca(p); }

// Two ways of handing a window's pairs to the slots:
//  kStatic = false: every round, the warp's empty slots take the window's
//    next pairs in order (ballot + popc), which balances lanes whose chains
//    differ in length (randomly numbered trees);
//  kStatic = true: lane l serves pairs wbeg + l, wbeg + l + 32, ... and loads
//    its next pair a round before a slot needs it: fewer instructions per
//    round and no exposed queue load (lattices).
template <bool kBatched, bool kStatic>
__global__ void __launch_bounds__(256) k_reduce(Params P) {
    __shared__ long long s_pref[kMaxBands + 1];
    if (threadIdx.x < 32) {
        // exclusive prefix of the band counts by warp 0: each lane sums a
        // contiguous slice, then a warp scan of the slice totals
        const int lane = threadIdx.x;
        const int per = (P.n_bands + 31) / 32;
        const int b0 = min(lane * per, P.n_bands), b1 = min(b0 + per, P.n_bands);
        long long part = 0;
        for (int b = b0; b < b1; ++b) part += (long long)P.band[b].cnt;
        long long incl = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        long long acc = incl - part;
        for (int b = b0; b < b1; ++b) {
            s_pref[b] = acc;
            acc += (long long)P.band[b].cnt;
        }
        if (lane == 31) s_pref[P.n_bands] = incl;
    }
    __syncthreads();
    const long long total = s_pref[P.n_bands];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wmax = P.red_window > 0 ? P.red_window : kRedWindowMax;
    long long win = (total + nwarps - 1) / nwarps;
    win = win < 64 ? 64 : (win > wmax ? wmax : win);
    const long long nwin = (total + win - 1) / win;
#ifdef CCL_DEVICE_STATS
    unsigned long long st_hops = 0, st_atom = 0, st_iter = 0;
#endif
    for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nwin; w += nwarps) {
        const long long wbeg = w * win;
        const int wlen = (int)(min(wbeg + win, total) - wbeg);
        // A pair needs at most 4n + 8 rounds (its chains and Algorithm 1's loop
        // are bounded by the instance's n <= 32 n_chunks); a lane serves at most
        // wlen pairs. Past this many rounds the window is abandoned with an error.
        const long long round_cap = P.iter_cap > 0 ? (long long)P.iter_cap
                                                    : (128ll * P.n_chunks + 8) * (long long)wlen;
        long long rounds = 0;
        // band of the window's first pair (all lanes search; smem broadcast)
        int band = 0;
        {
            int lo = 0, hi = P.n_bands - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_pref[mid] <= wbeg) lo = mid; else hi = mid - 1;
            }
            band = lo;
        }
        int nxt = 0;        // pairs of the window handed to slots so far
        // kStatic: the lane's next pair, loaded ahead
        long long pnext = wbeg + lane;
        const long long wend = wbeg + wlen;
        int cur = band;             // band cursor of this lane (its pairs increase)
        int2 pf = make_int2(0, 0);
        int pfk = 0;
        bool pf_ok = false;
        // batched: the labels of the lane's last instance (consecutive pairs
        // of a lane mostly come from one instance)
        int lk = 0;
        int32_t *llab = kBatched ? P.insts[0].labels : P.one.labels;
        // queue slot of pair p = qoff + p inside band `cur`
        long long qoff = P.band[cur].qbase - s_pref[cur];
        auto fetch = [&](long long p) {
            if (s_pref[cur + 1] <= p) {
                do { ++cur; } while (s_pref[cur + 1] <= p);
                qoff = P.band[cur].qbase - s_pref[cur];
            }
            const long long slot = qoff + p;
            pf = P.q[slot];
            if (kBatched) pfk = P.qk[slot];
            pf_ok = true;
        };
        if (kStatic && pnext < wend) { fetch(pnext); pnext += 32; }
        int32_t *L[kRedSlots];
        int32_t a[kRedSlots], b[kRedSlots], st[kRedSlots];
#pragma unroll
        for (int u = 0; u < kRedSlots; ++u) {
            st[u] = kTaskDone;
            L[u] = P.one.labels;
            a[u] = b[u] = 0;
        }
        for (;;) {
            if (kStatic) {
                // at most one empty slot per lane and round takes the prefetched pair
                int take = -1;
#pragma unroll
                for (int u = kRedSlots - 1; u >= 0; --u)
                    if (st[u] == kTaskDone) take = u;
                if (take >= 0 && pf_ok) {
                    const int32_t na = max(pf.x, pf.y), nb = min(pf.x, pf.y);
                    if (kBatched && pfk != lk) { lk = pfk; llab = P.insts[pfk].labels; }
                    int32_t *nl = llab;
#pragma unroll
                    for (int u = 0; u < kRedSlots; ++u)
                        if (u == take) { a[u] = na; b[u] = nb; st[u] = kTaskChase; L[u] = nl; }
                    pf_ok = false;
                    if (pnext < wend) { fetch(pnext); pnext += 32; }
                }
            } else {
                // refill empty slots with the window's next pairs, in order (the
                // tests are warp-uniform: nothing runs once the window is handed out)
                if (nxt < wlen) {
#pragma unroll
                    for (int u = 0; u < kRedSlots; ++u) {
                        const unsigned need = __ballot_sync(kFull, st[u] == kTaskDone);
                        if (need == 0) continue;
                        const int pos = nxt + __popc(need & lt);
                        if (st[u] == kTaskDone && pos < wlen) {
                            const long long p = wbeg + pos;
                            int bb = band;
                            while (s_pref[bb + 1] <= p) ++bb;
                            const long long slot = P.band[bb].qbase + (p - s_pref[bb]);
                            const int2 pr = P.q[slot];
                            if (kBatched) {
                                const int k = P.qk[slot];
                                if (k != lk) { lk = k; llab = P.insts[k].labels; }
                                L[u] = llab;
                            }
                            a[u] = max(pr.x, pr.y);
                            b[u] = min(pr.x, pr.y);
                            st[u] = kTaskChase;
                        }
                        nxt = min(nxt + __popc(need), wlen);
                        const long long pn = wbeg + nxt;
                        while (band < P.n_bands - 1 && s_pref[band + 1] <= pn) ++band;
                        if (nxt >= wlen) break;
                    }
                }
            }
#ifdef CCL_DEVICE_STATS
            st_iter++;
#endif
            // issue: one load or one atomicMin per live slot
            int32_t v[kRedSlots];
#pragma unroll
            for (int u = 0; u < kRedSlots; ++u) {
                int32_t *ptr = L[u] + (st[u] == kTaskRoot ? b[u] : a[u]);
                v[u] = 0;
                if (st[u] == kTaskMerge) v[u] = atomicMin(ptr, b[u]);
                else if (st[u] != kTaskDone) v[u] = red_load(ptr);
            }
            // use: the next state of every slot (no divergent paths). With
            // mx = max(y, b) and mn = min(y, b) every transition sets b = mn
            // and a = mx, except Root, which keeps a:
            //   Chase (y = label[a]): y == a means a root, so mx = a, mn = b;
            //     otherwise the walk goes on from the larger node;
            //   Root (y = label[b] <= b): b = y;
            //   Merge (y = old label[a]): Algorithm 1 continues with (old, b)
            //     when old > b and with (b, old) when old < b.
            // The next state is looked up by (state, y == a, y == b).
            const uint32_t table = P.link_mode ? kRedNextLink1 : kRedNextLink0;
            bool any = false;
#pragma unroll
            for (int u = 0; u < kRedSlots; ++u) {
                const int32_t y = v[u], A = a[u], Bv = b[u];
                const int s = st[u];
#ifdef CCL_DEVICE_STATS
                st_hops += (s == kTaskChase || s == kTaskRoot);
                st_atom += (s == kTaskMerge);
#endif
                const uint32_t idx = ((uint32_t)s << 2) | ((y == A) ? 2u : 0u) | ((y == Bv) ? 1u : 0u);
                a[u] = s == kTaskRoot ? A : max(y, Bv);
                b[u] = min(y, Bv);
                st[u] = (int32_t)((table >> (2u * idx)) & 3u);
                any |= st[u] != kTaskDone;
            }
            if (!__any_sync(kFull, any || pf_ok) && (kStatic || nxt >= wlen)) break;
            if (++rounds > round_cap) {
                raise_err(P.err, kErrNonconv);
                break;
            }
        }
    }
#ifdef CCL_DEVICE_STATS
    if (st_hops) atomicAdd(P.counters + 1, st_hops);
    if (st_atom) atomicAdd(P.counters + 2, st_atom);
    if (lane == 0 && st_iter) atomicAdd(P.counters + 3, st_iter);
#endif
}

// ---------------------------------------------------------------------------
// Input check for ccl_validate: one thread per site. (Only the translation
// unit that implements ccl_validate defines it.)

#ifndef CCL_NO_VALIDATE_KERNEL
__global__ void k_validate(int32_t n, int64_t nnz, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col_idx, const uint32_t *__restrict__ bits,
                           unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ii = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += stride) {
        const int32_t i = (int32_t)ii;
        const int32_t a = row_ptr[i], b = row_ptr[i + 1];
        if (i == 0 && a != 0) raise_err(err, kErrShape);
        if (i == n - 1 && b != nnz) raise_err(err, kErrShape);
        if (a < 0 || b < a || b > nnz) { raise_err(err, kErrIndex); continue; }
        for (int32_t e = a; e < b; ++e) {
            const int32_t j = col_idx[e];
            if ((uint32_t)j >= (uint32_t)n) { raise_err(err, kErrIndex); continue; }
            if (j == i) continue;
            const uint32_t bit = (bits[e >> 5] >> (e & 31)) & 1u;
            const int32_t c0 = row_ptr[j], c1 = row_ptr[j + 1];
            if (c0 < 0 || c1 < c0 || c1 > nnz) { raise_err(err, kErrIndex); continue; }
            bool found = false;
            for (int32_t f = c0; f < c1 && !found; ++f) {
                if (col_idx[f] == i && (((bits[f >> 5] >> (f & 31)) & 1u) == bit)) found = true;
            }
            if (!found) raise_err(err, kErrAsym);
        }
    }
}
#endif  // CCL_NO_VALIDATE_KERNEL

}  // namespace ccl
