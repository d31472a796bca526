// Device side of the labelling library: the four steps of Section 3 of
// Komura, "A generalized GPU-based connected component labeling algorithm",
// as sm_103a kernels over one or many instances.
//
// Work is cut into chunks of 32 consecutive sites of one instance; one warp
// owns a chunk at a time, persistent warps stride over all chunks of all
// instances. Step (i) stages a chunk's CSR segment (row pointers, column
// indices and the words of open bits) in the warp's shared memory with
// coalesced streaming loads and writes the chunk's residual pairs to a queue
// slot range that is fixed by the chunk's first CSR entry, so no global atomic
// counter is needed; step (iii) walks 32 chunk records per warp and
// flattens their pairs across the lanes.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "ccl_types.cuh"

namespace ccl {

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(p); }

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

// instance owning global chunk c: largest k with insts[k].chunk_begin <= c
__device__ __forceinline__ int find_inst(const Params &P, int64_t c) {
    int lo = 0, hi = P.K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.insts[mid].chunk_begin) <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool kBatched>
__device__ __forceinline__ Inst inst_of(const Params &P, int k) {
    if (!kBatched) return P.one;
    Inst I;
    const Inst *s = &P.insts[k];
    I.row_ptr = (const int32_t *)__ldg((const unsigned long long *)&s->row_ptr);
    I.col_idx = (const int32_t *)__ldg((const unsigned long long *)&s->col_idx);
    I.bits = (const uint32_t *)__ldg((const unsigned long long *)&s->bits);
    I.labels = (int32_t *)__ldg((const unsigned long long *)&s->labels);
    I.bit_off = __ldg(&s->bit_off);
    I.q_off = __ldg(&s->q_off);
    I.chunk_begin = __ldg(&s->chunk_begin);
    I.n = __ldg(&s->n);
    I.nnz = __ldg(&s->nnz);
    return I;
}

// Follows label[x] to its root (label[r] == r). Loads go to L2 (.cg) so that
// values written by atomics on other SMs are seen. Chains strictly decrease,
// so a walk longer than n means a corrupt array: flag it and stop.
__device__ __forceinline__ int32_t find_root_cg(const int32_t *L, int32_t x, int32_t cap,
                                                unsigned *err) {
    for (int32_t it = 0;; ++it) {
        int32_t p = __ldcg(L + x);
        if (p == x) return x;
        x = p;
        if (it > cap) { raise_err(err, kErrNonconv); return x; }
    }
}

// Algorithm 1, atomicMin loop, for two roots r1 > r2 found by the chase.
// Each atomicMin puts r2 under r1; a displaced parent `old` is merged next.
// `old == r1` means r1 was still a root, so nothing was displaced.
__device__ __forceinline__ void merge_roots(int32_t *L, int32_t r1, int32_t r2, int32_t cap,
                                            unsigned *err) {
    for (int32_t it = 0;; ++it) {
        int32_t old = atomicMin(L + r1, r2);
        if (old == r2 || old == r1) return;
        if (old > r2) {
            r1 = old;
        } else {
            r1 = r2;
            r2 = old;
        }
        if (it > cap) { raise_err(err, kErrNonconv); return; }
    }
}

// ---------------------------------------------------------------------------
// Step (i): initialisation. For site i: lower = open entries j < i of row i;
// label[i] = min(lower) or i; every other entry of `lower` (one occurrence of
// the minimum removed) is a residual pair (i, j).

template <bool kBatched>
__global__ void __launch_bounds__(512) k_init(Params P) {
    extern __shared__ int32_t s_stage[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int32_t *sc = s_stage + wib * (kStageEntries + kStageWords);
    uint32_t *sb = (uint32_t *)(sc + kStageEntries);
    unsigned long long my_pairs = 0;

    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; c < P.n_chunks; c += nwarps) {
        const int k = kBatched ? find_inst(P, c) : 0;
        const Inst I = inst_of<kBatched>(P, k);
        const int32_t n = I.n;
        const int32_t s0 = (int32_t)((c - I.chunk_begin) * kChunk);
        const int32_t i = s0 + lane;
        const int32_t slast = min(s0 + kChunk, n);          // one past the chunk's last site
        // lane l: start of its row; lanes past the end read row_ptr[slast]
        int32_t a = ld_stream(I.row_ptr + min(i, slast));
        int32_t tail = 0;
        if (lane == 0) tail = ld_stream(I.row_ptr + slast);
        tail = __shfl_sync(kFull, tail, 0);
        int32_t a_next = __shfl_down_sync(kFull, a, 1);
        if (lane == 31) a_next = tail;
        const bool ok = (a >= 0) && (a <= a_next) && (a_next <= I.nnz);
        const bool all_ok = __all_sync(kFull, ok);
        if (lane == 0) {
            if (s0 == 0 && a != 0) raise_err(P.err, kErrShape);
            if (slast == n && tail != I.nnz) raise_err(P.err, kErrShape);
        }
        if (!all_ok) {
            if (lane == 0) raise_err(P.err, kErrIndex);
            a = a_next = 0;
        }
        const int32_t beg = __shfl_sync(kFull, a, 0);
        const int32_t end = all_ok ? tail : 0;
        const int32_t E = end - beg;
        const bool staged = E <= kStageEntries;
        const int64_t g0 = I.bit_off + beg;
        const int64_t w0 = g0 >> 5;
        if (staged) {
            for (int t = lane; t < E; t += 32) sc[t] = ld_stream(I.col_idx + beg + t);
            const int nwords = E > 0 ? (int)(((I.bit_off + end - 1) >> 5) - w0 + 1) : 0;
            for (int t = lane; t < nwords; t += 32) sb[t] = ld_stream(I.bits + w0 + t);
        }
        __syncwarp();

        int32_t m = INT32_MAX, mpos = -1, cnt = 0;
        bool bad = false;
        for (int32_t e = a; e < a_next; ++e) {
            const int64_t g = I.bit_off + e;
            int32_t j;
            uint32_t w;
            if (staged) { j = sc[e - beg]; w = sb[(g >> 5) - w0]; }
            else { j = __ldg(I.col_idx + e); w = __ldg(I.bits + (g >> 5)); }
            if ((uint32_t)j >= (uint32_t)n) { bad = true; continue; }
            if (((w >> (g & 31)) & 1u) && j < i) {
                ++cnt;
                if (j < m) { m = j; mpos = e; }
            }
        }
        if (bad) raise_err(P.err, kErrIndex);
        if (i < n) I.labels[i] = cnt ? m : i;

        const int r = cnt > 1 ? cnt - 1 : 0;
        const int incl = warp_incl_scan(r, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        const int64_t qbeg = I.q_off + beg;
        if (r > 0) {
            int64_t slot = qbeg + (incl - r);
            for (int32_t e = a; e < a_next; ++e) {
                const int64_t g = I.bit_off + e;
                int32_t j;
                uint32_t w;
                if (staged) { j = sc[e - beg]; w = sb[(g >> 5) - w0]; }
                else { j = __ldg(I.col_idx + e); w = __ldg(I.bits + (g >> 5)); }
                if ((uint32_t)j >= (uint32_t)n) continue;
                if (((w >> (g & 31)) & 1u) && j < i && e != mpos) P.q[slot++] = make_int2(i, j);
            }
        }
        if (lane == 0) {
            ChunkRec rc;
            rc.qbeg = qbeg;
            rc.cnt = total;
            rc.inst = k;
            P.rec[c] = rc;
            my_pairs += (unsigned long long)total;
        }
        __syncwarp();
    }
    if (lane == 0 && my_pairs) atomicAdd(P.counters, my_pairs);
}

// ---------------------------------------------------------------------------
// Steps (ii) and (iv): analysis. Every site follows its label chain to the
// root and stores the root. No atomics run concurrently with this kernel, and
// every value written is an ancestor of the site, so plain stores are safe.

template <bool kBatched>
__global__ void __launch_bounds__(512) k_analysis(Params P) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < P.n_chunks;
         c += nwarps) {
        const int k = kBatched ? find_inst(P, c) : 0;
        const Inst I = inst_of<kBatched>(P, k);
        const int32_t i = (int32_t)((c - I.chunk_begin) * kChunk) + lane;
        if (i >= I.n) continue;
        int32_t *L = I.labels;
        const int32_t l = L[i];
        if (l == i) continue;
        int32_t x = L[l];
        if (x == l) continue;
        for (int32_t it = 0;; ++it) {
            const int32_t y = L[x];
            if (y == x) break;
            x = y;
            if (it > I.n) { raise_err(P.err, kErrNonconv); break; }
        }
        L[i] = x;
    }
}

// ---------------------------------------------------------------------------
// Step (iii): label reduction, Algorithm 1 for every residual pair. A warp
// takes 32 chunk records, prefix-sums their pair counts and spreads the pairs
// over its lanes. After the chase, lanes whose (instance, r1, r2) coincide
// elect one lane to run the atomicMin loop.

template <bool kBatched>
__global__ void __launch_bounds__(512) k_reduce(Params P) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ngroups = (P.n_chunks + 31) / 32;
    for (int64_t gidx = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gidx < ngroups;
         gidx += nwarps) {
        const int64_t c = gidx * 32 + lane;
        ChunkRec rc;
        if (c < P.n_chunks) rc = P.rec[c]; else { rc.qbeg = 0; rc.cnt = 0; rc.inst = 0; }
        const int incl = warp_incl_scan(rc.cnt, lane);
        const int excl = incl - rc.cnt;
        const int total = __shfl_sync(kFull, incl, 31);
        for (int base = 0; base < total; base += 32) {
            const int p = base + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = src + step;
                const int ex = __shfl_sync(kFull, excl, cand);
                if (ex <= p) src = cand;
            }
            const long long qb = __shfl_sync(kFull, (long long)rc.qbeg, src);
            const int ex_src = __shfl_sync(kFull, excl, src);
            const int k = __shfl_sync(kFull, rc.inst, src);
            const bool valid = p < total;
            int32_t r1 = -1, r2 = -1;
            int32_t *L = nullptr;
            int32_t cap = 0;
            if (valid) {
                const int2 pr = P.q[qb + (p - ex_src)];
                if (kBatched) {
                    L = (int32_t *)__ldg((const unsigned long long *)&P.insts[k].labels);
                    cap = __ldg(&P.insts[k].n);
                } else {
                    L = P.one.labels;
                    cap = P.one.n;
                }
                r1 = find_root_cg(L, __ldcg(L + pr.x), cap, P.err);
                r2 = find_root_cg(L, __ldcg(L + pr.y), cap, P.err);
                if (r1 < r2) { const int32_t t = r1; r1 = r2; r2 = t; }
            }
            bool need = valid && r1 != r2;
            if (P.dedup) {
                const unsigned long long key = need
                    ? (((unsigned long long)(uint32_t)r1 << 32) | (uint32_t)r2)
                    : (0xffffffff00000000ull | (unsigned)lane);
                unsigned peers = __match_any_sync(kFull, key);
                if (kBatched) peers &= __match_any_sync(kFull, need ? k : -1 - lane);
                need = need && ((__ffs(peers) - 1) == lane);
            }
            if (need) merge_roots(L, r1, r2, 2 * cap + 4, P.err);
        }
    }
}

// ---------------------------------------------------------------------------
// Input check for ccl_validate: one thread per site.

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

}  // namespace ccl
