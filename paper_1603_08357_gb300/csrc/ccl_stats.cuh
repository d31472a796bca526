// Kernels on finished canonical labels (the label of a site is the smallest
// site of its cluster, end of Section 3):
//  * sequential relabelling: clusters numbered 0..C-1 in the order of their
//    smallest sites (the renumbering the end of Section 3 mentions), plus
//    the size of every cluster;
//  * the spanning test of Section 4: the smallest label found both among the
//    labels of a set of "top" sites and among those of "bottom" sites;
//  * the largest cluster (its size and label).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "ccl_types.cuh"

namespace ccl {

constexpr int kRelThreads = 256;
constexpr int kRelPerThread = 32;
constexpr int kRelBlock = kRelThreads * kRelPerThread;   // sites per relabel block

// number of roots (label[i] == i) in each block of kRelBlock sites
__global__ void __launch_bounds__(kRelThreads) k_root_counts(int32_t n, const int32_t *__restrict__ lab,
                                                             int32_t *__restrict__ block_cnt) {
    __shared__ int s_w[kRelThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kRelBlock;
    int c = 0;
#pragma unroll 4
    for (int u = 0; u < kRelPerThread; ++u) {
        const int64_t i = base + (int64_t)u * kRelThreads + threadIdx.x;
        if (i < n) c += __ldg(lab + i) == (int32_t)i;
    }
    c = __reduce_add_sync(kFull, c);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kRelThreads / 32; ++w) t += s_w[w];
        block_cnt[blockIdx.x] = t;
    }
}

// exclusive scan of the block counts in place (one CTA); *total = sum
__global__ void __launch_bounds__(1024) k_scan_counts(int32_t nb, int32_t *__restrict__ cnt,
                                                      int32_t *__restrict__ total) {
    __shared__ int32_t s_part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = min((int)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
    int32_t part = 0;
    for (int b = b0; b < b1; ++b) part += cnt[b];
    s_part[threadIdx.x] = part;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {         // Hillis-Steele inclusive scan
        const int32_t v = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t acc = s_part[threadIdx.x] - part;
    for (int b = b0; b < b1; ++b) {
        const int32_t c = cnt[b];
        cnt[b] = acc;
        acc += c;
    }
    if (threadIdx.x == 1023) *total = s_part[1023];
}

// sequential id of every root: its block's offset plus the roots before it in
// the block, in site order; zeroes the size counter of each id
__global__ void __launch_bounds__(kRelThreads) k_root_ids(int32_t n, const int32_t *__restrict__ lab,
                                                          const int32_t *__restrict__ block_off,
                                                          int32_t *__restrict__ out, int32_t *__restrict__ sizes) {
    __shared__ int32_t s_w[kRelThreads / 32];
    __shared__ int32_t s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kRelBlock;
    if (threadIdx.x == 0) s_run = block_off[blockIdx.x];
    __syncthreads();
    for (int u = 0; u < kRelPerThread; ++u) {
        const int64_t i = base + (int64_t)u * kRelThreads + threadIdx.x;
        const bool root = i < n && __ldg(lab + i) == (int32_t)i;
        const unsigned b = __ballot_sync(kFull, root);
        if (lane == 0) s_w[warp] = __popc(b);
        __syncthreads();
        int before = s_run;
        for (int w = 0; w < warp; ++w) before += s_w[w];
        if (root) {
            const int32_t id = before + __popc(b & ((1u << lane) - 1u));
            out[i] = id;
            if (sizes) sizes[id] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < kRelThreads / 32; ++w) t += s_w[w];
            s_run += t;
        }
        __syncthreads();
    }
}

// every other site takes its root's id
__global__ void k_site_ids(int32_t n, const int32_t *__restrict__ lab, int32_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t l = __ldg(lab + i);
        if (l != (int32_t)i) out[i] = out[l];
    }
}

// cluster sizes; lanes of a warp holding the same id add once
__global__ void k_sizes(int32_t n, const int32_t *__restrict__ out, int32_t *__restrict__ sizes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const int32_t id = i < n ? out[i] : -1;
        const unsigned peers = __match_any_sync(kFull, id);
        if (id >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(sizes + id, __popc(peers));
    }
}

// spanning: mark the labels of the top sites, then look for them at the bottom
__global__ void k_span_mark(int32_t n, const int32_t *__restrict__ lab, const int32_t *__restrict__ top,
                            int32_t n_top, uint32_t *__restrict__ flags, int32_t *__restrict__ best,
                            unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_top; t += stride) {
        const int32_t s = top[t];
        if ((uint32_t)s >= (uint32_t)n) { atomicOr(err, kErrIndex); continue; }
        const int32_t l = lab[s];
        if ((uint32_t)l >= (uint32_t)n) { atomicOr(err, kErrIndex); continue; }
        atomicOr(flags + (l >> 5), 1u << (l & 31));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *best = INT32_MAX;
}

__global__ void k_span_check(int32_t n, const int32_t *__restrict__ lab, const int32_t *__restrict__ bottom,
                             int32_t n_bottom, const uint32_t *__restrict__ flags, int32_t *__restrict__ best,
                             unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_bottom; t += stride) {
        const int32_t s = bottom[t];
        if ((uint32_t)s >= (uint32_t)n) { atomicOr(err, kErrIndex); continue; }
        const int32_t l = lab[s];
        if ((uint32_t)l >= (uint32_t)n) { atomicOr(err, kErrIndex); continue; }
        if ((__ldg(flags + (l >> 5)) >> (l & 31)) & 1u) atomicMin(best, l);
    }
}

__global__ void k_span_finish(int32_t *best) {
    if (*best == INT32_MAX) *best = -1;
}

// Largest cluster (Section 4's largest-cluster statistic): cnt[l] = sites
// whose canonical label is l (lanes holding the same label add once), then the
// largest count over the roots, ties to the smallest label, as one 64-bit key
// (count << 32) | (0xffffffff - label) under atomicMax.
__global__ void k_label_counts(int32_t n, const int32_t *__restrict__ lab, int32_t *__restrict__ cnt,
                               unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        int32_t l = i < n ? __ldg(lab + i) : -1;
        if (i < n && (uint32_t)l >= (uint32_t)n) { atomicOr(err, kErrIndex); l = -1; }
        const unsigned peers = __match_any_sync(kFull, l);
        if (l >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(cnt + l, __popc(peers));
    }
}

__global__ void k_largest(int32_t n, const int32_t *__restrict__ cnt, unsigned long long *__restrict__ best) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long key = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t c = __ldg(cnt + i);
        if (c > 0) {
            const unsigned long long k = ((unsigned long long)(uint32_t)c << 32) | (0xffffffffu - (uint32_t)i);
            key = k > key ? k : key;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, key, o);
        key = t > key ? t : key;
    }
    if ((threadIdx.x & 31) == 0 && key) atomicMax(best, key);
}

__global__ void k_largest_finish(const unsigned long long *best, int32_t *result) {
    const unsigned long long k = *best;
    result[0] = (int32_t)(k >> 32);
    result[1] = k ? (int32_t)(0xffffffffu - (uint32_t)(k & 0xffffffffu)) : -1;
}

}  // namespace ccl
