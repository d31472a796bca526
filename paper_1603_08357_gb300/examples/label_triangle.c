/*
 * label_triangle.c -- using libccl.so from C, with no Python.
 *
 * Builds bond percolation on an L x L triangle lattice (periodic, bonds to
 * (x+1,y), (x,y+1), (x+1,y+1), each open with probability p) as a CSR
 * neighbour list with one open bit per entry, labels its clusters on the GPU
 * with ccl_label, and checks the result against a union-find on the host:
 * every site's label must be the smallest site of its cluster.
 *
 *   cc -O2 -I<repo>/include label_triangle.c -L<lib dir> -lccl \
 *      -L<cuda>/lib64 -lcudart -Wl,-rpath,<lib dir> -o label_triangle
 *   ./label_triangle [L] [p]
 */
#include <ccl.h>
#include <cuda_runtime.h>

#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

static uint64_t rng_state = 0x243F6A8885A308D3ull;
static double uniform(void) {          /* xorshift64*, enough for an example */
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (double)((rng_state * 0x2545F4914F6CDD1Dull) >> 11) * 0x1.0p-53;
}

static int32_t find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

#define CHECK_CUDA(call)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                  \
            return 2;                                                                    \
        }                                                                                \
    } while (0)

int main(int argc, char **argv) {
    const int32_t L = argc > 1 ? atoi(argv[1]) : 512;
    const double p = argc > 2 ? atof(argv[2]) : 0.3473;
    const int32_t n = L * L;
    const int64_t nnz = 6 * (int64_t)n;
    const int64_t nwords = (nnz + 31) / 32;

    /* bond b = 3*i + d of site i = y*L + x, d: 0 -> (x+1,y), 1 -> (x,y+1), 2 -> (x+1,y+1) */
    unsigned char *open = malloc((size_t)3 * n);
    for (int64_t b = 0; b < 3 * (int64_t)n; ++b) open[b] = uniform() < p;

    int32_t *row_ptr = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *col_idx = malloc(sizeof(int32_t) * (size_t)nnz);
    uint32_t *bits = calloc((size_t)nwords, sizeof(uint32_t));
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t x = i % L, y = i / L;
        const int32_t xp = (x + 1) % L, xm = (x + L - 1) % L, yp = (y + 1) % L, ym = (y + L - 1) % L;
        const int32_t nb[6] = {y * L + xp, yp * L + x, yp * L + xp, y * L + xm, ym * L + x, ym * L + xm};
        const int64_t bond[6] = {3 * (int64_t)i, 3 * (int64_t)i + 1, 3 * (int64_t)i + 2,
                                 3 * (int64_t)(y * L + xm), 3 * (int64_t)(ym * L + x) + 1,
                                 3 * (int64_t)(ym * L + xm) + 2};
        row_ptr[i] = (int32_t)e;
        for (int t = 0; t < 6; ++t, ++e) {
            col_idx[e] = nb[t];
            if (open[bond[t]]) bits[e >> 5] |= 1u << (e & 31);
        }
    }
    row_ptr[n] = (int32_t)e;

    int32_t *d_rp, *d_ci, *d_lab;
    uint32_t *d_bits;
    CHECK_CUDA(cudaMalloc((void **)&d_rp, sizeof(int32_t) * (size_t)(n + 1)));
    CHECK_CUDA(cudaMalloc((void **)&d_ci, sizeof(int32_t) * (size_t)nnz));
    CHECK_CUDA(cudaMalloc((void **)&d_bits, sizeof(uint32_t) * (size_t)nwords));
    CHECK_CUDA(cudaMalloc((void **)&d_lab, sizeof(int32_t) * (size_t)n));
    CHECK_CUDA(cudaMemcpy(d_rp, row_ptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d_ci, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d_bits, bits, sizeof(uint32_t) * (size_t)nwords, cudaMemcpyHostToDevice));

    ccl_context *ctx = NULL;
    ccl_status st = ccl_context_create(&ctx, 0);
    if (st == CCL_OK) st = ccl_label(ctx, n, nnz, d_rp, d_ci, d_bits, d_lab, NULL);
    if (st == CCL_OK) st = ccl_sync(ctx, NULL, -1);
    if (st != CCL_OK) {
        fprintf(stderr, "ccl: %s\n", ccl_status_string(st));
        return 1;
    }
    int32_t *labels = malloc(sizeof(int32_t) * (size_t)n);
    CHECK_CUDA(cudaMemcpy(labels, d_lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost));

    /* host check: union-find over the open bonds, then the least site of each set */
    int32_t *parent = malloc(sizeof(int32_t) * (size_t)n), *least = malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) parent[i] = i;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t x = i % L, y = i / L;
        const int32_t nb[3] = {y * L + (x + 1) % L, ((y + 1) % L) * L + x, ((y + 1) % L) * L + (x + 1) % L};
        for (int d = 0; d < 3; ++d) {
            if (!open[3 * (int64_t)i + d]) continue;
            const int32_t a = find(parent, i), b = find(parent, nb[d]);
            if (a != b) parent[a] = b;
        }
    }
    for (int32_t i = 0; i < n; ++i) least[i] = n;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t r = find(parent, i);
        if (i < least[r]) least[r] = i;
    }
    int64_t wrong = 0, clusters = 0;
    for (int32_t i = 0; i < n; ++i) {
        wrong += labels[i] != least[find(parent, i)];
        clusters += labels[i] == i;
    }
    printf("L=%d p=%.4f sites=%d clusters=%lld mismatches=%lld %s\n", L, p, n, (long long)clusters,
           (long long)wrong, wrong ? "FAIL" : "ok");

    ccl_context_destroy(ctx);
    cudaFree(d_rp);
    cudaFree(d_ci);
    cudaFree(d_bits);
    cudaFree(d_lab);
    free(open); free(row_ptr); free(col_idx); free(bits); free(labels); free(parent); free(least);
    return wrong ? 1 : 0;
}
