/*
 * CPU oracle for bond-percolation cluster labelling -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file. It shares no code with the CUDA library and the library never
 * calls it.
 *
 * Problem (Section 3): sites 0..n-1 carry a nearest-neighbour list, here in
 * CSR form (row_ptr[n+1], col_idx[nnz]) with one open/closed bit per entry
 * (entry e of the instance is bit bit_off + e of `bits`, word >> 5, bit & 31).
 * Only an entry j < i of row i is read, so the bond {i, j} is decided by the
 * bit stored in row max(i, j); self-loops and duplicate entries are allowed.
 * The result (end of Section 3) is the canonical label
 *     label[v] = min { u : u is connected to v through open bonds },
 * the smallest site number of v's cluster.
 *
 * Three independent routines compute it:
 *   oracle_uf_label    weighted union-find (union by size, path halving) over
 *                      the open bonds, then the minimum member per root;
 *   oracle_bfs_label   breadth-first search from each unvisited site in
 *                      ascending order, so the seed is its cluster's minimum;
 *   oracle_steps_label the four steps of Section 3 executed one after the
 *                      other on one core: (i) initialisation with residual
 *                      lists, (ii) analysis, (iii) label reduction of
 *                      Algorithm 1, (iv) analysis. It also returns the
 *                      intermediate label arrays and the residual lists, which
 *                      the tests check by hand on a worked example.
 *
 * Return value of every routine: 0 on success, -1 if a row pointer or a
 * column index is out of range, -2 on allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int bit_at(const uint32_t *bits, int64_t g) {
    return (int)((bits[g >> 5] >> (g & 31)) & 1u);
}

static int check_csr(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx) {
    if (n < 0 || nnz < 0) return -1;
    if (row_ptr[0] != 0 || row_ptr[n] != nnz) return -1;
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return -1;
    for (int64_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= n) return -1;
    return 0;
}

/* ---------------- O1: weighted union-find --------------------------------- */

static int32_t uf_find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {           /* path halving */
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

int oracle_uf_label(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                    const uint32_t *bits, int64_t bit_off, int32_t *label) {
    if (check_csr(n, nnz, row_ptr, col_idx)) return -1;
    if (n == 0) return 0;
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *minv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!parent || !size || !minv) { free(parent); free(size); free(minv); return -2; }
    for (int32_t v = 0; v < n; ++v) { parent[v] = v; size[v] = 1; minv[v] = -1; }
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i && bit_at(bits, bit_off + e)) {
                int32_t a = uf_find(parent, i), b = uf_find(parent, j);
                if (a == b) continue;
                if (size[a] < size[b]) { int32_t t = a; a = b; b = t; }
                parent[b] = a;
                size[a] += size[b];
            }
        }
    }
    /* ascending sweep: the first member met of each root is its minimum */
    for (int32_t v = 0; v < n; ++v) {
        int32_t r = uf_find(parent, v);
        if (minv[r] < 0) minv[r] = v;
        label[v] = minv[r];
    }
    free(parent); free(size); free(minv);
    return 0;
}

/* ---------------- O2: breadth-first search ---------------------------------- */

int oracle_bfs_label(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                     const uint32_t *bits, int64_t bit_off, int32_t *label) {
    if (check_csr(n, nnz, row_ptr, col_idx)) return -1;
    if (n <= 0) return 0;
    /* adjacency of the open bond set, both directions */
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -2;
    int64_t nb = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i && bit_at(bits, bit_off + e)) { deg[i + 1]++; deg[j + 1]++; nb++; }
        }
    for (int32_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    const size_t un = (size_t)(uint32_t)n;
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nb + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * un);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * un);
    if (!adj || !fill || !queue) { free(deg); free(adj); free(fill); free(queue); return -2; }
    for (int32_t v = 0; v < n; ++v) fill[v] = deg[v];
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i && bit_at(bits, bit_off + e)) { adj[fill[i]++] = j; adj[fill[j]++] = i; }
        }
    for (int32_t v = 0; v < n; ++v) label[v] = -1;
    for (int32_t s = 0; s < n; ++s) {
        if (label[s] >= 0) continue;
        int32_t head = 0, tail = 0;
        label[s] = s; queue[tail++] = s;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int64_t t = deg[v]; t < deg[v + 1]; ++t) {
                int32_t w = adj[t];
                if (label[w] < 0) { label[w] = s; queue[tail++] = w; }
            }
        }
    }
    free(deg); free(adj); free(fill); free(queue);
    return 0;
}

/* ---------------- the four steps of Section 3, sequentially ----------------- */

/* analysis: every site follows label[label[i]] until it stops changing */
static void analysis(int32_t n, int32_t *label) {
    for (int32_t i = 0; i < n; ++i)
        while (label[i] != label[label[i]]) label[i] = label[label[i]];
}

/* label reduction for one pair (i, j), Algorithm 1 with atomicMin executed as a
 * plain read-then-minimum (there is only one executor here) */
static void reduce_pair(int32_t *label, int32_t i, int32_t j) {
    int32_t l1 = label[i];
    while (l1 != label[l1]) l1 = label[l1];
    int32_t l2 = label[j];
    while (l2 != label[l2]) l2 = label[l2];
    int flag = (l1 == l2);
    if (l1 < l2) { int32_t t = l1; l1 = l2; l2 = t; }
    while (!flag) {
        int32_t l3 = label[l1];                 /* atomicMin(&label[l1], l2) */
        if (l2 < l3) label[l1] = l2;
        if (l3 == l2) flag = 1;
        else if (l3 > l2) l1 = l3;
        else { l1 = l2; l2 = l3; }
    }
}

/*
 * Runs steps (i)-(iv). Outputs (each optional except `label`):
 *   after_init[n], after_ii[n], after_iii[n]: label array after those steps;
 *   res_ptr[n+1], res_j[nnz]: the residual list of every site after step (i),
 *   in row order (the open lower neighbours with one occurrence of the
 *   minimum removed);
 *   n_residual: total length of the residual lists.
 */
int oracle_steps_label(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                       const uint32_t *bits, int64_t bit_off, int32_t *label,
                       int32_t *after_init, int32_t *after_ii, int32_t *after_iii,
                       int64_t *res_ptr, int32_t *res_j, int64_t *n_residual) {
    if (check_csr(n, nnz, row_ptr, col_idx)) return -1;
    int64_t *rp = res_ptr ? res_ptr : (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *rj = res_j ? res_j : (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    if (!rp || !rj) { if (!res_ptr) free(rp); if (!res_j) free(rj); return -2; }
    /* (i) initialisation */
    int64_t q = 0;
    rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t mn = -1; int64_t mpos = -1;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i && bit_at(bits, bit_off + e) && (mn < 0 || j < mn)) { mn = j; mpos = e; }
        }
        label[i] = (mn < 0) ? i : mn;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i && bit_at(bits, bit_off + e) && e != mpos) rj[q++] = j;
        }
        rp[i + 1] = q;
    }
    if (after_init) memcpy(after_init, label, sizeof(int32_t) * (size_t)n);
    /* (ii) analysis */
    analysis(n, label);
    if (after_ii) memcpy(after_ii, label, sizeof(int32_t) * (size_t)n);
    /* (iii) label reduction: every site, every entry of its residual list */
    for (int32_t i = 0; i < n; ++i)
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) reduce_pair(label, i, rj[t]);
    if (after_iii) memcpy(after_iii, label, sizeof(int32_t) * (size_t)n);
    /* (iv) analysis */
    analysis(n, label);
    if (n_residual) *n_residual = q;
    if (!res_ptr) free(rp);
    if (!res_j) free(rj);
    return 0;
}

/* ---------------- bonds drawn from a counter-based generator ----------------- */

/* SplitMix64 (Steele, Lea & Flood 2014; the reference implementation adds
 * 0x9E3779B97F4A7C15 to the state and mixes): output number k (k >= 0) of the
 * generator started from state `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The realisation a graph gets when its bonds are drawn from (seed, p): the
 * bond {lo, hi} is open iff (output number lo * 2^32 + hi) >> 11, scaled by
 * 2^-53, is below p. Writes one bit per CSR entry (both copies of a bond get
 * the same bit). bits must hold ceil(nnz / 32) zeroed words. */
int oracle_keyed_bits(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                      uint64_t seed, double p, uint32_t *bits) {
    if (check_csr(n, nnz, row_ptr, col_idx)) return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col_idx[e];
            const uint64_t lo = (uint64_t)(j < i ? j : i), hi = (uint64_t)(j < i ? i : j);
            const uint64_t out = oracle_splitmix64(seed, (lo << 32) | hi);
            if ((double)(out >> 11) * 0x1.0p-53 < p) bits[e >> 5] |= 1u << (e & 31);
        }
    return 0;
}

/* ---------------- batched: K instances in concatenated form ------------------ */

/* Instance k: sites [site_off[k], site_off[k+1]), local row pointers at
 * row_ptr + site_off[k] + k, entries [ent_off[k], ent_off[k+1]) of col_idx,
 * bits at global bit ent_off[k] + e. Labels are instance-local. Instances
 * [k0, k1) only. */
int oracle_uf_label_batched(int32_t k0, int32_t k1, const int64_t *site_off, const int64_t *ent_off,
                            const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *bits,
                            int32_t *labels) {
    for (int32_t k = k0; k < k1; ++k) {
        int64_t s0 = site_off[k], e0 = ent_off[k];
        int32_t n = (int32_t)(site_off[k + 1] - s0);
        int64_t nnz = ent_off[k + 1] - e0;
        int rc = oracle_uf_label(n, nnz, row_ptr + s0 + k, col_idx + e0, bits, e0, labels + s0);
        if (rc) return rc;
    }
    return 0;
}
