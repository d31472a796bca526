/*
 * Seeded synthetic inputs for bond-percolation labelling: neighbour lists of
 * the honeycomb, triangle and Bethe (Cayley tree) lattices of Section 4, in
 * CSR form, plus one open/closed bit per CSR entry.
 *
 * This module holds none of the labelling method's arithmetic. It is shared
 * by the CPU oracle and the CUDA path purely as a source of inputs.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used in counter form: output number k
 * (k = 0, 1, ...) of the generator started from state `seed` is
 *     mix(seed + (k + 1) * 0x9E3779B97F4A7C15).
 * Bond b is open iff (out(seed, b) >> 11) * 2^-53 < p, an exact double
 * comparison. Both CSR directions of a bond carry the bond's one id, so the
 * two bits always agree. (The paper drew its bonds with cuRAND XORWOW in
 * double precision; the statistics, not the stream, are what Section 4 uses.)
 *
 * Lattices (geometry and numbering are not stated in the paper; these are the
 * readings used throughout):
 *   honeycomb(L): L x L unit cells c = y*L + x, sites A = 2c and B = 2c + 1.
 *                 Bond 3c   : A(x,y) - B(x,y)
 *                 Bond 3c+1 : A(x,y) - B(x-1,y)
 *                 Bond 3c+2 : A(x,y) - B(x,y-1)
 *                 N = 2 L^2, 3 L^2 bonds when periodic in both directions.
 *   triangle(L):  L x L sites i = y*L + x.
 *                 Bond 3i   : (x,y) - (x+1,y)
 *                 Bond 3i+1 : (x,y) - (x,y+1)
 *                 Bond 3i+2 : (x,y) - (x+1,y+1)
 *                 N = L^2, 3 L^2 bonds, coordination 6 when periodic.
 *   cayley(z,S):  a centre site (index 0) with z children, every other
 *                 interior site with z-1 children, S shells, numbered shell
 *                 by shell from the centre ("standard position"). The bond
 *                 between a site s > 0 and its parent has id s - 1.
 *                 "Random position" stores standard site s at index perm[s].
 *   square(L):    L x L sites i = y*L + x (the 2D lattice the four steps were
 *                 first written for). Bond 2i : (x,y) - (x+1,y)
 *                                     Bond 2i+1 : (x,y) - (x,y+1)
 *   cubic(L):     L^3 sites i = (z*L + y)*L + x (simple cubic).
 *                 Bond 3i + d : i - (its neighbour one step up along axis d,
 *                 d = 0: x, 1: y, 2: z)
 * x is always periodic; y (z for cubic) is periodic unless periodic_y == 0,
 * in which case bonds that would wrap in that direction are absent (the
 * spanning direction). cubic's y is always periodic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t lat_splitmix64(uint64_t seed, uint64_t k) {
    return sm64_mix(seed + (k + 1) * GOLDEN_GAMMA);
}

int lat_bond_open(uint64_t seed, uint64_t bond, double p) {
    uint64_t h = lat_splitmix64(seed, bond);
    return (double)(h >> 11) * 0x1.0p-53 < p;
}

enum { LAT_HONEYCOMB = 0, LAT_TRIANGLE = 1, LAT_CAYLEY = 2, LAT_SQUARE = 3, LAT_CUBIC = 4 };

typedef struct {
    int32_t kind;
    int32_t L;            /* honeycomb / triangle size */
    int32_t periodic_y;
    int32_t z;            /* cayley coordination */
    int32_t shells;       /* cayley shell count */
    int32_t pad_;
    const int32_t *perm;      /* cayley: standard index -> stored index, or NULL */
    const int32_t *perm_inv;  /* cayley: stored index -> standard index, or NULL */
    int64_t n;            /* number of sites */
} lat_desc;

/* ---- Cayley tree shell arithmetic ---------------------------------------- */

/* first standard index of shell k (shell 0 is the centre) */
static int64_t cay_shell_start(int32_t z, int32_t k) {
    if (k == 0) return 0;
    int64_t start = 1, size = z;
    for (int32_t s = 1; s < k; ++s) { start += size; size *= (z - 1); }
    return start;
}

int64_t lat_cayley_nsites(int32_t z, int32_t shells) {
    return cay_shell_start(z, shells + 1);
}

/* neighbours of standard site s: parent first (if any), then children */
static int cay_neighbors_std(int32_t z, int32_t shells, int64_t s,
                             int64_t *nb, int64_t *bond) {
    int cnt = 0;
    if (s == 0) {
        if (shells >= 1)
            for (int c = 0; c < z; ++c) { nb[cnt] = 1 + c; bond[cnt] = c; ++cnt; }
        return cnt;
    }
    /* locate the shell of s */
    int32_t k = 1; int64_t start = 1, size = z;
    while (s >= start + size) { start += size; size *= (z - 1); ++k; }
    int64_t off = s - start;
    int64_t parent = (k == 1) ? 0 : cay_shell_start(z, k - 1) + off / (z - 1);
    nb[cnt] = parent; bond[cnt] = s - 1; ++cnt;
    if (k < shells) {
        int64_t cstart = start + size + off * (z - 1);
        for (int c = 0; c < z - 1; ++c) {
            nb[cnt] = cstart + c; bond[cnt] = cstart + c - 1; ++cnt;
        }
    }
    return cnt;
}

/* ---- generic neighbour enumeration ---------------------------------------- */

#define MAXNB 64

static int neighbors(const lat_desc *d, int64_t i, int64_t *nb, int64_t *bond) {
    if (d->kind == LAT_HONEYCOMB) {
        int64_t L = d->L, c = i >> 1;
        int64_t x = c % L, y = c / L;
        int cnt = 0;
        if ((i & 1) == 0) { /* A(x,y) */
            nb[cnt] = 2 * c + 1; bond[cnt] = 3 * c; ++cnt;
            nb[cnt] = 2 * (y * L + (x + L - 1) % L) + 1; bond[cnt] = 3 * c + 1; ++cnt;
            if (d->periodic_y || y > 0) {
                nb[cnt] = 2 * (((y + L - 1) % L) * L + x) + 1; bond[cnt] = 3 * c + 2; ++cnt;
            }
        } else {            /* B(x,y) */
            int64_t cr = y * L + (x + 1) % L;
            int64_t cu = ((y + 1) % L) * L + x;
            nb[cnt] = 2 * c; bond[cnt] = 3 * c; ++cnt;
            nb[cnt] = 2 * cr; bond[cnt] = 3 * cr + 1; ++cnt;
            if (d->periodic_y || y < L - 1) {
                nb[cnt] = 2 * cu; bond[cnt] = 3 * cu + 2; ++cnt;
            }
        }
        return cnt;
    }
    if (d->kind == LAT_TRIANGLE) {
        int64_t L = d->L, x = i % L, y = i / L;
        int64_t xp = (x + 1) % L, xm = (x + L - 1) % L;
        int64_t yp = (y + 1) % L, ym = (y + L - 1) % L;
        int up = d->periodic_y || y < L - 1, dn = d->periodic_y || y > 0;
        int cnt = 0;
        nb[cnt] = y * L + xp; bond[cnt] = 3 * i; ++cnt;
        if (up) { nb[cnt] = yp * L + x;  bond[cnt] = 3 * i + 1; ++cnt; }
        if (up) { nb[cnt] = yp * L + xp; bond[cnt] = 3 * i + 2; ++cnt; }
        nb[cnt] = y * L + xm; bond[cnt] = 3 * (y * L + xm); ++cnt;
        if (dn) { nb[cnt] = ym * L + x;  bond[cnt] = 3 * (ym * L + x) + 1; ++cnt; }
        if (dn) { nb[cnt] = ym * L + xm; bond[cnt] = 3 * (ym * L + xm) + 2; ++cnt; }
        return cnt;
    }
    if (d->kind == LAT_SQUARE) {
        int64_t L = d->L, x = i % L, y = i / L;
        int cnt = 0;
        nb[cnt] = y * L + (x + 1) % L; bond[cnt] = 2 * i; ++cnt;
        if (d->periodic_y || y < L - 1) { nb[cnt] = ((y + 1) % L) * L + x; bond[cnt] = 2 * i + 1; ++cnt; }
        int64_t l = y * L + (x + L - 1) % L;
        nb[cnt] = l; bond[cnt] = 2 * l; ++cnt;
        if (d->periodic_y || y > 0) {
            int64_t dn = ((y + L - 1) % L) * L + x;
            nb[cnt] = dn; bond[cnt] = 2 * dn + 1; ++cnt;
        }
        return cnt;
    }
    if (d->kind == LAT_CUBIC) {
        int64_t L = d->L, x = i % L, y = (i / L) % L, z = i / (L * L);
        int64_t c[3] = {x, y, z}, stride[3] = {1, L, L * L};
        int cnt = 0;
        for (int a = 0; a < 3; ++a) {       /* upward neighbours: bond 3i + a */
            if (a == 2 && !d->periodic_y && z == L - 1) continue;
            int64_t j = i + (((c[a] + 1) % L) - c[a]) * stride[a];
            nb[cnt] = j; bond[cnt] = 3 * i + a; ++cnt;
        }
        for (int a = 0; a < 3; ++a) {       /* downward neighbours: their bond 3j + a */
            if (a == 2 && !d->periodic_y && z == 0) continue;
            int64_t j = i + (((c[a] + L - 1) % L) - c[a]) * stride[a];
            nb[cnt] = j; bond[cnt] = 3 * j + a; ++cnt;
        }
        return cnt;
    }
    /* Cayley tree, optionally stored under a permutation */
    int64_t s = d->perm_inv ? d->perm_inv[i] : i;
    int cnt = cay_neighbors_std(d->z, d->shells, s, nb, bond);
    if (d->perm)
        for (int t = 0; t < cnt; ++t) nb[t] = d->perm[nb[t]];
    return cnt;
}

int lat_site_degree(const lat_desc *d, int64_t i) {
    int64_t nb[MAXNB], bond[MAXNB];
    return neighbors(d, i, nb, bond);
}

/* ---- parallel fill ---------------------------------------------------------- */

typedef struct {
    const lat_desc *d;
    int64_t r0, r1;        /* row range */
    int32_t *row_ptr;      /* [n+1], already holds the prefix (phase 2) */
    int32_t *col_idx;
    uint32_t *bits;
    int64_t bit_off;
    uint64_t seed;
    double p;
    int phase;             /* 1: degrees into row_ptr[i+1]; 2: entries */
    int64_t open_lower;    /* phase 2: number of open bonds counted once */
} fill_job;

static void flush_word(uint32_t *bits, int64_t w, uint32_t v, int shared) {
    if (!v) return;
    if (shared) __atomic_fetch_or(&bits[w], v, __ATOMIC_RELAXED);
    else bits[w] |= v;
}

static void *fill_worker(void *arg) {
    fill_job *J = (fill_job *)arg;
    int64_t nb[MAXNB], bond[MAXNB];
    if (J->phase == 1) {
        for (int64_t i = J->r0; i < J->r1; ++i)
            J->row_ptr[i + 1] = neighbors(J->d, i, nb, bond);
        return NULL;
    }
    if (J->r0 >= J->r1) return NULL;
    int64_t e0 = J->row_ptr[J->r0], e1 = J->row_ptr[J->r1];
    int64_t gfirst = J->bit_off + e0, glast = J->bit_off + e1 - 1;
    int64_t wfirst = gfirst >> 5, wlast = glast >> 5;
    int64_t cur_w = -1; uint32_t cur_v = 0;
    int64_t open_lower = 0;
    for (int64_t i = J->r0; i < J->r1; ++i) {
        int cnt = neighbors(J->d, i, nb, bond);
        int64_t e = J->row_ptr[i];
        for (int t = 0; t < cnt; ++t, ++e) {
            J->col_idx[e] = (int32_t)nb[t];
            if (lat_bond_open(J->seed, (uint64_t)bond[t], J->p)) {
                int64_t g = J->bit_off + e, w = g >> 5;
                if (w != cur_w) {
                    if (cur_w >= 0) flush_word(J->bits, cur_w, cur_v, cur_w == wfirst || cur_w == wlast);
                    cur_w = w; cur_v = 0;
                }
                cur_v |= 1u << (g & 31);
                if (nb[t] < i) ++open_lower;
            }
        }
    }
    if (cur_w >= 0) flush_word(J->bits, cur_w, cur_v, cur_w == wfirst || cur_w == wlast);
    J->open_lower = open_lower;
    return NULL;
}

static void run_jobs(fill_job *jobs, int nt) {
    if (nt == 1) { fill_worker(&jobs[0]); return; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, fill_worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    free(th);
}

/* Number of CSR entries of the lattice (sum of degrees). */
int64_t lat_count_entries(const lat_desc *d) {
    int64_t n = d->n;
    if (d->kind != LAT_CAYLEY) {
        int64_t tot = 0;
        for (int64_t i = 0; i < n; ++i) tot += lat_site_degree(d, i);
        return tot;
    }
    return 2 * (n - 1);
}

/*
 * Fill row_ptr[n+1] (local entry indices), col_idx[nnz] and the bits of
 * entries 0..nnz-1 at global bit positions bit_off + e of `bits` (which the
 * caller has zeroed). Returns nnz, or -1 if it exceeds nnz_cap. `open_bonds`
 * (optional) receives the number of open bonds, each counted once.
 */
int64_t lat_fill(const lat_desc *d, uint64_t seed, double p,
                 int32_t *row_ptr, int32_t *col_idx, int64_t nnz_cap,
                 uint32_t *bits, int64_t bit_off, int nthreads,
                 int64_t *open_bonds) {
    int64_t n = d->n;
    if (nthreads < 1) nthreads = 1;
    if (n < 4096) nthreads = 1;
    fill_job *jobs = (fill_job *)calloc(nthreads, sizeof(fill_job));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].d = d; jobs[t].row_ptr = row_ptr; jobs[t].col_idx = col_idx;
        jobs[t].bits = bits; jobs[t].bit_off = bit_off; jobs[t].seed = seed; jobs[t].p = p;
        jobs[t].r0 = n * t / nthreads; jobs[t].r1 = n * (t + 1) / nthreads;
        jobs[t].phase = 1;
    }
    run_jobs(jobs, nthreads);
    row_ptr[0] = 0;
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        acc += row_ptr[i + 1];
        if (acc > nnz_cap || acc > INT32_MAX) { free(jobs); return -1; }
        row_ptr[i + 1] = (int32_t)acc;
    }
    for (int t = 0; t < nthreads; ++t) jobs[t].phase = 2;
    run_jobs(jobs, nthreads);
    int64_t open = 0;
    for (int t = 0; t < nthreads; ++t) open += jobs[t].open_lower;
    if (open_bonds) *open_bonds = open;
    free(jobs);
    return acc;
}

/* Copies n_bits bits from bit position src_off of src to bit position dst_off
 * of dst (dst words outside the copied range keep their other bits). */
void lat_copy_bits(const uint32_t *src, int64_t src_off, int64_t n_bits, uint32_t *dst,
                   int64_t dst_off) {
    for (int64_t t = 0; t < n_bits; ++t) {
        const int64_t gs = src_off + t, gd = dst_off + t;
        const uint32_t bit = (src[gs >> 5] >> (gs & 31)) & 1u;
        if (bit) dst[gd >> 5] |= 1u << (gd & 31);
        else dst[gd >> 5] &= ~(1u << (gd & 31));
    }
}

/* Seeded uniform permutation by Fisher-Yates; the swap index for position i
 * (i = n-1 .. 1) is floor(out * (i+1) / 2^64) with out = SplitMix64 output
 * number n-1-i from `seed`. perm[s] = stored index of standard site s. */
void lat_permutation(int64_t n, uint64_t seed, int32_t *perm, int32_t *perm_inv) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i >= 1; --i) {
        uint64_t h = lat_splitmix64(seed, (uint64_t)(n - 1 - i));
        int64_t j = (int64_t)(((unsigned __int128)h * (uint64_t)(i + 1)) >> 64);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    if (perm_inv)
        for (int64_t s = 0; s < n; ++s) perm_inv[perm[s]] = (int32_t)s;
}
