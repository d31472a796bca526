/*
 * ccl.h -- C ABI of the GB300 (sm_103a) cluster-labelling library.
 *
 * The library labels the clusters of open bonds on an arbitrary site graph
 * given as a nearest-neighbour list, by the four-step generalized method of
 * Komura, "A generalized GPU-based connected component labeling algorithm"
 * (arXiv 1603.08357), Section 3:
 *   (i)   initialisation: label[i] = smallest open neighbour numbered below i,
 *         or i; the other open lower neighbours form i's residual list;
 *   (ii)  analysis: label[i] = label[label[i]] until it stops changing;
 *   (iii) label reduction (Algorithm 1): for every residual pair, follow both
 *         label chains to their roots and merge them with atomicMin;
 *   (iv)  analysis again.
 * The result is the canonical cluster label of Section 3: label[v] is the
 * smallest site number of v's cluster. It is unique, so any correct run gives
 * the same bits.
 *
 * Sizes: n <= CCL_MAX_SITES sites per instance (2^31 - 4097: the kernels
 * number sites in 32-bit integers and keep that much headroom above the last
 * site), nnz < 2^31 CSR entries per instance.
 *
 * Input format (the "NN list" of Section 3, here in CSR form):
 *   row_ptr[n+1]  int32, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz;
 *   col_idx[nnz]  int32 neighbour site numbers in [0, n);
 *   open_bits     uint32 words, at least ceil(nnz/32); bit e (word e >> 5,
 *                 bit e & 31) is 1 iff the bond of CSR entry e is open.
 * Only an entry j < i of row i is read, so the bond {i, j} is decided by the
 * bit stored in row max(i, j). Self-loops are ignored; duplicate entries are
 * allowed. A symmetric list (j in row i <=> i in row j, equal bits) is the
 * normal case; ccl_validate checks it.
 *
 * Ownership: every array argument belongs to the caller. The library
 * allocates device memory only inside a ccl_context (its workspace) or a
 * ccl_server. Streams are passed as `void*` holding a cudaStream_t
 * (NULL = the legacy default stream); the library never synchronises a
 * caller's stream except in the calls documented as synchronous.
 *
 * Errors: argument errors are returned synchronously. Errors found by the
 * kernels (an index out of range, an inconsistent row_ptr, a loop that hit its
 * iteration cap) are latched in a per-context device word and returned by
 * ccl_sync. No function aborts, traps or prints.
 */
#ifndef CCL_H_
#define CCL_H_

#include <stdint.h>

#if defined(__GNUC__)
#define CCL_API __attribute__((visibility("default")))
#else
#define CCL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCL_OK = 0,
    CCL_ERR_INVALID_ARGUMENT = 1,   /* bad pointer/size, or row_ptr[n] != nnz */
    CCL_ERR_INDEX_OUT_OF_RANGE = 2, /* a col_idx outside [0, n) or a row_ptr outside [0, nnz] */
    CCL_ERR_ASYMMETRIC = 3,         /* ccl_validate: an entry without its mirror entry/bit */
    CCL_ERR_OUT_OF_MEMORY = 4,
    CCL_ERR_NONCONVERGED = 5,       /* a chase or atomicMin loop hit its iteration cap */
    CCL_ERR_TIMEOUT = 6,            /* a wait passed its deadline */
    CCL_ERR_REJECTED = 7,           /* the request loop refused a request */
    CCL_ERR_CUDA = 8,               /* a CUDA runtime call failed */
    CCL_ERR_NOT_FOUND = 9           /* unknown ticket */
} ccl_status;

/* Most sites of one instance (2^31 - 4097); larger counts are rejected with
 * CCL_ERR_INVALID_ARGUMENT by every entry point. */
#define CCL_MAX_SITES 2147479551

typedef struct ccl_context ccl_context;

/* Human-readable name of a status code (static storage). */
CCL_API const char *ccl_status_string(int status);

/* Library ABI version, major * 100 + minor. */
CCL_API int ccl_version(void);

/* Creates a context on CUDA device `device`: it owns the workspace (residual
 * pair queue, band records), the error word, the tuning table and the
 * captured CUDA graphs. Not thread-safe: one host thread per context. */
CCL_API ccl_status ccl_context_create(ccl_context **ctx, int device);
CCL_API void ccl_context_destroy(ccl_context *ctx);

/* Tunable options (ccl_set_option / ccl_get_option). */
typedef enum {
    CCL_OPT_PRE_ANALYSIS = 0,  /* 1 (default): run step (ii) before (iii); 0: skip it */
    CCL_OPT_BLOCK_THREADS = 1, /* threads per CTA of the analysis kernel (64..512, multiple of 32) */
    CCL_OPT_USE_GRAPHS = 2,    /* 1 (default): replay captured CUDA graphs for repeated shapes */
    CCL_OPT_PROFILE = 3,       /* 1: record CUDA events between the steps (ccl_get_step_times);
                                  setting it restarts the averaging */
    CCL_OPT_CTAS_PER_SM = 4,   /* persistent CTAs per SM of the analysis kernel; 0 (default) = occupancy maximum */
    CCL_OPT_LINK_MODE = 5,     /* step (iii): 0 (default) a root is linked under the other tree's
                                  root, as in Algorithm 1; 1 under the node the other chain has
                                  reached (same atomicMin loop, shorter walks on trees) */
    CCL_OPT_REFILL = 6,        /* step (iii): 1 (default) each thread serves a fixed stride of the
                                  residual pairs and loads its next one ahead; 0 a warp hands its
                                  pairs out in order to whichever threads are free (balances
                                  uneven chains) */
    CCL_OPT_ANALYSIS_ORDER = 7, /* steps (ii)/(iv): 1 (default) each warp walks a contiguous range of
                                  sites in increasing order (chains meet roots it already stored);
                                  0 the sites are interleaved over the warps (balances inputs
                                  without locality) */
    CCL_OPT_ITER_CAP = 8,      /* 0 (default): the loops of steps (ii)-(iv) stop only at caps
                                  derived from the input size, which a valid input never reaches.
                                  v > 0: a chase of step (ii)/(iv) gives up after v iterations and
                                  a warp of step (iii) abandons its window after v rounds, latching
                                  CCL_ERR_NONCONVERGED (ccl_sync); the labels are then incomplete.
                                  For testing the failure path; setting it drops cached graphs. */
    CCL_OPT_REDUCE_WINDOW = 9, /* step (iii): most residual pairs a warp drains per window
                                  (64..65536); 0 (default): 2048 when the call's labels fit in
                                  three quarters of L2, else 512 */
    CCL_OPT_ANALYSIS_GROUP = 10, /* steps (ii)/(iv) in contiguous order: G > 0 visits the sites in
                                  super-chunks, every warp taking its next G groups of 64 sites
                                  of each, so the labels in use stay in L2; 0 one range per
                                  warp; -1 (default): 0 when the call's labels fit in three
                                  quarters of L2, else 16 */
    CCL_OPT_ANALYSIS_PARK = 11 /* steps (ii)/(iv) in contiguous order: 1 chains still unfinished
                                  after 4 rounds are set aside and finished 32 at a time, one per
                                  lane; 0 every warp runs its longest chain to the end; -1
                                  (default): 1 when the call's labels fit in three quarters of
                                  L2, else 0 */
} ccl_option;

CCL_API ccl_status ccl_set_option(ccl_context *ctx, int option, int64_t value);
CCL_API ccl_status ccl_get_option(ccl_context *ctx, int option, int64_t *value);

/*
 * ccl_label -- label one instance (Section 3, steps (i)-(iv)).
 *   n_sites    number of sites, 0 <= n <= CCL_MAX_SITES (n = 0 returns CCL_OK,
 *              writes nothing)
 *   nnz        number of CSR entries, 0 <= nnz < 2^31
 *   row_ptr    DEVICE int32[n+1]
 *   col_idx    DEVICE int32[nnz]       (may be NULL when nnz = 0)
 *   open_bits  DEVICE uint32[ceil(nnz/32)] (may be NULL when nnz = 0)
 *   labels     DEVICE int32[n], output: canonical labels
 *   stream     cudaStream_t the work is enqueued on; asynchronous
 * The first call with a larger nnz than any before grows the context
 * workspace (one 8-byte residual-pair slot per CSR entry; batched calls add a
 * 4-byte instance id per entry) with cudaMalloc; make that call (or
 * ccl_reserve) before capturing a stream into a graph.
 */
CCL_API ccl_status ccl_label(ccl_context *ctx, int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                     const int32_t *col_idx, const uint32_t *open_bits, int32_t *labels,
                     void *stream);

/*
 * ccl_label_batched -- label K independent instances in one pass of the
 * four steps (one launch per step over all instances).
 *   n_inst     K >= 0
 *   site_off   HOST int64[K+1]: instance k owns sites [site_off[k], site_off[k+1])
 *   ent_off    HOST int64[K+1]: instance k owns entries [ent_off[k], ent_off[k+1])
 *   row_ptr    DEVICE int32: instance k's n_k + 1 row pointers, local entry
 *              numbers 0..nnz_k, start at row_ptr + site_off[k] + k
 *   col_idx    DEVICE int32[ent_off[K]]: instance-local site numbers
 *   open_bits  DEVICE uint32: local entry e of instance k is global bit ent_off[k] + e
 *   labels     DEVICE int32[site_off[K]]: labels[site_off[k] + i] = instance-local label
 * Each instance needs n_k <= CCL_MAX_SITES and nnz_k < 2^31. Asynchronous on `stream`.
 * Repeated calls with the same arguments replay a captured CUDA graph.
 */
CCL_API ccl_status ccl_label_batched(ccl_context *ctx, int32_t n_inst, const int64_t *site_off,
                             const int64_t *ent_off, const int32_t *row_ptr,
                             const int32_t *col_idx, const uint32_t *open_bits, int32_t *labels,
                             void *stream);

/*
 * ccl_label_random -- ccl_label with the bonds drawn on the device instead of
 * read from open_bits: the realisation of bond percolation (Section 4) with
 * open probability p for seed `seed`. The bond {i, j} (i < j) is open iff
 * (SplitMix64 output number i * 2^32 + j of the generator started from state
 * `seed`) >> 11, times 2^-53, is below p (SplitMix64: Steele, Lea & Flood
 * 2014; output number k is mix(seed + (k + 1) * 0x9E3779B97F4A7C15)). Only the
 * CSR structure is read, so many realisations of one graph need only new
 * seeds. 0 <= p <= 1. Asynchronous on `stream`; never replays a graph.
 */
CCL_API ccl_status ccl_label_random(ccl_context *ctx, int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                                    const int32_t *col_idx, uint64_t seed, double p, int32_t *labels,
                                    void *stream);

/*
 * ccl_label_dense -- ccl_label on the dense strided nearest-neighbour list of
 * Section 3: the list has `width` slots per site (the largest neighbour count
 * of any site) and slot k of site i is nn[i + k * n_sites].
 *   nn         device int32[n_sites * width]; a slot holds a site in
 *              [0, n_sites) or -1 (empty: the site has fewer neighbours).
 *              Any other value sets CCL_ERR_INDEX_OUT_OF_RANGE at ccl_sync.
 *   open_bits  device uint32[ceil(n_sites * width / 32)]: slot e = i + k*n_sites
 *              has its open bit at word e >> 5, bit e & 31.
 *   labels     device int32[n_sites], written as by ccl_label.
 * As for CSR input, the bond {i, j} is read from the slots of the larger site
 * only, and a neighbour may appear in several slots (a multigraph).
 * 0 <= width <= CCL_DENSE_MAX_WIDTH; width 0 labels every site by itself.
 * The call uses n_sites * width queue slots of workspace (8 bytes each).
 * Asynchronous on `stream`; replays a CUDA graph for repeated identical calls.
 */
#define CCL_DENSE_MAX_WIDTH 4096
CCL_API ccl_status ccl_label_dense(ccl_context *ctx, int32_t n_sites, int32_t width, const int32_t *nn,
                                   const uint32_t *open_bits, int32_t *labels, void *stream);

/*
 * ccl_label_dense_random -- ccl_label_dense with the bonds drawn on the
 * device exactly as ccl_label_random draws them (bond {i, j}, i < j, keyed by
 * i * 2^32 + j), so a dense list and a CSR list of the same graph give the
 * same realisation for the same (seed, p). 0 <= p <= 1.
 */
CCL_API ccl_status ccl_label_dense_random(ccl_context *ctx, int32_t n_sites, int32_t width,
                                          const int32_t *nn, uint64_t seed, double p, int32_t *labels,
                                          void *stream);

/*
 * ccl_label_host -- ccl_label on HOST arrays: copies the inputs to context
 * buffers, labels, copies the labels back and waits. Synchronous. Pinned
 * (page-locked) host memory gives the full copy bandwidth.
 */
CCL_API ccl_status ccl_label_host(ccl_context *ctx, int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const uint32_t *open_bits, int32_t *labels,
                          void *stream);

/*
 * ccl_label_batched_host -- ccl_label_batched on HOST arrays (the same
 * layout, offsets and meaning): copies the concatenated inputs to context
 * buffers, labels, copies the labels back to `labels` (HOST
 * int32[site_off[K]]) and waits. Synchronous. The instances are labelled in
 * eight groups of about equal site counts, each through all four steps: the
 * upload of later groups and the download of the labels of earlier ones run
 * on two streams of their own while a group is labelled, so the two
 * directions of the host link are busy at once. The result is the same as
 * one ccl_label_batched call; ccl_get_stats afterwards reports the whole
 * batch (pair counts summed over the groups, the settings of the last
 * group). The context keeps device buffers of the inputs' size (plus the
 * labels) for later calls. Pinned host memory gives the full copy bandwidth.
 * Errors: as ccl_label_batched, plus the device status of ccl_sync.
 */
CCL_API ccl_status ccl_label_batched_host(ccl_context *ctx, int32_t n_inst, const int64_t *site_off,
                                          const int64_t *ent_off, const int32_t *row_ptr,
                                          const int32_t *col_idx, const uint32_t *open_bits,
                                          int32_t *labels, void *stream);

/*
 * ccl_label_noalloc -- ccl_label for callers that cannot allocate device
 * memory at run time (the paper has no counterpart; it is a deployment aid).
 * Some programs must not call cudaMalloc once running: a latency-bound loop
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause, and a process whose device memory is handed out by another allocator
 * may have none left for a library. This call needs no context and allocates
 * nothing: its working memory is one fixed device array inside the library
 * (about 17 MB, held by every GPU that loads the library until exit).
 *   n_sites, nnz, row_ptr, col_idx, open_bits, labels, stream: as ccl_label
 *   (device pointers owned by the caller, work on `stream`).
 * Limit: nnz <= 2,097,152 CSR entries; larger inputs return
 * CCL_ERR_INVALID_ARGUMENT without touching the device.
 * Synchronous: enqueues the kernels and the read of the status word on
 * `stream`, waits for `stream` alone, then returns the kernels' status
 * (CCL_OK, CCL_ERR_INDEX_OUT_OF_RANGE, CCL_ERR_INVALID_ARGUMENT,
 * CCL_ERR_NONCONVERGED) or CCL_ERR_CUDA.
 * The first call on a device takes the array's device address and sets up
 * the kernels for that device; make that first call before any stream capture.
 * With CUDA's lazy module loading (the default since CUDA 12.2) the array
 * itself comes into being during that first call, when the library's device
 * code is loaded, so the first call can still fail (CCL_ERR_OUT_OF_MEMORY or
 * CCL_ERR_CUDA) if the device is full: make it at start-up. Later calls
 * allocate nothing.
 * All calls share the one array, so calls that overlap on the GPU (other
 * streams, other host threads) race; serialise them.
 */
CCL_API ccl_status ccl_label_noalloc(int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                                     const int32_t *col_idx, const uint32_t *open_bits,
                                     int32_t *labels, void *stream);

/* Pre-sizes the workspace for calls of up to nnz CSR entries in total (one
 * queue slot each), so later calls up to that size allocate nothing (e.g.
 * before capturing a stream into a graph). n_sites and n_chunks are checked
 * for sign only (the workspace does not depend on them). */
CCL_API ccl_status ccl_reserve(ccl_context *ctx, int64_t n_sites, int64_t nnz, int64_t n_chunks);

/*
 * ccl_sync -- waits until `stream` has drained, polling with a deadline of
 * timeout_ms (< 0: no deadline), then returns and clears the context's latched
 * device error: CCL_OK, CCL_ERR_INDEX_OUT_OF_RANGE, CCL_ERR_INVALID_ARGUMENT
 * or CCL_ERR_NONCONVERGED; CCL_ERR_TIMEOUT if the deadline passed first.
 */
CCL_API ccl_status ccl_sync(ccl_context *ctx, void *stream, int64_t timeout_ms);

/*
 * ccl_validate -- synchronous input check on the device: row_ptr shape and
 * monotonicity, col_idx range, and that every entry (i -> j, bit b) with
 * j != i has a mirror entry (j -> i) in row j carrying the same bit.
 * Returns CCL_OK, CCL_ERR_INVALID_ARGUMENT, CCL_ERR_INDEX_OUT_OF_RANGE or
 * CCL_ERR_ASYMMETRIC.
 */
CCL_API ccl_status ccl_validate(ccl_context *ctx, int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, const uint32_t *open_bits, void *stream);

/*
 * ccl_relabel -- sequential cluster numbers from canonical labels (the
 * renumbering mentioned at the end of Section 3): seq[i] = number of clusters
 * whose smallest site is below label[i], so clusters are numbered 0..C-1 in
 * the order of their smallest sites.
 *   labels      DEVICE int32[n], canonical labels (ccl_label output)
 *   seq         DEVICE int32[n], output; must not alias labels
 *   n_clusters  DEVICE int32, output: C
 *   sizes       DEVICE int32[n] or NULL: sizes[c] = sites of cluster c (c < C)
 * Asynchronous on `stream`; labels that are not canonical give undefined ids.
 */
CCL_API ccl_status ccl_relabel(ccl_context *ctx, int32_t n, const int32_t *labels, int32_t *seq,
                               int32_t *n_clusters, int32_t *sizes, void *stream);

/*
 * ccl_largest_cluster -- the largest cluster of finished canonical labels
 * (the largest-cluster statistic of Section 4's threshold study):
 * result[0] = its number of sites, result[1] = its label (the smallest label
 * when several clusters share the largest size); {0, -1} when n = 0.
 *   labels  DEVICE int32[n], canonical labels (ccl_label output)
 *   result  DEVICE int32[2], output
 * Uses 4n + 16 bytes of context scratch (grown with cudaMalloc when needed).
 * Out-of-range labels are skipped and latched as CCL_ERR_INDEX_OUT_OF_RANGE
 * (ccl_sync). Asynchronous on `stream`.
 */
CCL_API ccl_status ccl_largest_cluster(ccl_context *ctx, int32_t n, const int32_t *labels, int32_t *result,
                                       void *stream);

/*
 * ccl_spanning -- the spanning test of Section 4: *result = the smallest label
 * carried both by a site of `top` and by a site of `bottom` (a cluster that
 * connects the two sets), or -1 if there is none.
 *   labels  DEVICE int32[n]; top DEVICE int32[n_top]; bottom DEVICE int32[n_bottom]
 *   result  DEVICE int32
 * Out-of-range site numbers are skipped and latched as
 * CCL_ERR_INDEX_OUT_OF_RANGE (ccl_sync). Asynchronous on `stream`.
 */
CCL_API ccl_status ccl_spanning(ccl_context *ctx, int32_t n, const int32_t *labels, const int32_t *top,
                                int32_t n_top, const int32_t *bottom, int32_t n_bottom, int32_t *result,
                                void *stream);

/* Counters of the last completed labelling call (synchronous read). */
typedef struct {
    int64_t residual_pairs;   /* pairs handled by step (iii), summed over instances */
    int64_t n_sites;          /* sites labelled */
    int64_t nnz;              /* CSR entries read */
    int32_t n_inst;           /* instances */
    int32_t used_graph;       /* 1 if the call replayed a captured CUDA graph */
    /* step (iii) work counters, filled only by a library built with
       -DCCL_DEVICE_STATS (else 0): label loads of the root chases, atomicMin
       operations of the merge loops, warp iterations of the reduction */
    int64_t chase_loads, merge_atomics, reduce_iterations;
    /* the settings the last call ran with (tuned, set, or chosen by size):
       step (ii) on, step (iii) link mode and hand-out, step (ii)/(iv) order,
       step (iii) window, step (ii)/(iv) super-chunk run length (0: one range
       per warp), step (ii)/(iv) parking -- see ccl_option */
    int32_t pre_analysis, link_mode, refill, analysis_order, reduce_window, analysis_group, analysis_park;
} ccl_run_stats;

/* Statistics of the context's last labelling call; waits for that call to
 * finish (not for other work on the device). */
CCL_API ccl_status ccl_get_stats(ccl_context *ctx, ccl_run_stats *stats);

/* Per-step device times (ms), averaged over the calls made since
 * CCL_OPT_PROFILE was last set to 1 (up to the last 4096 such calls): ms[0]
 * init, ms[1] analysis (ii), ms[2] reduction (iii), ms[3] analysis (iv); ms[4]
 * (if n > 4) the number of calls averaged. Profiled calls record CUDA events
 * between the steps on the caller's stream and do not replay graphs.
 * Synchronous. */
CCL_API ccl_status ccl_get_step_times(ccl_context *ctx, float *ms, int32_t n);

/*
 * ccl_autotune -- synchronous: times the labelling of the given instance under
 * candidate settings (analysis threads per CTA, step (ii) on/off, link mode,
 * refill mode, analysis order)
 * and keeps the fastest for instances of this size class (log2 of the site
 * count, mean degree rounded); the choice also becomes the context's
 * options (ccl_get_option reports it). Every candidate writes the same labels,
 * so `labels` holds the correct result afterwards. best_ms (optional)
 * receives the best time.
 * If the environment variable CCL_TUNE_CACHE names a file, ccl_autotune
 * writes the context's whole table there (one line per size class: class,
 * threads, CTAs per SM, step (ii), link mode, refill mode, analysis order)
 * and ccl_context_create reads it back; lines that do not parse are ignored.
 */
CCL_API ccl_status ccl_autotune(ccl_context *ctx, int32_t n_sites, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, const uint32_t *open_bits, int32_t *labels,
                        void *stream, float *best_ms);

/*
 * ccl_autotune_batched -- ccl_autotune for ccl_label_batched: times one
 * batched call of these K instances under each candidate setting (step (ii)
 * on/off, link mode, refill mode, analysis order) and keeps the fastest for
 * batches of this mean instance size and degree (a class of its own, apart
 * from single instances). Arguments as ccl_label_batched; `labels` holds the
 * correct result afterwards; best_ms (optional) receives the best time.
 * Synchronous; each candidate runs three times, so budget ~50 calls.
 */
CCL_API ccl_status ccl_autotune_batched(ccl_context *ctx, int32_t n_inst, const int64_t *site_off,
                                        const int64_t *ent_off, const int32_t *row_ptr,
                                        const int32_t *col_idx, const uint32_t *open_bits,
                                        int32_t *labels, void *stream, float *best_ms);

/* ---------------------------------------------------------------------------
 * Request loop (continuous batching). A server thread admits submitted
 * requests while the device memory they need is free (free HBM minus a
 * reserve, and at most hbm_budget bytes held), uploads each into device
 * memory of its own, gathers every uploaded request into one batched launch
 * per tick on one of n_streams compute streams, so later arrivals are labelled
 * while earlier batches are still on the GPU, and copies labels back.
 *
 * Memory counted against the budget: each admitted request's device buffer
 * (inputs and labels, 4(n+1) + 4 nnz + 4 ceil(nnz/32) + 4n bytes, each part
 * rounded up to 256) and, until its batch is launched, 12 bytes per CSR entry
 * for its share of the batched workspace; plus the workspace every compute
 * stream's context keeps after its largest batch. When only that kept
 * workspace stands in the way of the next request, idle contexts free it.
 * A request whose buffer cannot be allocated (other programs hold the memory)
 * while the server holds nothing for other requests ends after 2 s with
 * CCL_ERR_OUT_OF_MEMORY. A batch whose launch fails ends each of its
 * requests with that error.
 * Test hook: the environment variable CCL_SERVER_FAIL_BATCH=k, read by
 * ccl_server_create, makes the k-th batch launch of that server fail with
 * CCL_ERR_OUT_OF_MEMORY without running (as a failed workspace allocation).
 * ------------------------------------------------------------------------- */

typedef struct ccl_server ccl_server;

typedef struct {
    int32_t device;
    int32_t n_streams;       /* concurrent compute streams (default 2) */
    int64_t hbm_reserve;     /* bytes of free HBM never used (default 2 GiB) */
    int64_t hbm_budget;      /* most bytes held by admitted requests (0 = no limit) */
    int32_t max_batch;       /* most requests per launch (default 1024) */
    int32_t max_pending;     /* most requests waiting for admission (default 1<<20) */
    int64_t host_staging_bytes; /* pinned host arena for request copies (0: default 1 GiB,
                                   < 0: none, requests then stay in pageable memory) */
} ccl_server_config;

typedef struct {
    int32_t n_sites;
    int32_t pad_;
    int64_t nnz;
    const int32_t *row_ptr;     /* HOST int32[n+1] */
    const int32_t *col_idx;     /* HOST int32[nnz] */
    const uint32_t *open_bits;  /* HOST uint32[ceil(nnz/32)] */
} ccl_request;

typedef struct {
    int64_t submitted, completed, rejected, batches;
    int64_t sites_completed;
    double p50_ms, p99_ms, max_ms;   /* submit -> labels on host */
    double busy_seconds;             /* wall time from first submit to last completion */
    double sites_per_second;
    int64_t waiting;                 /* threads inside ccl_server_wait now */
    int64_t arena_misses;            /* requests whose host copy (ccl_server_submit) or labels
                                        (ccl_server_submit_nocopy) did not fit the pinned staging
                                        arena and went through pageable memory */
    /* latency by phase, p50 and p99 over completed requests:
       [0] submit -> admitted (upload started), [1] -> upload seen complete,
       [2] -> launched in a batch, [3] -> labels on host */
    double phase_p50_ms[4], phase_p99_ms[4];
} ccl_server_stats;

/* Starts the server thread. cfg may be NULL for defaults. */
CCL_API ccl_status ccl_server_create(ccl_server **srv, const ccl_server_config *cfg);

/* Copies the request (so the caller may free it on return) and queues it.
 * CCL_ERR_REJECTED if it can never fit the budget or the queue is full. */
CCL_API ccl_status ccl_server_submit(ccl_server *srv, const ccl_request *req, uint64_t *ticket);

/* As ccl_server_submit, without copying the request: the caller keeps
 * req->row_ptr, col_idx and open_bits allocated and unchanged until
 * ccl_server_wait has returned for the ticket (CCL_OK or an error other than
 * CCL_ERR_TIMEOUT). The server uploads them from where they are (pinned or
 * pageable host memory), which saves a host copy of the whole request. */
CCL_API ccl_status ccl_server_submit_nocopy(ccl_server *srv, const ccl_request *req, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: forever) for the ticket, copies its labels to
 * labels_host (int32[n]) and forgets the ticket. */
CCL_API ccl_status ccl_server_wait(ccl_server *srv, uint64_t ticket, int32_t *labels_host,
                           int64_t timeout_ms);

CCL_API ccl_status ccl_server_stats_get(ccl_server *srv, ccl_server_stats *stats);

/* Stops the server's threads. Batches already on the device finish; requests
 * not yet launched are dropped: a ccl_server_wait blocked on one in another
 * thread returns CCL_ERR_REJECTED without writing labels_host, and destroy
 * returns only after every such waiter has left. No call may use srv once
 * destroy has started, except those waits already in progress. */
CCL_API void ccl_server_destroy(ccl_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* CCL_H_ */
