// Host side of the C ABI declared in include/ccl.h: contexts, workspace,
// launch shapes, CUDA-graph replay, validation, tuning and statistics.
#include <ccl.h>

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "ccl_device.cuh"
#include "ccl_dense.cuh"
#include "ccl_stats.cuh"

using namespace ccl;

namespace {

struct TuneChoice {
    int threads = 256;
    int ctas_per_sm = 0;
    int pre_analysis = 1;
    int link_mode = 0;
    int refill = 1;         // step (iii): 1 static per-lane pairs, 0 in-order hand-out
    int ana_seq = 1;        // steps (ii)/(iv): 1 contiguous ranges per warp, 0 interleaved
    int red_window = 0;     // step (iii): most pairs per warp window; 0 by size (see resolve_tail)
    int ana_group = -1;     // steps (ii)/(iv), contiguous order: super-chunk run length; -1 by size
    int ana_park = -1;      // steps (ii)/(iv), contiguous order: 1 park long chains, 0 not; -1 by size
};

struct GraphEntry {
    // key
    int32_t K = 0;
    int64_t n_chunks = 0;
    const void *row_ptr = nullptr, *col_idx = nullptr, *bits = nullptr;
    int32_t dense = 0;               // dense neighbour-list call
    const void *nn = nullptr;
    int64_t nn_width = 0;
    void *labels = nullptr;
    uint64_t shape_hash = 0;
    Inst one{};                      // the instance (single path), compared exactly
    std::vector<int64_t> offsets;    // site_off and ent_off (batched), compared exactly
    TuneChoice tc;
    // value
    cudaGraphExec_t exec = nullptr;
    Inst *d_insts = nullptr;     // owned table (batched)
    uint64_t last_use = 0;
};

}  // namespace

struct ccl_context {
    int device = 0;
    int num_sms = 0;
    int64_t l2_bytes = 0;
    // workspace
    int2 *d_q = nullptr;
    int64_t q_cap = 0;
    int32_t *d_qk = nullptr;     // instance of each pair (batched calls)
    int64_t qk_cap = 0;
    BandRec *d_band = nullptr;   // [kMaxBands]
    unsigned *d_err = nullptr;
    unsigned long long *d_counters = nullptr;
    // batched descriptor table (non-graph path)
    Inst *d_insts = nullptr;
    int64_t insts_cap = 0;
    Inst *h_insts = nullptr;     // pinned staging
    int64_t h_insts_cap = 0;
    cudaEvent_t staging_free = nullptr;
    // recorded after each labelling call (outside stream capture): statistics
    // reads wait for it instead of the whole device
    cudaEvent_t stats_ev = nullptr;
    // host-buffer path: device copies of the inputs, and the copy stream and
    // events that overlap the upload of later parts with step (i) on earlier ones
    void *d_host_in = nullptr;
    int64_t host_in_cap = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t part_ev[5] = {};
    // batched host-buffer path: the label download stream and, per instance
    // group, the events of its upload and of its labelling
    cudaStream_t d2h_stream = nullptr;
    cudaEvent_t bh_up[8] = {}, bh_done[9] = {};
    // relabel / spanning scratch
    void *d_aux = nullptr;
    int64_t aux_cap = 0;
    // options
    TuneChoice opt;
    int use_graphs = 1;
    int profile = 0;
    int32_t iter_cap = 0;       // CCL_OPT_ITER_CAP
    double ws_growth = 1.0;     // a growing workspace takes max(need, ws_growth * current) slots
    std::map<int64_t, TuneChoice> tune_table;
    // graphs
    std::vector<GraphEntry> graphs;
    uint64_t use_clock = 0;
    cudaStream_t cap_stream = nullptr;
    // profiling: one set of 5 events per profiled call, kept in a ring so that
    // many calls can be timed without a host synchronisation in between
    std::vector<std::array<cudaEvent_t, 5>> prof;
    int64_t prof_count = 0;     // calls recorded since the last reset
    cudaEvent_t *ev = nullptr;  // the set of the call being enqueued
    int have_times = 0;
    // stats of the last call
    ccl_run_stats last{};
    // occupancy cache: (kernel id, threads) -> blocks per SM
    std::map<std::pair<int, int>, int> occ;
};

namespace {

constexpr size_t kMaxGraphs = 16;
constexpr uint64_t kNoGen = ~0ull;     // Params::gen_thr of calls that read open_bits
constexpr int64_t kProfRing = 4096;

ccl_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CCL_OK;
    if (e == cudaErrorMemoryAllocation) return CCL_ERR_OUT_OF_MEMORY;
    return CCL_ERR_CUDA;
}

#define CCL_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            (void)cudaGetLastError();                       \
            return cuda_status(e_);                         \
        }                                                   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};


int blocks_per_sm(ccl_context *ctx, int kernel_id, int threads) {
    auto key = std::make_pair(kernel_id, threads);
    auto it = ctx->occ.find(key);
    if (it != ctx->occ.end()) return it->second;
    int nb = 1;
    cudaError_t e = cudaSuccess;
    switch (kernel_id) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init<false>, kInitThreads, kInitSmem); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init<true>, kInitThreads, kInitSmem); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_analysis<false, true>, threads, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_analysis<true, true, kAnaChunksBatched>, threads, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_reduce<false, true>, threads, 0); break;
        case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_reduce<true, true>, threads, 0); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init<false, true>, kInitThreads, kInitSmem); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init_dense<false>, kDenseThreads, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init_dense<true>, kDenseThreads, 0); break;
        case 9: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init_dense_tma<false>, kInitThreads, kDenseSmem); break;
        case 10: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_init_dense_tma<true>, kInitThreads, kDenseSmem); break;
        case 11: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_analysis_park<false>, 32 * kParkWarps, 0); break;
        case 12: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_analysis_park<true>, 32 * kParkWarps, 0); break;
        default: break;
    }
    if (e != cudaSuccess || nb < 1) { (void)cudaGetLastError(); nb = 1; }
    ctx->occ[key] = nb;
    return nb;
}

int64_t grid_for(ccl_context *ctx, int kernel_id, const TuneChoice &tc, int64_t warps_needed) {
    int per_sm = blocks_per_sm(ctx, kernel_id, tc.threads);
    if (tc.ctas_per_sm > 0) per_sm = std::min(per_sm, tc.ctas_per_sm);
    int64_t g = (int64_t)ctx->num_sms * per_sm;
    const int64_t wpb = tc.threads / 32;
    const int64_t need = (warps_needed + wpb - 1) / wpb;
    return std::max<int64_t>(1, std::min(g, need));
}

// step (i): fixed CTA shape; CTA b takes the band of tiles [b*per, (b+1)*per),
// so launch just enough CTAs for every band to be non-empty
int64_t grid_init(ccl_context *ctx, int kernel_id, int threads, int64_t n_tiles) {
    const int per_sm = blocks_per_sm(ctx, kernel_id, threads);
    int64_t g = std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * per_sm, n_tiles));
    g = std::min<int64_t>(g, kMaxBands);
    const int64_t per = (n_tiles + g - 1) / g;
    return std::max<int64_t>(1, (n_tiles + per - 1) / per);
}

void drop_graphs(ccl_context *ctx) {
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.d_insts) cudaFree(g.d_insts);
    }
    ctx->graphs.clear();
}

// Residual-pair queue: one slot per CSR entry of the call (a pair never needs
// more), plus the per-pair instance for batched calls.
ccl_status ensure_workspace(ccl_context *ctx, int64_t q_slots, bool batched) {
    if (q_slots > ctx->q_cap || (batched && q_slots > ctx->qk_cap)) drop_graphs(ctx);  // graphs hold the pointers
    // a grown allocation of `want` elements (at least `need`), or of exactly
    // `need` when the larger one does not fit
    auto grow = [](void **p, int64_t &cap, int64_t need, int64_t want, size_t elem) {
        if (*p) cudaFree(*p);
        *p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(p, (size_t)want * elem);
        if (e == cudaErrorMemoryAllocation && want > need) {
            (void)cudaGetLastError();
            want = need;
            e = cudaMalloc(p, (size_t)want * elem);
        }
        if (e == cudaSuccess) cap = want;
        return e;
    };
    if (q_slots > ctx->q_cap) {
        const int64_t need = std::max<int64_t>(q_slots, 1024);
        const int64_t want = std::max<int64_t>(need, (int64_t)(ctx->ws_growth * (double)ctx->q_cap));
        CCL_CUDA(grow((void **)&ctx->d_q, ctx->q_cap, need, want, sizeof(int2)));
    }
    if (batched && q_slots > ctx->qk_cap) {
        const int64_t need = std::max<int64_t>(q_slots, 1024);
        const int64_t want = std::max<int64_t>(need, (int64_t)(ctx->ws_growth * (double)ctx->qk_cap));
        CCL_CUDA(grow((void **)&ctx->d_qk, ctx->qk_cap, need, want, sizeof(int32_t)));
    }
    return CCL_OK;
}

int64_t size_class(int64_t n, int64_t nnz) {
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= std::max<int64_t>(n, 1)) ++lg;
    const int64_t deg = n > 0 ? (nnz + n / 2) / n : 0;
    return (int64_t)lg * 1024 + std::min<int64_t>(deg, 1023);
}

// Batched calls are keyed by their mean instance size and degree, in a range
// of classes of their own (a batch of K instances of n sites and a single
// instance of n sites behave differently).
int64_t batch_class(int64_t n_tot, int64_t nnz_tot, int64_t K) {
    const int64_t c = size_class(n_tot / std::max<int64_t>(K, 1), nnz_tot / std::max<int64_t>(K, 1));
    return K > 1 ? (int64_t(1) << 30) + c : c;
}

// Times each candidate (first run untimed, then `reps` - 1 timed runs, the
// fastest counted) and returns the best in best/best_t. The profiling events
// are off meanwhile.
template <typename Runner>
ccl_status tune_over(ccl_context *ctx, cudaStream_t s, const std::vector<TuneChoice> &cands, int reps,
                     TuneChoice &best, float &best_t, Runner runner) {
    cudaEvent_t a = nullptr, b = nullptr;
    CCL_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return CCL_ERR_CUDA; }
    const int saved_profile = ctx->profile;
    ctx->profile = 0;
    ccl_status st = CCL_OK;
    for (const TuneChoice &tc : cands) {
        float tmin = 1e30f;
        for (int rep = 0; rep < reps && st == CCL_OK; ++rep) {
            cudaError_t e = cudaEventRecord(a, s);
            if (e == cudaSuccess) st = runner(tc);
            if (e == cudaSuccess && st == CCL_OK) e = cudaEventRecord(b, s);
            if (e == cudaSuccess && st == CCL_OK) e = cudaEventSynchronize(b);
            if (e != cudaSuccess) st = cuda_status(e);
            float t = 0;
            if (st == CCL_OK) cudaEventElapsedTime(&t, a, b);
            if (rep > 0) tmin = std::min(tmin, t);
        }
        if (st != CCL_OK) break;
        if (tmin < best_t) { best_t = tmin; best = tc; }
    }
    ctx->profile = saved_profile;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

// Second tuning stage on the best first-stage choice: the step (iii) window,
// then (contiguous order only) the step (ii)/(iv) super-chunk run length.
template <typename Runner>
ccl_status tune_tail(ccl_context *ctx, cudaStream_t s, int reps, TuneChoice &best, float &best_t, Runner runner) {
    std::vector<TuneChoice> c;
    for (int w : {256, 512, 1024, 2048}) {
        TuneChoice t = best;
        t.red_window = w;
        c.push_back(t);
    }
    ccl_status st = tune_over(ctx, s, c, reps, best, best_t, runner);
    if (st != CCL_OK || !best.ana_seq) return st;
    c.clear();
    for (int g : {0, 8, 16, 32}) {
        TuneChoice t = best;
        t.ana_group = g;
        c.push_back(t);
    }
    st = tune_over(ctx, s, c, reps, best, best_t, runner);
    if (st != CCL_OK) return st;
    c.clear();
    for (int k : {0, 1}) {
        TuneChoice t = best;
        t.ana_park = k;
        c.push_back(t);
    }
    return tune_over(ctx, s, c, reps, best, best_t, runner);
}

TuneChoice choice_for_class(ccl_context *ctx, int64_t cls) {
    auto it = ctx->tune_table.find(cls);
    if (it != ctx->tune_table.end()) return it->second;
    return ctx->opt;
}

TuneChoice choice_for(ccl_context *ctx, int64_t n, int64_t nnz) {
    auto it = ctx->tune_table.find(size_class(n, nnz));
    if (it != ctx->tune_table.end()) return it->second;
    return ctx->opt;
}

// Grid of step (i) over P.n_tiles tiles: CTAs (bands) of the kernel variant P
// selects, at most max_bands.
int64_t init_grid(ccl_context *ctx, const Params &P, bool batched, int64_t max_bands) {
    const bool gen = P.gen_thr != kNoGen;
    int64_t g;
    if (P.dense && P.nn_width <= kRowRegs) g = grid_init(ctx, gen ? 10 : 9, kInitThreads, P.n_tiles);
    else if (P.dense) g = grid_init(ctx, gen ? 8 : 7, kDenseThreads, P.n_tiles);
    else g = grid_init(ctx, batched ? 1 : (gen ? 6 : 0), kInitThreads, P.n_tiles);
    if (g > max_bands) {     // fewer, longer bands
        const int64_t per = (P.n_tiles + max_bands - 1) / max_bands;
        g = (P.n_tiles + per - 1) / per;
    }
    return g;
}

ccl_status launch_init(const Params &P, bool batched, int64_t g, cudaStream_t s) {
    const bool gen = P.gen_thr != kNoGen;
    if (P.dense && P.nn_width <= kRowRegs) {
        if (gen) k_init_dense_tma<true><<<(unsigned)g, kInitThreads, kDenseSmem, s>>>(P);
        else k_init_dense_tma<false><<<(unsigned)g, kInitThreads, kDenseSmem, s>>>(P);
    } else if (P.dense) {
        if (gen) k_init_dense<true><<<(unsigned)g, kDenseThreads, 0, s>>>(P);
        else k_init_dense<false><<<(unsigned)g, kDenseThreads, 0, s>>>(P);
    } else if (batched) {
        k_init<true><<<(unsigned)g, kInitThreads, kInitSmem, s>>>(P);
    } else if (gen) {
        k_init<false, true><<<(unsigned)g, kInitThreads, kInitSmem, s>>>(P);
    } else {
        k_init<false><<<(unsigned)g, kInitThreads, kInitSmem, s>>>(P);
    }
    CCL_CUDA(cudaGetLastError());
    return CCL_OK;
}

// The step (iii) window and the step (ii)/(iv) visiting order of a call:
// explicit settings win; otherwise, when the call's labels fit in three
// quarters of L2, long windows and one contiguous range per warp (every
// gather hits L2 anyway), else windows of 512 pairs and super-chunks of 16
// chunk groups per warp, so the labels the warps touch at once stay in L2.
bool labels_fit_l2(const ccl_context *ctx, const Params &P) {
    return 4 * kChunk * P.n_chunks <= ctx->l2_bytes * 3 / 4;
}

void resolve_tail(const ccl_context *ctx, const TuneChoice &tc, Params &P) {
    const bool fits = labels_fit_l2(ctx, P);
    P.red_window = tc.red_window > 0 ? tc.red_window : (fits ? kRedWindowMax : 512);
    P.ana_group = tc.ana_group >= 0 ? tc.ana_group : (fits ? 0 : 16);
}

// Parking of long chains in steps (ii)/(iv) (contiguous order only): explicit
// setting, else on when the call's labels fit in three quarters of L2.
bool resolve_park(const ccl_context *ctx, const TuneChoice &tc, const Params &P) {
    if (!tc.ana_seq || P.iter_cap > 0) return false;    // the iteration-cap test option uses k_analysis
    return tc.ana_park >= 0 ? tc.ana_park != 0 : labels_fit_l2(ctx, P);
}

// Records in the context's statistics the settings a call runs with.
void note_settings(ccl_context *ctx, const TuneChoice &tc, const Params &P) {
    ctx->last.pre_analysis = tc.pre_analysis;
    ctx->last.link_mode = tc.link_mode;
    ctx->last.refill = tc.refill;
    ctx->last.analysis_order = tc.ana_seq;
    ctx->last.reduce_window = P.red_window;
    ctx->last.analysis_group = tc.ana_seq ? P.ana_group : 0;
    ctx->last.analysis_park = resolve_park(ctx, tc, P) ? 1 : 0;
}

// Steps (ii)-(iv) after step (i) has filled P.n_bands band records.
ccl_status enqueue_tail(ccl_context *ctx, const Params &P0, bool batched, const TuneChoice &tc, cudaStream_t s,
                        bool profile) {
    Params P = P0;
    resolve_tail(ctx, tc, P);
    note_settings(ctx, tc, P);
    const int T = tc.threads;
    const int64_t warps_chunks = (P.n_chunks + kAnaChunks - 1) / kAnaChunks;
    const int64_t warps_chunks_b = (P.n_chunks + kAnaChunksBatched - 1) / kAnaChunksBatched;
    const int64_t g_red = (int64_t)ctx->num_sms * blocks_per_sm(ctx, batched ? 5 : 4, 256);
    if (profile) CCL_CUDA(cudaEventRecord(ctx->ev[1], s));
    const bool park = resolve_park(ctx, tc, P);
    auto analysis = [&]() {
        if (park) {
            // a full SM of warps (the kernel's registers and shared memory allow
            // it; the occupancy query can assume a smaller shared-memory carveout)
            const int64_t per_sm = std::max<int64_t>(blocks_per_sm(ctx, batched ? 12 : 11, 32 * kParkWarps),
                                                     2048 / (32 * kParkWarps));
            const int64_t need = (warps_chunks + kParkWarps - 1) / kParkWarps;
            const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * per_sm, need));
            if (batched) k_analysis_park<true><<<gp, 32 * kParkWarps, 0, s>>>(P);
            else k_analysis_park<false><<<gp, 32 * kParkWarps, 0, s>>>(P);
            return;
        }
        const unsigned g = (unsigned)grid_for(ctx, batched ? 3 : 2, tc, batched ? warps_chunks_b : warps_chunks);
        if (batched) {
            if (tc.ana_seq) k_analysis<true, true, kAnaChunksBatched><<<g, T, 0, s>>>(P);
            else k_analysis<true, false, kAnaChunksBatched><<<g, T, 0, s>>>(P);
        } else {
            if (tc.ana_seq) k_analysis<false, true><<<g, T, 0, s>>>(P);
            else k_analysis<false, false><<<g, T, 0, s>>>(P);
        }
    };
    if (tc.pre_analysis) {
        analysis();
        CCL_CUDA(cudaGetLastError());
    }
    if (profile) CCL_CUDA(cudaEventRecord(ctx->ev[2], s));
    if (batched) {
        if (tc.refill) k_reduce<true, true><<<(unsigned)g_red, 256, 0, s>>>(P);
        else k_reduce<true, false><<<(unsigned)g_red, 256, 0, s>>>(P);
    } else {
        if (tc.refill) k_reduce<false, true><<<(unsigned)g_red, 256, 0, s>>>(P);
        else k_reduce<false, false><<<(unsigned)g_red, 256, 0, s>>>(P);
    }
    CCL_CUDA(cudaGetLastError());
    if (profile) CCL_CUDA(cudaEventRecord(ctx->ev[3], s));
    analysis();
    CCL_CUDA(cudaGetLastError());
    if (profile) CCL_CUDA(cudaEventRecord(ctx->ev[4], s));
    return CCL_OK;
}

// Enqueues the four steps. All kernels read their sizes from Params, so the
// sequence contains no host synchronisation and can be captured.
ccl_status enqueue_steps(ccl_context *ctx, const Params &P0, bool batched, const TuneChoice &tc,
                         cudaStream_t s, bool profile) {
    Params P = P0;
    const int64_t g_init = init_grid(ctx, P, batched, kMaxBands);
    P.n_bands = (int32_t)g_init;
    CCL_CUDA(cudaMemsetAsync(P.counters, 0, 4 * sizeof(unsigned long long), s));
    CCL_CUDA(cudaMemsetAsync(P.band, 0, (size_t)g_init * sizeof(BandRec), s));
    if (profile) CCL_CUDA(cudaEventRecord(ctx->ev[0], s));
    ccl_status st = launch_init(P, batched, g_init, s);
    if (st != CCL_OK) return st;
    return enqueue_tail(ctx, P, batched, tc, s, profile);
}

uint64_t fnv1a(const void *data, size_t bytes, uint64_t h = 1469598103934665603ull) {
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < bytes; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

bool same_choice(const TuneChoice &a, const TuneChoice &b) {
    return a.threads == b.threads && a.ctas_per_sm == b.ctas_per_sm &&
           a.pre_analysis == b.pre_analysis && a.link_mode == b.link_mode && a.refill == b.refill &&
           a.ana_seq == b.ana_seq && a.red_window == b.red_window && a.ana_group == b.ana_group &&
           a.ana_park == b.ana_park;
}

GraphEntry *find_graph(ccl_context *ctx, const GraphEntry &key) {
    for (auto &g : ctx->graphs) {
        if (g.K == key.K && g.n_chunks == key.n_chunks && g.row_ptr == key.row_ptr &&
            g.col_idx == key.col_idx && g.bits == key.bits && g.labels == key.labels &&
            g.dense == key.dense && g.nn == key.nn && g.nn_width == key.nn_width &&
            g.shape_hash == key.shape_hash && same_choice(g.tc, key.tc) &&
            memcmp(&g.one, &key.one, sizeof(Inst)) == 0 && g.offsets == key.offsets)
            return &g;
    }
    return nullptr;
}

void evict_graph_if_full(ccl_context *ctx) {
    if (ctx->graphs.size() < kMaxGraphs) return;
    size_t lru = 0;
    for (size_t i = 1; i < ctx->graphs.size(); ++i)
        if (ctx->graphs[i].last_use < ctx->graphs[lru].last_use) lru = i;
    if (ctx->graphs[lru].exec) cudaGraphExecDestroy(ctx->graphs[lru].exec);
    if (ctx->graphs[lru].d_insts) cudaFree(ctx->graphs[lru].d_insts);
    ctx->graphs.erase(ctx->graphs.begin() + (long)lru);
}

// Captures the step sequence for Params P on the context's capture stream.
ccl_status capture_graph(ccl_context *ctx, const Params &P, bool batched, const TuneChoice &tc,
                         cudaGraphExec_t *exec) {
    cudaGraph_t graph = nullptr;
    CCL_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    ccl_status st = enqueue_steps(ctx, P, batched, tc, ctx->cap_stream, false);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (st != CCL_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    CCL_CUDA(e);
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    CCL_CUDA(e);
    return CCL_OK;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) { (void)cudaGetLastError(); return false; }
    return cs != cudaStreamCaptureStatusNone;
}

// Uploads an instance table to ctx->d_insts on stream s through the pinned
// staging buffer, after the previous upload has left that buffer.
ccl_status upload_table(ccl_context *ctx, const std::vector<Inst> &table, cudaStream_t s) {
    const int64_t K = (int64_t)table.size();
    // tables grow at least twofold (each growth synchronises the device)
    if (K > ctx->h_insts_cap) {
        const int64_t want = std::max<int64_t>({K, 64, 2 * ctx->h_insts_cap});
        if (ctx->h_insts) { cudaEventSynchronize(ctx->staging_free); cudaFreeHost(ctx->h_insts); }
        ctx->h_insts = nullptr;
        ctx->h_insts_cap = 0;
        CCL_CUDA(cudaMallocHost(&ctx->h_insts, (size_t)want * sizeof(Inst)));
        ctx->h_insts_cap = want;
    }
    if (K > ctx->insts_cap) {
        const int64_t want = std::max<int64_t>({K, 64, 2 * ctx->insts_cap});
        if (ctx->d_insts) cudaFree(ctx->d_insts);
        ctx->d_insts = nullptr;
        ctx->insts_cap = 0;
        CCL_CUDA(cudaMalloc(&ctx->d_insts, (size_t)want * sizeof(Inst)));
        ctx->insts_cap = want;
    }
    CCL_CUDA(cudaEventSynchronize(ctx->staging_free));
    memcpy(ctx->h_insts, table.data(), (size_t)K * sizeof(Inst));
    CCL_CUDA(cudaMemcpyAsync(ctx->d_insts, ctx->h_insts, (size_t)K * sizeof(Inst), cudaMemcpyHostToDevice, s));
    CCL_CUDA(cudaEventRecord(ctx->staging_free, s));
    return CCL_OK;
}

// Runs P on stream s: through a cached graph when allowed, else directly.
ccl_status run(ccl_context *ctx, Params P, bool batched, const TuneChoice &tc, cudaStream_t s,
               const std::vector<Inst> *table, uint64_t shape_hash, bool allow_graph = true,
               const std::vector<int64_t> *offsets = nullptr) {
    for (int kid = 0; kid < 13; ++kid)
        (void)blocks_per_sm(ctx, kid, kid >= 11 ? 32 * kParkWarps : kid >= 9 ? kInitThreads : kid >= 7 ? kDenseThreads
                                               : (kid < 2 || kid == 6) ? kInitThreads : (kid >= 4 ? 256 : tc.threads));
    ctx->last.used_graph = 0;
    const bool capturing = stream_capturing(s);
    if (ctx->profile || !ctx->use_graphs || capturing || !allow_graph) {
        if (batched) {
            ccl_status st = upload_table(ctx, *table, s);
            if (st != CCL_OK) return st;
            P.insts = ctx->d_insts;
        }
        if (ctx->profile) {
            const size_t slot = (size_t)(ctx->prof_count % kProfRing);
            if (slot >= ctx->prof.size()) {
                std::array<cudaEvent_t, 5> set{};
                for (auto &e : set) CCL_CUDA(cudaEventCreate(&e));
                ctx->prof.push_back(set);
            }
            ctx->ev = ctx->prof[slot].data();
        }
        ccl_status st = enqueue_steps(ctx, P, batched, tc, s, ctx->profile != 0);
        if (st == CCL_OK && ctx->profile) { ctx->have_times = 1; ctx->prof_count++; }
        if (st == CCL_OK && !capturing) CCL_CUDA(cudaEventRecord(ctx->stats_ev, s));
        return st;
    }
    GraphEntry key;
    key.K = P.K;
    key.n_chunks = P.n_chunks;
    key.row_ptr = batched ? (const void *)(*table)[0].row_ptr : P.one.row_ptr;
    key.col_idx = batched ? (const void *)(*table)[0].col_idx : P.one.col_idx;
    key.bits = batched ? (const void *)(*table)[0].bits : P.one.bits;
    key.labels = batched ? (void *)(*table)[0].labels : P.one.labels;
    key.dense = P.dense;
    key.nn = P.nn;
    key.nn_width = P.nn_width;
    key.shape_hash = shape_hash;
    key.tc = tc;
    if (!batched) key.one = P.one;
    if (offsets) key.offsets = *offsets;
    GraphEntry *g = find_graph(ctx, key);
    if (!g) {
        evict_graph_if_full(ctx);
        GraphEntry ne = key;
        if (batched) {
            const size_t bytes = table->size() * sizeof(Inst);
            CCL_CUDA(cudaMalloc(&ne.d_insts, bytes));
            cudaError_t e = cudaMemcpy(ne.d_insts, table->data(), bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cudaFree(ne.d_insts); return cuda_status(e); }
            P.insts = ne.d_insts;
        }
        ccl_status st = capture_graph(ctx, P, batched, tc, &ne.exec);
        if (st != CCL_OK) { if (ne.d_insts) cudaFree(ne.d_insts); return st; }
        ctx->graphs.push_back(ne);
        g = &ctx->graphs.back();
    }
    g->last_use = ++ctx->use_clock;
    {
        Params R = P;
        resolve_tail(ctx, tc, R);
        note_settings(ctx, tc, R);
    }
    CCL_CUDA(cudaGraphLaunch(g->exec, s));
    CCL_CUDA(cudaEventRecord(ctx->stats_ev, s));
    ctx->last.used_graph = 1;
    return CCL_OK;
}

// readable memory of the three input arrays of an instance (the whole
// concatenated arrays for a batch)
void set_bounds(Inst &I, const int32_t *rp, int64_t rp_len, const int32_t *ci, int64_t ci_len,
                const uint32_t *bits, int64_t bits_len) {
    I.rp_lo = rp;
    I.rp_hi = rp + rp_len;
    I.ci_lo = ci;
    I.ci_hi = ci ? ci + ci_len : ci;
    I.bits_lo = bits;
    I.bits_hi = bits ? bits + bits_len : bits;
}

Params base_params(ccl_context *ctx, const TuneChoice &tc) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.link_mode = tc.link_mode;
    P.band = ctx->d_band;
    P.q = ctx->d_q;
    P.qk = ctx->d_qk;
    P.q_cap = ctx->q_cap;
    P.gen_thr = kNoGen;
    P.err = ctx->d_err;
    P.counters = ctx->d_counters;
    P.iter_cap = ctx->iter_cap;
    return P;
}

// Argument checks of the single-instance calls; need_bits is false for the
// calls that draw the bonds on the device.
ccl_status check_single_args(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                             const int32_t *col_idx, const uint32_t *bits, const int32_t *labels,
                             bool need_bits = true) {
    if (!ctx) return CCL_ERR_INVALID_ARGUMENT;
    if (n < 0 || n > CCL_MAX_SITES || nnz < 0 || nnz > INT32_MAX) return CCL_ERR_INVALID_ARGUMENT;
    if (n == 0) return CCL_OK;
    if (!row_ptr || !labels) return CCL_ERR_INVALID_ARGUMENT;
    if (nnz > 0 && (!col_idx || (need_bits && !bits))) return CCL_ERR_INVALID_ARGUMENT;
    return CCL_OK;
}

ccl_status label_single(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, const uint32_t *bits, int32_t *labels,
                        cudaStream_t s, const TuneChoice &tc, uint64_t gen_seed = 0,
                        uint64_t gen_thr = kNoGen) {
    const int64_t chunks = ((int64_t)n + kChunk - 1) / kChunk;
    ccl_status st = ensure_workspace(ctx, nnz, false);
    if (st != CCL_OK) return st;
    Params P = base_params(ctx, tc);
    P.K = 1;
    P.n_chunks = chunks;
    P.n_tiles = ((int64_t)n + kTileSites - 1) / kTileSites;
    P.one.row_ptr = row_ptr;
    P.one.col_idx = col_idx;
    P.one.bits = bits;
    P.one.labels = labels;
    set_bounds(P.one, row_ptr, (int64_t)n + 1, col_idx, nnz, bits, (nnz + 31) / 32);
    P.one.bit_off = 0;
    P.one.q_off = 0;
    P.one.chunk_begin = 0;
    P.one.tile_begin = 0;
    P.one.n = n;
    P.one.nnz = (int32_t)nnz;
    ctx->last.n_sites = n;
    ctx->last.nnz = nnz;
    ctx->last.n_inst = 1;
    if (gen_thr != kNoGen) {
        // bonds drawn on the device: a new seed every call, so no graph reuse
        P.gen_seed = gen_seed;
        P.gen_thr = gen_thr;
        return run(ctx, P, false, tc, s, nullptr, 0, false);
    }
    // the graph key covers every field of the instance (sizes included)
    return run(ctx, P, false, tc, s, nullptr, fnv1a(&P.one, sizeof(Inst)));
}

// Dense strided neighbour list: step (i) reads nn[i + k*n] (k < width) in
// place of a CSR row; the queue has n*width slots.
ccl_status label_dense(ccl_context *ctx, int32_t n, int32_t width, const int32_t *nn, const uint32_t *bits,
                       int32_t *labels, cudaStream_t s, const TuneChoice &tc, uint64_t gen_seed = 0,
                       uint64_t gen_thr = kNoGen) {
    const int64_t slots = (int64_t)n * width;
    ccl_status st = ensure_workspace(ctx, slots, false);
    if (st != CCL_OK) return st;
    Params P = base_params(ctx, tc);
    P.K = 1;
    P.n_chunks = ((int64_t)n + kChunk - 1) / kChunk;
    P.n_tiles = ((int64_t)n + kTileSites - 1) / kTileSites;
    P.dense = 1;
    P.nn = nn;
    P.nn_width = width;
    P.one.bits = bits;
    P.one.labels = labels;
    P.one.n = n;
    ctx->last.n_sites = n;
    ctx->last.nnz = slots;
    ctx->last.n_inst = 1;
    if (gen_thr != kNoGen) {
        P.gen_seed = gen_seed;
        P.gen_thr = gen_thr;
        return run(ctx, P, false, tc, s, nullptr, 0, false);
    }
    return run(ctx, P, false, tc, s, nullptr, fnv1a(&P.one, sizeof(Inst)) ^ (uint64_t)width);
}

// threshold of "(output >> 11) * 2^-53 < p": the smallest integer >= p * 2^53
uint64_t gen_threshold(double p) {
    return (uint64_t)std::ceil(p * 9007199254740992.0);
}

}  // namespace

namespace ccl {

// Labels the instances of `table` (row_ptr, col_idx, bits, bit_off, labels,
// n, nnz filled in by the caller) in one pass of the four steps on stream s.
// Used by the request loop, whose instances live in separate allocations.
ccl_status label_instances(ccl_context *ctx, std::vector<Inst> &table, cudaStream_t s) {
    int64_t chunks = 0, q = 0, tiles = 0;
    for (Inst &I : table) {
        I.q_off = q;
        I.chunk_begin = chunks;
        I.tile_begin = tiles;
        q += I.nnz;
        chunks += ((int64_t)I.n + kChunk - 1) / kChunk;
        tiles += ((int64_t)I.n + kTileSites - 1) / kTileSites;
    }
    if (chunks == 0) return CCL_OK;
    DeviceGuard guard(ctx->device);
    ccl_status st = ensure_workspace(ctx, q, table.size() > 1);
    if (st != CCL_OK) return st;
    const TuneChoice tc = ctx->opt;
    Params P = base_params(ctx, tc);
    P.K = (int32_t)table.size();
    P.n_chunks = chunks;
    P.n_tiles = tiles;
    if (table.size() == 1) {
        P.one = table[0];
        return run(ctx, P, false, tc, s, nullptr, 0, false);
    }
    return run(ctx, P, true, tc, s, &table, 0, false);
}

// Device bytes the context's residual-pair workspace holds now (it grows with
// the largest call and is kept until released).
int64_t workspace_bytes(const ccl_context *ctx) {
    return ctx->q_cap * (int64_t)sizeof(int2) + ctx->qk_cap * (int64_t)sizeof(int32_t);
}

// Growth factor of the residual-pair workspace: a call that needs more slots
// than the context holds takes max(need, factor * held) (1 = exactly the need).
void set_workspace_growth(ccl_context *ctx, double factor) {
    ctx->ws_growth = factor < 1.0 ? 1.0 : factor;
}

// Frees the residual-pair workspace (and the graphs that point into it); the
// next call allocates it again. The caller makes sure no work of the context
// is still running.
void release_workspace(ccl_context *ctx) {
    DeviceGuard guard(ctx->device);
    drop_graphs(ctx);
    if (ctx->d_q) cudaFree(ctx->d_q);
    if (ctx->d_qk) cudaFree(ctx->d_qk);
    ctx->d_q = nullptr;
    ctx->d_qk = nullptr;
    ctx->q_cap = ctx->qk_cap = 0;
    (void)cudaGetLastError();
}

}  // namespace ccl

extern "C" {

const char *ccl_status_string(int status) {
    switch (status) {
        case CCL_OK: return "CCL_OK";
        case CCL_ERR_INVALID_ARGUMENT: return "CCL_ERR_INVALID_ARGUMENT";
        case CCL_ERR_INDEX_OUT_OF_RANGE: return "CCL_ERR_INDEX_OUT_OF_RANGE";
        case CCL_ERR_ASYMMETRIC: return "CCL_ERR_ASYMMETRIC";
        case CCL_ERR_OUT_OF_MEMORY: return "CCL_ERR_OUT_OF_MEMORY";
        case CCL_ERR_NONCONVERGED: return "CCL_ERR_NONCONVERGED";
        case CCL_ERR_TIMEOUT: return "CCL_ERR_TIMEOUT";
        case CCL_ERR_REJECTED: return "CCL_ERR_REJECTED";
        case CCL_ERR_CUDA: return "CCL_ERR_CUDA";
        case CCL_ERR_NOT_FOUND: return "CCL_ERR_NOT_FOUND";
        default: return "CCL_ERR_UNKNOWN";
    }
}

int ccl_version(void) { return 100; }

ccl_status ccl_context_create(ccl_context **out, int device) {
    if (!out) return CCL_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    int ndev = 0;
    CCL_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(device);
    CCL_CUDA(cudaSetDevice(device));
    ccl_context *ctx = new ccl_context();
    ctx->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    int l2 = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    ctx->l2_bytes = l2;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_band, kMaxBands * sizeof(BandRec));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staging_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->stats_ev, cudaEventDisableTiming);
    // the opt-in shared memory of the staging buffers
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_init<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kInitSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_init<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kInitSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_init<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kInitSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_init_dense_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDenseSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_init_dense_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDenseSmem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ccl_context_destroy(ctx);
        return cuda_status(e);
    }
    if (const char *env = getenv("CCL_TUNE_CACHE")) {
        if (FILE *f = fopen(env, "r")) {
            char line[256];
            while (fgets(line, sizeof line, f)) {     // a line that does not parse is skipped
                long long cls;
                int a, b, c, d, r, q, w = 0, g = -1, k = -1;
                const int nf = sscanf(line, "%lld %d %d %d %d %d %d %d %d %d", &cls, &a, &b, &c, &d, &r, &q, &w, &g, &k);
                if (nf != 7 && nf != 10) continue;
                TuneChoice t;
                t.threads = a; t.ctas_per_sm = b < 0 ? 0 : b; t.pre_analysis = c ? 1 : 0;
                t.link_mode = d ? 1 : 0; t.refill = r ? 1 : 0; t.ana_seq = q ? 1 : 0;
                t.red_window = (w >= 64 && w <= 65536) ? w : 0;
                t.ana_group = g >= 0 ? g : -1;
                t.ana_park = k >= 0 ? (k ? 1 : 0) : -1;
                if (t.threads >= 64 && t.threads <= 512 && t.threads % 32 == 0) ctx->tune_table[cls] = t;
            }
            fclose(f);
        }
    }
    *out = ctx;
    return CCL_OK;
}

void ccl_context_destroy(ccl_context *ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.d_insts) cudaFree(g.d_insts);
    }
    if (ctx->d_q) cudaFree(ctx->d_q);
    if (ctx->d_qk) cudaFree(ctx->d_qk);
    if (ctx->d_band) cudaFree(ctx->d_band);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->d_insts) cudaFree(ctx->d_insts);
    if (ctx->h_insts) cudaFreeHost(ctx->h_insts);
    if (ctx->d_host_in) cudaFree(ctx->d_host_in);
    if (ctx->d_aux) cudaFree(ctx->d_aux);
    for (auto &e : ctx->part_ev) if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (auto &e : ctx->bh_up) if (e) cudaEventDestroy(e);
    for (auto &e : ctx->bh_done) if (e) cudaEventDestroy(e);
    if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
    if (ctx->staging_free) cudaEventDestroy(ctx->staging_free);
    if (ctx->stats_ev) cudaEventDestroy(ctx->stats_ev);
    for (auto &set : ctx->prof)
        for (auto &e : set) if (e) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    (void)cudaGetLastError();
    delete ctx;
}

ccl_status ccl_set_option(ccl_context *ctx, int option, int64_t value) {
    if (!ctx) return CCL_ERR_INVALID_ARGUMENT;
    switch (option) {
        case CCL_OPT_PRE_ANALYSIS: ctx->opt.pre_analysis = value ? 1 : 0; break;
        case CCL_OPT_BLOCK_THREADS:
            if (value < 64 || value > 512 || value % 32) return CCL_ERR_INVALID_ARGUMENT;
            ctx->opt.threads = (int)value;
            break;
        case CCL_OPT_USE_GRAPHS: ctx->use_graphs = value ? 1 : 0; return CCL_OK;
        case CCL_OPT_PROFILE:
            ctx->profile = value ? 1 : 0;
            ctx->prof_count = 0;
            ctx->have_times = 0;
            return CCL_OK;      // does not touch the tuning table
        case CCL_OPT_CTAS_PER_SM:
            if (value < 0 || value > 64) return CCL_ERR_INVALID_ARGUMENT;
            ctx->opt.ctas_per_sm = (int)value;
            break;
        case CCL_OPT_LINK_MODE: ctx->opt.link_mode = value ? 1 : 0; break;
        case CCL_OPT_REFILL: ctx->opt.refill = value ? 1 : 0; break;
        case CCL_OPT_ANALYSIS_ORDER: ctx->opt.ana_seq = value ? 1 : 0; break;
        case CCL_OPT_REDUCE_WINDOW:
            if (value != 0 && (value < 64 || value > 65536)) return CCL_ERR_INVALID_ARGUMENT;
            ctx->opt.red_window = (int)value;
            break;
        case CCL_OPT_ANALYSIS_GROUP:
            if (value < -1 || value > (int64_t)1 << 30) return CCL_ERR_INVALID_ARGUMENT;
            ctx->opt.ana_group = (int)value;
            break;
        case CCL_OPT_ANALYSIS_PARK:
            if (value < -1 || value > 1) return CCL_ERR_INVALID_ARGUMENT;
            ctx->opt.ana_park = (int)value;
            break;
        case CCL_OPT_ITER_CAP:
            if (value < 0 || value > INT32_MAX) return CCL_ERR_INVALID_ARGUMENT;
            ctx->iter_cap = (int32_t)value;
            {
                DeviceGuard guard(ctx->device);
                drop_graphs(ctx);     // captured graphs hold the old cap
            }
            return CCL_OK;            // does not touch the tuning table
        default: return CCL_ERR_INVALID_ARGUMENT;
    }
    // explicit options take effect over any tuned entry
    ctx->tune_table.clear();
    return CCL_OK;
}

ccl_status ccl_get_option(ccl_context *ctx, int option, int64_t *value) {
    if (!ctx || !value) return CCL_ERR_INVALID_ARGUMENT;
    switch (option) {
        case CCL_OPT_PRE_ANALYSIS: *value = ctx->opt.pre_analysis; break;
        case CCL_OPT_BLOCK_THREADS: *value = ctx->opt.threads; break;
        case CCL_OPT_USE_GRAPHS: *value = ctx->use_graphs; break;
        case CCL_OPT_PROFILE: *value = ctx->profile; break;
        case CCL_OPT_CTAS_PER_SM: *value = ctx->opt.ctas_per_sm; break;
        case CCL_OPT_LINK_MODE: *value = ctx->opt.link_mode; break;
        case CCL_OPT_REFILL: *value = ctx->opt.refill; break;
        case CCL_OPT_ANALYSIS_ORDER: *value = ctx->opt.ana_seq; break;
        case CCL_OPT_ITER_CAP: *value = ctx->iter_cap; break;
        case CCL_OPT_REDUCE_WINDOW: *value = ctx->opt.red_window; break;
        case CCL_OPT_ANALYSIS_GROUP: *value = ctx->opt.ana_group; break;
        case CCL_OPT_ANALYSIS_PARK: *value = ctx->opt.ana_park; break;
        default: return CCL_ERR_INVALID_ARGUMENT;
    }
    return CCL_OK;
}

ccl_status ccl_reserve(ccl_context *ctx, int64_t n_sites, int64_t nnz, int64_t n_chunks) {
    if (!ctx || n_sites < 0 || nnz < 0 || n_chunks < 0) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    (void)n_chunks;
    return ensure_workspace(ctx, nnz, true);
}

ccl_status ccl_label(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                     const int32_t *col_idx, const uint32_t *bits, int32_t *labels, void *stream) {
    ccl_status st = check_single_args(ctx, n, nnz, row_ptr, col_idx, bits, labels);
    if (st != CCL_OK || n == 0) {
        if (ctx && n == 0 && st == CCL_OK) { ctx->last = ccl_run_stats{}; ctx->last.n_inst = 1; }
        return st;
    }
    DeviceGuard guard(ctx->device);
    const TuneChoice tc = choice_for(ctx, n, nnz);
    return label_single(ctx, n, nnz, row_ptr, col_idx, bits, labels, (cudaStream_t)stream, tc);
}

namespace {
// The instance table of a batched call over the concatenated arrays (row_ptr,
// col_idx, bits, labels; any may be null when the matching total is 0), with
// the running chunk and tile counts. Checks the offsets.
ccl_status batch_table(int32_t K, const int64_t *site_off, const int64_t *ent_off, const int32_t *row_ptr,
                       const int32_t *col_idx, const uint32_t *bits, int32_t *labels, std::vector<Inst> &table,
                       int64_t &chunks, int64_t &tiles) {
    if (site_off[0] != 0 || ent_off[0] != 0) return CCL_ERR_INVALID_ARGUMENT;
    table.clear();
    table.reserve((size_t)K);
    chunks = 0;
    tiles = 0;
    const int64_t rp_len = site_off[K] + K, ci_len = ent_off[K], bits_len = (ent_off[K] + 31) / 32;
    for (int32_t k = 0; k < K; ++k) {
        const int64_t n = site_off[k + 1] - site_off[k];
        const int64_t nnz = ent_off[k + 1] - ent_off[k];
        if (n < 0 || nnz < 0 || n > CCL_MAX_SITES || nnz > INT32_MAX) return CCL_ERR_INVALID_ARGUMENT;
        Inst I;
        I.row_ptr = row_ptr + site_off[k] + k;
        I.col_idx = col_idx + ent_off[k];
        I.bits = bits;
        I.labels = labels + site_off[k];
        set_bounds(I, row_ptr, rp_len, col_idx, ci_len, bits, bits_len);
        I.bit_off = ent_off[k];
        I.q_off = ent_off[k];
        I.chunk_begin = chunks;
        I.tile_begin = tiles;
        I.n = (int32_t)n;
        I.nnz = (int32_t)nnz;
        table.push_back(I);
        chunks += (n + kChunk - 1) / kChunk;
        tiles += (n + kTileSites - 1) / kTileSites;
    }
    const int64_t n_tot = site_off[K], nnz_tot = ent_off[K];
    if (n_tot > 0 && (!row_ptr || !labels)) return CCL_ERR_INVALID_ARGUMENT;
    if (nnz_tot > 0 && (!col_idx || !bits)) return CCL_ERR_INVALID_ARGUMENT;
    return CCL_OK;
}

// ccl_label_batched with the launch settings given (tc) or looked up (null)
ccl_status label_batched(ccl_context *ctx, int32_t K, const int64_t *site_off, const int64_t *ent_off,
                         const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *bits,
                         int32_t *labels, void *stream, const TuneChoice *force_tc) {
    if (!ctx || K < 0) return CCL_ERR_INVALID_ARGUMENT;
    if (K == 0) { ctx->last = ccl_run_stats{}; return CCL_OK; }
    if (!site_off || !ent_off) return CCL_ERR_INVALID_ARGUMENT;
    std::vector<Inst> table;
    int64_t chunks = 0, tiles = 0;
    ccl_status st0 = batch_table(K, site_off, ent_off, row_ptr, col_idx, bits, labels, table, chunks, tiles);
    if (st0 != CCL_OK) return st0;
    const int64_t n_tot = site_off[K], nnz_tot = ent_off[K];
    ctx->last = ccl_run_stats{};
    ctx->last.n_inst = K;
    ctx->last.n_sites = n_tot;
    ctx->last.nnz = nnz_tot;
    if (chunks == 0) return CCL_OK;
    DeviceGuard guard(ctx->device);
    ccl_status st = ensure_workspace(ctx, nnz_tot, K > 1);
    if (st != CCL_OK) return st;
    const TuneChoice tc = force_tc ? *force_tc : choice_for_class(ctx, batch_class(n_tot, nnz_tot, K));
    Params P = base_params(ctx, tc);
    P.K = K;
    P.n_chunks = chunks;
    P.n_tiles = tiles;
    if (K == 1) {
        P.one = table[0];
        return run(ctx, P, false, tc, (cudaStream_t)stream, nullptr, fnv1a(&P.one, sizeof(Inst)));
    }
    uint64_t h = fnv1a(site_off, sizeof(int64_t) * (size_t)(K + 1));
    h = fnv1a(ent_off, sizeof(int64_t) * (size_t)(K + 1), h);
    std::vector<int64_t> offs(site_off, site_off + K + 1);
    offs.insert(offs.end(), ent_off, ent_off + K + 1);
    return run(ctx, P, true, tc, (cudaStream_t)stream, &table, h, true, &offs);
}
}  // namespace

ccl_status ccl_label_batched(ccl_context *ctx, int32_t K, const int64_t *site_off,
                             const int64_t *ent_off, const int32_t *row_ptr,
                             const int32_t *col_idx, const uint32_t *bits, int32_t *labels,
                             void *stream) {
    return label_batched(ctx, K, site_off, ent_off, row_ptr, col_idx, bits, labels, stream, nullptr);
}

ccl_status ccl_autotune_batched(ccl_context *ctx, int32_t K, const int64_t *site_off,
                                const int64_t *ent_off, const int32_t *row_ptr, const int32_t *col_idx,
                                const uint32_t *bits, int32_t *labels, void *stream, float *best_ms) {
    if (!ctx || K < 0) return CCL_ERR_INVALID_ARGUMENT;
    if (K == 0) return CCL_OK;
    if (!site_off || !ent_off) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<TuneChoice> cands;
    for (int pre = 0; pre < 2; ++pre)
        for (int lm = 0; lm < 2; ++lm)
            for (int rf = 0; rf < 2; ++rf)
                for (int sq = 0; sq < 2; ++sq) {
                    TuneChoice tc;
                    tc.threads = 256; tc.ctas_per_sm = 0; tc.pre_analysis = pre; tc.link_mode = lm;
                    tc.refill = rf; tc.ana_seq = sq;
                    cands.push_back(tc);
                }
    TuneChoice best = ctx->opt;
    float best_t = 1e30f;
    auto runner = [&](const TuneChoice &tc) {
        return label_batched(ctx, K, site_off, ent_off, row_ptr, col_idx, bits, labels, stream, &tc);
    };
    ccl_status st = tune_over(ctx, s, cands, 3, best, best_t, runner);
    if (st == CCL_OK) st = tune_tail(ctx, s, 3, best, best_t, runner);
    if (st != CCL_OK) return st;
    const int64_t n_tot = site_off[K], nnz_tot = ent_off[K];
    ctx->tune_table[batch_class(n_tot, nnz_tot, K)] = best;
    if (best_ms) *best_ms = best_t;
    // leave the correct labels with the chosen settings
    return label_batched(ctx, K, site_off, ent_off, row_ptr, col_idx, bits, labels, stream, &best);
}

ccl_status ccl_label_random(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                            const int32_t *col_idx, uint64_t seed, double p, int32_t *labels,
                            void *stream) {
    ccl_status st = check_single_args(ctx, n, nnz, row_ptr, col_idx, nullptr, labels, false);
    if (st != CCL_OK || n == 0) return st;
    if (!(p >= 0.0 && p <= 1.0)) return CCL_ERR_INVALID_ARGUMENT;
    // open iff (output >> 11) * 2^-53 < p  <=>  (output >> 11) < ceil(p * 2^53)
    const uint64_t thr = gen_threshold(p);
    DeviceGuard guard(ctx->device);
    const TuneChoice tc = choice_for(ctx, n, nnz);
    return label_single(ctx, n, nnz, row_ptr, col_idx, nullptr, labels, (cudaStream_t)stream, tc, seed, thr);
}

namespace {
ccl_status check_dense_args(ccl_context *ctx, int32_t n, int32_t width, const int32_t *nn, const void *bits,
                            const int32_t *labels, bool need_bits = true) {
    if (!ctx || n < 0 || n > CCL_MAX_SITES || width < 0 || width > CCL_DENSE_MAX_WIDTH)
        return CCL_ERR_INVALID_ARGUMENT;
    if (n == 0) return CCL_OK;
    if (!labels || (width > 0 && (!nn || (need_bits && !bits)))) return CCL_ERR_INVALID_ARGUMENT;
    return CCL_OK;
}
}  // namespace

ccl_status ccl_label_dense(ccl_context *ctx, int32_t n, int32_t width, const int32_t *nn,
                           const uint32_t *open_bits, int32_t *labels, void *stream) {
    ccl_status st = check_dense_args(ctx, n, width, nn, open_bits, labels);
    if (st != CCL_OK || n == 0) return st;
    DeviceGuard guard(ctx->device);
    const TuneChoice tc = choice_for(ctx, n, (int64_t)n * width);
    return label_dense(ctx, n, width, width ? nn : nullptr, width ? open_bits : nullptr, labels,
                       (cudaStream_t)stream, tc);
}

ccl_status ccl_label_dense_random(ccl_context *ctx, int32_t n, int32_t width, const int32_t *nn,
                                  uint64_t seed, double p, int32_t *labels, void *stream) {
    ccl_status st = check_dense_args(ctx, n, width, nn, nullptr, labels, false);
    if (st != CCL_OK || n == 0) return st;
    if (!(p >= 0.0 && p <= 1.0)) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    const TuneChoice tc = choice_for(ctx, n, (int64_t)n * width);
    return label_dense(ctx, n, width, width ? nn : nullptr, nullptr, labels, (cudaStream_t)stream, tc, seed,
                       gen_threshold(p));
}

namespace {
ccl_status ensure_aux(ccl_context *ctx, int64_t bytes) {
    if (bytes <= ctx->aux_cap) return CCL_OK;
    if (ctx->d_aux) cudaFree(ctx->d_aux);
    ctx->d_aux = nullptr;
    ctx->aux_cap = 0;
    CCL_CUDA(cudaMalloc(&ctx->d_aux, (size_t)bytes));
    ctx->aux_cap = bytes;
    return CCL_OK;
}
}  // namespace

ccl_status ccl_relabel(ccl_context *ctx, int32_t n, const int32_t *labels, int32_t *seq,
                       int32_t *n_clusters, int32_t *sizes, void *stream) {
    if (!ctx || n < 0 || !n_clusters) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        CCL_CUDA(cudaMemsetAsync(n_clusters, 0, sizeof(int32_t), s));
        return CCL_OK;
    }
    if (!labels || !seq || labels == seq) return CCL_ERR_INVALID_ARGUMENT;
    const int64_t nb = ((int64_t)n + kRelBlock - 1) / kRelBlock;
    ccl_status st = ensure_aux(ctx, nb * (int64_t)sizeof(int32_t));
    if (st != CCL_OK) return st;
    int32_t *cnt = (int32_t *)ctx->d_aux;
    k_root_counts<<<(unsigned)nb, kRelThreads, 0, s>>>(n, labels, cnt);
    k_scan_counts<<<1, 1024, 0, s>>>((int32_t)nb, cnt, n_clusters);
    k_root_ids<<<(unsigned)nb, kRelThreads, 0, s>>>(n, labels, cnt, seq, sizes);
    const int64_t g = std::min<int64_t>((int64_t)ctx->num_sms * 8, ((int64_t)n + 255) / 256);
    k_site_ids<<<(unsigned)g, 256, 0, s>>>(n, labels, seq);
    if (sizes) k_sizes<<<(unsigned)g, 256, 0, s>>>(n, seq, sizes);
    CCL_CUDA(cudaGetLastError());
    return CCL_OK;
}

ccl_status ccl_spanning(ccl_context *ctx, int32_t n, const int32_t *labels, const int32_t *top,
                        int32_t n_top, const int32_t *bottom, int32_t n_bottom, int32_t *result,
                        void *stream) {
    if (!ctx || n < 0 || n_top < 0 || n_bottom < 0 || !result) return CCL_ERR_INVALID_ARGUMENT;
    if (n > 0 && !labels) return CCL_ERR_INVALID_ARGUMENT;
    if ((n_top > 0 && !top) || (n_bottom > 0 && !bottom)) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t words = ((int64_t)n + 31) / 32;
    ccl_status st = ensure_aux(ctx, std::max<int64_t>(words, 1) * (int64_t)sizeof(uint32_t));
    if (st != CCL_OK) return st;
    uint32_t *flags = (uint32_t *)ctx->d_aux;
    if (words) CCL_CUDA(cudaMemsetAsync(flags, 0, (size_t)words * sizeof(uint32_t), s));
    const int64_t gt = std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms * 4, ((int64_t)n_top + 255) / 256));
    const int64_t gb = std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms * 4, ((int64_t)n_bottom + 255) / 256));
    k_span_mark<<<(unsigned)gt, 256, 0, s>>>(n, labels, top, n_top, flags, result, ctx->d_err);
    k_span_check<<<(unsigned)gb, 256, 0, s>>>(n, labels, bottom, n_bottom, flags, result, ctx->d_err);
    k_span_finish<<<1, 1, 0, s>>>(result);
    CCL_CUDA(cudaGetLastError());
    return CCL_OK;
}

ccl_status ccl_largest_cluster(ccl_context *ctx, int32_t n, const int32_t *labels, int32_t *result,
                               void *stream) {
    if (!ctx || n < 0 || !result) return CCL_ERR_INVALID_ARGUMENT;
    if (n > 0 && !labels) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: the 64-bit best key, then one count per site
    ccl_status st = ensure_aux(ctx, 16 + (int64_t)n * (int64_t)sizeof(int32_t));
    if (st != CCL_OK) return st;
    unsigned long long *best = (unsigned long long *)ctx->d_aux;
    int32_t *cnt = (int32_t *)((char *)ctx->d_aux + 16);
    CCL_CUDA(cudaMemsetAsync(ctx->d_aux, 0, 16 + (size_t)n * sizeof(int32_t), s));
    if (n > 0) {
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 8, ((int64_t)n + 255) / 256));
        k_label_counts<<<(unsigned)g, 256, 0, s>>>(n, labels, cnt, ctx->d_err);
        k_largest<<<(unsigned)g, 256, 0, s>>>(n, cnt, best);
    }
    k_largest_finish<<<1, 1, 0, s>>>(best, result);
    CCL_CUDA(cudaGetLastError());
    return CCL_OK;
}

ccl_status ccl_sync(ccl_context *ctx, void *stream, int64_t timeout_ms) {
    if (!ctx) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) { (void)cudaGetLastError(); return cuda_status(e); }
        if (timeout_ms >= 0) {
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_ms) return CCL_ERR_TIMEOUT;
        }
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // the error word is read (and cleared) on the context's own non-blocking
    // stream, so the read waits for nothing else on the device
    unsigned err = 0;
    CCL_CUDA(cudaMemcpyAsync(&err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->cap_stream));
    CCL_CUDA(cudaStreamSynchronize(ctx->cap_stream));
    if (err) {
        CCL_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->cap_stream));
        CCL_CUDA(cudaStreamSynchronize(ctx->cap_stream));
    }
    if (err & kErrIndex) return CCL_ERR_INDEX_OUT_OF_RANGE;
    if (err & kErrShape) return CCL_ERR_INVALID_ARGUMENT;
    if (err & kErrNonconv) return CCL_ERR_NONCONVERGED;
    if (err & kErrAsym) return CCL_ERR_ASYMMETRIC;
    return CCL_OK;
}

namespace {
constexpr int kHostParts = 4;        // upload parts of the single-instance host-buffer path

// The host-buffer path for inputs of at least 64 tiles: the input goes up in
// kHostParts site ranges on the copy stream, and step (i) on each range starts
// as soon as its rows, columns and bits have arrived (step (i) reads only the
// rows of its own tiles), so the upload of the later ranges overlaps it.
// Steps (ii)-(iv) then run once over all band records.
ccl_status label_host_parts(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                            const int32_t *col_idx, const uint32_t *bits, int32_t *d_rp, int32_t *d_ci,
                            uint32_t *d_bits, int32_t *d_lab, cudaStream_t s, const TuneChoice &tc) {
    if (!ctx->copy_stream) {
        CCL_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (auto &e : ctx->part_ev) CCL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const int64_t tiles = ((int64_t)n + kTileSites - 1) / kTileSites;
    int64_t ts[kHostParts + 1], es[kHostParts + 1];       // part boundaries: tiles, CSR entries
    for (int k = 0; k <= kHostParts; ++k) {
        ts[k] = tiles * k / kHostParts;
        es[k] = row_ptr[std::min<int64_t>(ts[k] * kTileSites, n)];
        if (es[k] < 0 || es[k] > nnz || (k > 0 && es[k] < es[k - 1])) return CCL_ERR_INVALID_ARGUMENT;
    }
    ccl_status st = ensure_workspace(ctx, nnz, false);
    if (st != CCL_OK) return st;
    Params P = base_params(ctx, tc);
    P.K = 1;
    P.n_chunks = ((int64_t)n + kChunk - 1) / kChunk;
    P.one.row_ptr = d_rp;
    P.one.col_idx = d_ci;
    P.one.bits = d_bits;
    P.one.labels = d_lab;
    set_bounds(P.one, d_rp, (int64_t)n + 1, d_ci, nnz, d_bits, (nnz + 31) / 32);
    P.one.n = n;
    P.one.nnz = (int32_t)nnz;
    ctx->last.n_sites = n;
    ctx->last.nnz = nnz;
    ctx->last.n_inst = 1;
    ctx->last.used_graph = 0;
    CCL_CUDA(cudaMemsetAsync(P.counters, 0, 4 * sizeof(unsigned long long), s));
    CCL_CUDA(cudaMemsetAsync(P.band, 0, (size_t)kMaxBands * sizeof(BandRec), s));
    // the uploads may not overwrite the buffers before earlier work on s is done
    CCL_CUDA(cudaEventRecord(ctx->part_ev[kHostParts], s));
    CCL_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->part_ev[kHostParts], 0));
    int32_t band_off = 0;
    for (int k = 0; k < kHostParts; ++k) {
        const int64_t t0 = ts[k], t1 = ts[k + 1];
        const int64_t s0 = t0 * kTileSites, s1 = std::min<int64_t>(t1 * kTileSites, n);
        const int64_t e0 = es[k], e1 = es[k + 1];
        CCL_CUDA(cudaMemcpyAsync(d_rp + s0, row_ptr + s0, (size_t)(s1 - s0 + 1) * 4, cudaMemcpyHostToDevice,
                                 ctx->copy_stream));
        if (e1 > e0) {
            CCL_CUDA(cudaMemcpyAsync(d_ci + e0, col_idx + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
            const int64_t w0 = e0 >> 5, w1 = ((e1 - 1) >> 5) + 1;
            CCL_CUDA(cudaMemcpyAsync(d_bits + w0, bits + w0, (size_t)(w1 - w0) * 4, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
        }
        CCL_CUDA(cudaEventRecord(ctx->part_ev[k], ctx->copy_stream));
        CCL_CUDA(cudaStreamWaitEvent(s, ctx->part_ev[k], 0));
        P.tile_off = t0;
        P.n_tiles = t1 - t0;
        P.band_off = band_off;
        const int64_t g = init_grid(ctx, P, false, kMaxBands / kHostParts);
        st = launch_init(P, false, g, s);
        if (st != CCL_OK) return st;
        band_off += (int32_t)g;
    }
    P.tile_off = 0;
    P.n_tiles = tiles;
    P.band_off = 0;
    P.n_bands = band_off;
    st = enqueue_tail(ctx, P, false, tc, s, false);
    if (st == CCL_OK) CCL_CUDA(cudaEventRecord(ctx->stats_ev, s));
    return st;
}
}  // namespace

ccl_status ccl_label_host(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const uint32_t *bits, int32_t *labels,
                          void *stream) {
    ccl_status st = check_single_args(ctx, n, nnz, row_ptr, col_idx, bits, labels);
    if (st != CCL_OK || n == 0) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nwords = (nnz + 31) / 32;
    const size_t b_rp = (size_t)(n + 1) * 4, b_ci = (size_t)nnz * 4, b_bits = (size_t)nwords * 4,
                 b_lab = (size_t)n * 4;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al(b_rp) + al(b_ci) + al(b_bits) + al(b_lab);
    if ((int64_t)need > ctx->host_in_cap) {
        CCL_CUDA(cudaStreamSynchronize(s));
        if (ctx->d_host_in) cudaFree(ctx->d_host_in);
        ctx->d_host_in = nullptr;
        ctx->host_in_cap = 0;
        drop_graphs(ctx);    // graphs may hold pointers into the old buffer
        CCL_CUDA(cudaMalloc(&ctx->d_host_in, need));
        ctx->host_in_cap = (int64_t)need;
    }
    char *base = (char *)ctx->d_host_in;
    int32_t *d_rp = (int32_t *)base;
    int32_t *d_ci = (int32_t *)(base + al(b_rp));
    uint32_t *d_bits = (uint32_t *)(base + al(b_rp) + al(b_ci));
    int32_t *d_lab = (int32_t *)(base + al(b_rp) + al(b_ci) + al(b_bits));
    const TuneChoice tc = choice_for(ctx, n, nnz);
    const int64_t tiles = ((int64_t)n + kTileSites - 1) / kTileSites;
    if (tiles >= 64 && nnz > 0 && !ctx->profile && !stream_capturing(s)) {
        st = label_host_parts(ctx, n, nnz, row_ptr, col_idx, bits, d_rp, d_ci, d_bits, d_lab, s, tc);
    } else {
        CCL_CUDA(cudaMemcpyAsync(d_rp, row_ptr, b_rp, cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            CCL_CUDA(cudaMemcpyAsync(d_ci, col_idx, b_ci, cudaMemcpyHostToDevice, s));
            CCL_CUDA(cudaMemcpyAsync(d_bits, bits, b_bits, cudaMemcpyHostToDevice, s));
        }
        st = label_single(ctx, n, nnz, d_rp, nnz ? d_ci : nullptr, nnz ? d_bits : nullptr, d_lab, s, tc);
    }
    if (st != CCL_OK) return st;
    CCL_CUDA(cudaMemcpyAsync(labels, d_lab, b_lab, cudaMemcpyDeviceToHost, s));
    return ccl_sync(ctx, stream, -1);
}

ccl_status ccl_label_batched_host(ccl_context *ctx, int32_t K, const int64_t *site_off, const int64_t *ent_off,
                                  const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *bits,
                                  int32_t *labels, void *stream) {
    if (!ctx || K < 0) return CCL_ERR_INVALID_ARGUMENT;
    if (K == 0) { ctx->last = ccl_run_stats{}; return CCL_OK; }
    if (!site_off || !ent_off) return CCL_ERR_INVALID_ARGUMENT;
    if (site_off[0] != 0 || ent_off[0] != 0 || site_off[K] < 0 || ent_off[K] < 0) return CCL_ERR_INVALID_ARGUMENT;
    const int64_t n_tot = site_off[K], nnz_tot = ent_off[K];
    if (n_tot > 0 && (!row_ptr || !labels)) return CCL_ERR_INVALID_ARGUMENT;
    if (nnz_tot > 0 && (!col_idx || !bits)) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rp_len = n_tot + K, words = (nnz_tot + 31) / 32;
    const size_t b_rp = (size_t)rp_len * 4, b_ci = (size_t)nnz_tot * 4, b_bits = (size_t)words * 4,
                 b_lab = (size_t)n_tot * 4;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al(b_rp) + al(b_ci) + al(b_bits) + al(b_lab);
    if ((int64_t)need > ctx->host_in_cap) {
        CCL_CUDA(cudaStreamSynchronize(s));
        if (ctx->d_host_in) cudaFree(ctx->d_host_in);
        ctx->d_host_in = nullptr;
        ctx->host_in_cap = 0;
        drop_graphs(ctx);    // graphs may hold pointers into the old buffer
        CCL_CUDA(cudaMalloc(&ctx->d_host_in, need));
        ctx->host_in_cap = (int64_t)need;
    }
    char *base = (char *)ctx->d_host_in;
    int32_t *d_rp = (int32_t *)base;
    int32_t *d_ci = (int32_t *)(base + al(b_rp));
    uint32_t *d_bits = (uint32_t *)(base + al(b_rp) + al(b_ci));
    int32_t *d_lab = (int32_t *)(base + al(b_rp) + al(b_ci) + al(b_bits));
    std::vector<Inst> table;
    int64_t chunks = 0, tiles = 0;
    ccl_status st = batch_table(K, site_off, ent_off, d_rp, nnz_tot ? d_ci : nullptr, nnz_tot ? d_bits : nullptr,
                                d_lab, table, chunks, tiles);
    if (st != CCL_OK) return st;
    ctx->last = ccl_run_stats{};
    ctx->last.n_inst = K;
    ctx->last.n_sites = n_tot;
    ctx->last.nnz = nnz_tot;
    if (chunks == 0) return CCL_OK;
    st = ensure_workspace(ctx, nnz_tot, K > 1);
    if (st != CCL_OK) return st;
    if (!ctx->copy_stream) {
        CCL_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (auto &e : ctx->part_ev) CCL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (!ctx->d2h_stream) {
        CCL_CUDA(cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking));
        for (auto &e : ctx->bh_up) CCL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : ctx->bh_done) CCL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const TuneChoice tc = choice_for_class(ctx, batch_class(n_tot, nnz_tot, K));
    // The instances are independent, so the batch runs as kParts groups of
    // instances of about equal site counts, each through all four steps: the
    // upload of later groups (copy stream) and the download of the labels of
    // earlier ones (download stream) overlap the labelling of a group (the
    // caller's stream), and uploads and downloads use the two directions of
    // the link at once.
    constexpr int kParts = (int)(sizeof(ctx->bh_up) / sizeof(ctx->bh_up[0]));
    int32_t kb[kParts + 1];
    kb[0] = 0;
    kb[kParts] = K;
    for (int part = 1; part < kParts; ++part) {
        const int64_t target = n_tot * part / kParts;
        const int32_t k = (int32_t)(std::upper_bound(site_off, site_off + K + 1, target) - site_off - 1);
        kb[part] = std::min(K, std::max(k, kb[part - 1]));
    }
    // the uploads may not overwrite the buffers before earlier work on s is done
    CCL_CUDA(cudaEventRecord(ctx->bh_done[kParts], s));
    CCL_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->bh_done[kParts], 0));
    CCL_CUDA(cudaStreamWaitEvent(ctx->d2h_stream, ctx->bh_done[kParts], 0));
    for (int part = 0; part < kParts; ++part) {
        const int32_t k0 = kb[part], k1 = kb[part + 1];
        const int64_t r0 = site_off[k0] + k0, r1 = site_off[k1] + k1;    // row pointers of instances [k0, k1)
        const int64_t e0 = ent_off[k0], e1 = ent_off[k1];
        if (r1 > r0)
            CCL_CUDA(cudaMemcpyAsync(d_rp + r0, row_ptr + r0, (size_t)(r1 - r0) * 4, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
        if (e1 > e0) {
            CCL_CUDA(cudaMemcpyAsync(d_ci + e0, col_idx + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
            const int64_t w0 = e0 >> 5, w1 = ((e1 - 1) >> 5) + 1;    // a word shared by two groups comes twice
            CCL_CUDA(cudaMemcpyAsync(d_bits + w0, bits + w0, (size_t)(w1 - w0) * 4, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
        }
        CCL_CUDA(cudaEventRecord(ctx->bh_up[part], ctx->copy_stream));
    }
    // the statistics counters add up over the groups
    CCL_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), s));
    // an error after the first download was queued: wait for the downloads
    // already queued, so none writes into `labels` after the return
    auto fail = [&](ccl_status e) {
        (void)cudaStreamSynchronize(ctx->d2h_stream);
        (void)cudaGetLastError();
        return e;
    };
    std::vector<Inst> tg;
    for (int part = 0; part < kParts; ++part) {
        const int32_t k0 = kb[part], k1 = kb[part + 1];
        const int64_t c0 = k0 < K ? table[(size_t)k0].chunk_begin : chunks;
        const int64_t c1 = k1 < K ? table[(size_t)k1].chunk_begin : chunks;
        if (c1 == c0) continue;                 // no sites in this group
        const int64_t t0 = table[(size_t)k0].tile_begin;
        const int64_t t1 = k1 < K ? table[(size_t)k1].tile_begin : tiles;
        // the group's entries of the batch table, chunk, tile and queue
        // offsets counted from the group's first instance (pointers, bit
        // offsets and copy bounds stay those of the whole batch)
        tg.assign(table.begin() + k0, table.begin() + k1);
        for (Inst &I : tg) {
            I.chunk_begin -= c0;
            I.tile_begin -= t0;
            I.q_off -= ent_off[k0];
        }
        const bool bat = k1 - k0 > 1;
        Params P = base_params(ctx, tc);
        P.K = k1 - k0;
        P.n_chunks = c1 - c0;
        if (bat) {
            st = upload_table(ctx, tg, s);
            if (st != CCL_OK) return fail(st);
            P.insts = ctx->d_insts;
        } else {
            P.one = tg[0];
        }
        if (cudaMemsetAsync(P.band, 0, (size_t)kMaxBands * sizeof(BandRec), s) != cudaSuccess ||
            cudaStreamWaitEvent(s, ctx->bh_up[part], 0) != cudaSuccess)
            return fail(CCL_ERR_CUDA);
        P.tile_off = 0;
        P.n_tiles = t1 - t0;
        P.band_off = 0;
        const int64_t g = init_grid(ctx, P, bat, kMaxBands);
        st = launch_init(P, bat, g, s);
        if (st != CCL_OK) return fail(st);
        P.n_bands = (int32_t)g;
        st = enqueue_tail(ctx, P, bat, tc, s, false);
        if (st != CCL_OK) return fail(st);
        if (cudaEventRecord(ctx->bh_done[part], s) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->d2h_stream, ctx->bh_done[part], 0) != cudaSuccess ||
            cudaMemcpyAsync(labels + site_off[k0], d_lab + site_off[k0], (size_t)(site_off[k1] - site_off[k0]) * 4,
                            cudaMemcpyDeviceToHost, ctx->d2h_stream) != cudaSuccess)
            return fail(CCL_ERR_CUDA);
    }
    // later work on s (and ccl_sync) comes after the downloads
    if (cudaEventRecord(ctx->stats_ev, s) != cudaSuccess ||
        cudaEventRecord(ctx->bh_done[kParts], ctx->d2h_stream) != cudaSuccess ||
        cudaStreamWaitEvent(s, ctx->bh_done[kParts], 0) != cudaSuccess)
        return fail(CCL_ERR_CUDA);
    ctx->last.n_inst = K;
    ctx->last.n_sites = n_tot;
    ctx->last.nnz = nnz_tot;
    return ccl_sync(ctx, stream, -1);
}

ccl_status ccl_validate(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, const uint32_t *bits, void *stream) {
    ccl_status st = check_single_args(ctx, n, nnz, row_ptr, col_idx, bits, (const int32_t *)1);
    if (st != CCL_OK || n == 0) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // drain earlier work so that its latched errors are not reported here
    st = ccl_sync(ctx, stream, -1);
    (void)st;
    const int threads = 256;
    const int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * 8, ((int64_t)n + threads - 1) / threads);
    k_validate<<<(unsigned)std::max<int64_t>(grid, 1), threads, 0, s>>>(n, nnz, row_ptr, col_idx, bits,
                                                                      ctx->d_err);
    CCL_CUDA(cudaGetLastError());
    return ccl_sync(ctx, stream, -1);
}

ccl_status ccl_get_stats(ccl_context *ctx, ccl_run_stats *out) {
    if (!ctx || !out) return CCL_ERR_INVALID_ARGUMENT;
    DeviceGuard guard(ctx->device);
    CCL_CUDA(cudaEventSynchronize(ctx->stats_ev));    // the last labelling call has finished
    unsigned long long c[4] = {0, 0, 0, 0};
    // read on the context's own non-blocking stream: no wait on other streams
    CCL_CUDA(cudaMemcpyAsync(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->cap_stream));
    CCL_CUDA(cudaStreamSynchronize(ctx->cap_stream));
    *out = ctx->last;
    out->residual_pairs = (int64_t)c[0];
    out->chase_loads = (int64_t)c[1];
    out->merge_atomics = (int64_t)c[2];
    out->reduce_iterations = (int64_t)c[3];
    return CCL_OK;
}

ccl_status ccl_get_step_times(ccl_context *ctx, float *ms, int32_t n) {
    if (!ctx || !ms || n < 0) return CCL_ERR_INVALID_ARGUMENT;
    if (!ctx->have_times || ctx->prof_count == 0) return CCL_ERR_NOT_FOUND;
    DeviceGuard guard(ctx->device);
    const int64_t calls = std::min<int64_t>(ctx->prof_count, kProfRing);
    const size_t last = (size_t)((ctx->prof_count - 1) % kProfRing);
    CCL_CUDA(cudaEventSynchronize(ctx->prof[last][4]));
    double acc[4] = {0, 0, 0, 0};
    for (int64_t c = 0; c < calls; ++c) {
        const size_t slot = (size_t)((ctx->prof_count - 1 - c) % kProfRing);
        for (int i = 0; i < 4; ++i) {
            float t = 0;
            CCL_CUDA(cudaEventElapsedTime(&t, ctx->prof[slot][(size_t)i], ctx->prof[slot][(size_t)i + 1]));
            acc[i] += t;
        }
    }
    for (int i = 0; i < std::min<int32_t>(n, 4); ++i) ms[i] = (float)(acc[i] / (double)calls);
    if (n > 4) ms[4] = (float)calls;
    return CCL_OK;
}

ccl_status ccl_autotune(ccl_context *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, const uint32_t *bits, int32_t *labels, void *stream,
                        float *best_ms) {
    ccl_status st = check_single_args(ctx, n, nnz, row_ptr, col_idx, bits, labels);
    if (st != CCL_OK || n == 0) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TuneChoice best = ctx->opt;
    float best_t = 1e30f;
    std::vector<TuneChoice> cands;
    for (int T : {128, 256, 512})
        for (int pre = 0; pre < 2; ++pre)
            for (int lm = 0; lm < 2; ++lm)
                for (int rf = 0; rf < 2; ++rf)
                    for (int sq = 0; sq < 2; ++sq) {
                        TuneChoice tc;
                        tc.threads = T; tc.ctas_per_sm = 0; tc.pre_analysis = pre; tc.link_mode = lm;
                        tc.refill = rf; tc.ana_seq = sq;
                        cands.push_back(tc);
                    }
    auto runner = [&](const TuneChoice &tc) {
        return label_single(ctx, n, nnz, row_ptr, col_idx, bits, labels, s, tc);
    };
    st = tune_over(ctx, s, cands, 4, best, best_t, runner);
    if (st == CCL_OK) st = tune_tail(ctx, s, 4, best, best_t, runner);
    if (st != CCL_OK) return st;
    ctx->tune_table[size_class(n, nnz)] = best;
    // also the default for other size classes, except the settings that
    // follow the size of the call
    ctx->opt = best;
    ctx->opt.red_window = 0;
    ctx->opt.ana_group = -1;
    ctx->opt.ana_park = -1;
    if (const char *env = getenv("CCL_TUNE_CACHE")) {
        if (FILE *f = fopen(env, "w")) {
            for (auto &kv : ctx->tune_table)
                fprintf(f, "%lld %d %d %d %d %d %d %d %d %d\n", (long long)kv.first, kv.second.threads,
                        kv.second.ctas_per_sm, kv.second.pre_analysis, kv.second.link_mode, kv.second.refill,
                        kv.second.ana_seq, kv.second.red_window, kv.second.ana_group, kv.second.ana_park);
            fclose(f);
        }
    }
    // leave the correct labels in `labels` with the chosen shape
    st = label_single(ctx, n, nnz, row_ptr, col_idx, bits, labels, s, best);
    if (st != CCL_OK) return st;
    if (best_ms) *best_ms = best_t;
    return ccl_sync(ctx, stream, -1);
}

}  // extern "C"
