// Request loop of include/ccl.h: continuous batching of labelling requests.
//
// Two threads own the GPU side.
//   The uploader admits pending requests while their device bytes fit the
//   budget (the free HBM seen at start minus a reserve, and the configured
//   cap), allocates their buffers from a stream-ordered pool and uploads
//   them on an upload stream (copies from pageable memory block it while
//   the driver stages them, so they are kept off the launch loop).
//   The server thread, each tick,
//   1. gathers every request whose upload has finished into one batched
//      launch of the four labelling steps on a free compute stream (each
//      compute stream has a labelling context of its own), followed by the
//      copies of the labels back to host memory;
//   2. retires finished batches: frees their buffers, stamps latencies and
//      wakes waiters.
// Later requests are therefore uploaded and labelled while earlier batches
// are still running. Every wait on the device is an event query; nothing
// spins on the GPU.
#include <ccl.h>

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ccl_types.cuh"

namespace ccl {
ccl_status label_instances(ccl_context *ctx, std::vector<Inst> &table, cudaStream_t s);
int64_t workspace_bytes(const ccl_context *ctx);
void release_workspace(ccl_context *ctx);
void set_workspace_growth(ccl_context *ctx, double factor);
}

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kUploaders = 2;    // uploader threads, each with a stream of its own
// a request whose device buffer cannot be allocated although the server holds
// nothing for other requests fails with CCL_ERR_OUT_OF_MEMORY after this long
constexpr auto kAllocGiveUp = std::chrono::milliseconds(2000);

struct Req {
    uint64_t ticket = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    // host copy: one block of the pinned staging arena when it had room
    // (row_ptr | col_idx | bits | labels), else pageable vectors
    char *h = nullptr;
    size_t h_bytes = 0;
    // no-copy requests: the caller's arrays, uploaded from where they are;
    // only the labels come back through an arena block (lab_h) when it has room
    const int32_t *ext_rp = nullptr, *ext_ci = nullptr;
    const uint32_t *ext_bits = nullptr;
    int32_t *lab_h = nullptr;
    size_t lab_bytes = 0;
    std::vector<int32_t> v_row_ptr, v_col_idx, v_labels;
    std::vector<uint32_t> v_bits;
    int64_t dev_bytes = 0;      // its device buffer: inputs and labels
    int64_t ws_bytes = 0;       // its share of a batched launch's workspace (until launched)
    bool alloc_failing = false; // the pool could not allocate its buffer ...
    Clock::time_point t_alloc_fail;  // ... since then
    char *d_mem = nullptr;
    cudaEvent_t uploaded = nullptr;
    Clock::time_point t_submit, t_done;
    Clock::time_point t_admit, t_ready, t_launch;   // upload started, upload seen done, batch launched
    ccl_status status = CCL_OK;
    bool done = false;
    bool dropped = false;   // ended by ccl_server_destroy before it was labelled
};

struct Batch {
    std::vector<std::shared_ptr<Req>> reqs;
    int slot = -1;
    cudaEvent_t finished = nullptr;
};

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct HostLayout {
    size_t rp, ci, bits, lab, total;
    HostLayout(int32_t n, int64_t nnz) {
        rp = 0;
        ci = al256((size_t)(n + 1) * 4);
        bits = ci + al256((size_t)nnz * 4);
        lab = bits + al256((size_t)std::max<int64_t>(1, (nnz + 31) / 32) * 4);
        total = lab + al256((size_t)n * 4);
    }
};

const int32_t *h_row_ptr(const Req &r) {
    if (r.ext_rp) return r.ext_rp;
    return r.h ? (const int32_t *)(r.h) : r.v_row_ptr.data();
}
const int32_t *h_col_idx(const Req &r) {
    if (r.ext_rp) return r.ext_ci;
    return r.h ? (const int32_t *)(r.h + HostLayout(r.n, r.nnz).ci) : r.v_col_idx.data();
}
const uint32_t *h_bits(const Req &r) {
    if (r.ext_rp) return r.ext_bits;
    return r.h ? (const uint32_t *)(r.h + HostLayout(r.n, r.nnz).bits) : r.v_bits.data();
}
int32_t *h_labels(Req &r) {
    if (r.lab_h) return r.lab_h;
    return r.h ? (int32_t *)(r.h + HostLayout(r.n, r.nnz).lab) : r.v_labels.data();
}
// labels come back by an asynchronous copy into pinned memory (else retire copies them)
bool pinned_labels(const Req &r) { return r.h != nullptr || r.lab_h != nullptr; }

// Host copies between caller memory and the pinned staging arena, split
// across a few persistent threads: one thread moves about 10 GB/s, well
// below what the host memory and the host-device link sustain, and a
// request of 10^6 sites carries about 16 MB.
class CopyPool {
  public:
    explicit CopyPool(int n_threads) {
        for (int t = 0; t < n_threads; ++t) workers_.emplace_back([this] { run(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &w : workers_) w.join();
    }
    // Copies `bytes` from src to dst; returns when the copy is complete.
    void copy(void *dst, const void *src, size_t bytes) {
        const size_t parts = std::min<size_t>(workers_.size() + 1, bytes / kMinPiece);
        if (parts <= 1) { memcpy(dst, src, bytes); return; }
        const size_t piece = ((bytes + parts - 1) / parts + 63) & ~size_t(63);
        std::atomic<size_t> left{0};
        size_t queued = 0;
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (size_t off = piece; off < bytes; off += piece) {
                q_.push_back(Piece{(char *)dst + off, (const char *)src + off, std::min(piece, bytes - off), &left});
                ++queued;
            }
            left.store(queued);
        }
        cv_.notify_all();
        memcpy(dst, src, std::min(piece, bytes));     // the caller copies the first piece
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [&] { return left.load() == 0; });
    }

  private:
    struct Piece {
        char *dst;
        const char *src;
        size_t bytes;
        std::atomic<size_t> *left;
    };
    static constexpr size_t kMinPiece = 1 << 20;
    void run() {
        for (;;) {
            Piece pc;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
                if (stop_ && q_.empty()) return;
                pc = q_.front();
                q_.pop_front();
            }
            memcpy(pc.dst, pc.src, pc.bytes);
            std::lock_guard<std::mutex> lk(mu_);
            if (pc.left->fetch_sub(1) == 1) cv_done_.notify_all();
        }
    }
    std::mutex mu_;
    std::condition_variable cv_, cv_done_;
    std::deque<Piece> q_;
    std::vector<std::thread> workers_;
    bool stop_ = false;
};

// First-fit allocator over one pinned host buffer (callers hold the server mutex).
struct HostArena {
    char *base = nullptr;
    size_t cap = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    void init(char *b, size_t c) { base = b; cap = c; free_.clear(); if (c) free_[0] = c; }
    char *alloc(size_t bytes) {
        bytes = al256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[off + bytes] = sz - bytes;
            return base + off;
        }
        return nullptr;
    }
    void release(char *p, size_t bytes) {
        bytes = al256(bytes);
        size_t off = (size_t)(p - base);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) { bytes += next->second; next = free_.erase(next); }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) { prev->second += bytes; return; }
        }
        free_[off] = bytes;
    }
};


}  // namespace

struct ccl_server {
    ccl_server_config cfg{};
    int64_t budget = 0;
    // Device bytes counted against the budget: every admitted request's buffer
    // (held_req) and, until it is launched, its workspace share; plus the
    // workspace each context keeps after its largest batch (ws_slot).
    int64_t held = 0;
    int64_t held_req = 0;
    std::vector<int64_t> ws_slot;
    bool trim_ws = false;       // the uploader asks the server thread to free idle workspaces
    int64_t launches = 0;
    int64_t fail_batch = 0;     // test hook (CCL_SERVER_FAIL_BATCH): this launch fails, 0 = none
    std::vector<ccl_context *> ctxs;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    cudaStream_t upload = nullptr;                 // the first uploader's stream (teardown frees)
    std::vector<cudaStream_t> upload_streams;     // one per uploader thread
    cudaMemPool_t pool = nullptr;
    char *h_stage = nullptr;
    HostArena arena;
    std::unique_ptr<CopyPool> copier;

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_upload;
    std::deque<std::shared_ptr<Req>> pending;
    std::map<uint64_t, std::shared_ptr<Req>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    int waiters = 0;        // threads inside ccl_server_wait (destroy waits for them to leave)

    // uploads in flight (uploader thread pushes, server thread pops; under mu)
    std::deque<std::shared_ptr<Req>> uploading;
    int uploaders_running = 0;
    // owned by the server thread
    std::vector<std::shared_ptr<Req>> ready;
    std::vector<Batch> inflight;

    // statistics (under mu)
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, sites_completed = 0, arena_misses = 0;
    std::vector<double> lat_ms;
    std::vector<double> phase_ms[4];    // submit->admit, admit->ready, ready->launch, launch->done
    bool have_first = false;
    Clock::time_point t_first, t_last;

    std::thread th;
    std::vector<std::thread> uploaders;
};

namespace {

void retire(ccl_server *S, Batch &b) {
    ccl_status st = ccl_sync(S->ctxs[(size_t)b.slot], S->streams[(size_t)b.slot], 0);
    for (auto &r : b.reqs) {
        if (!pinned_labels(*r) && r->n > 0) {   // pageable request: its labels come back now
            r->v_labels.resize((size_t)r->n);
            const size_t off = HostLayout(r->n, r->nnz).lab;
            if (cudaMemcpy(r->v_labels.data(), r->d_mem + off, (size_t)r->n * 4, cudaMemcpyDeviceToHost) !=
                cudaSuccess) { (void)cudaGetLastError(); st = CCL_ERR_CUDA; }
        }
    }
    const auto now = Clock::now();
    for (auto &r : b.reqs) {
        if (r->d_mem) cudaFreeAsync(r->d_mem, S->streams[(size_t)b.slot]);
        r->d_mem = nullptr;
        if (r->uploaded) cudaEventDestroy(r->uploaded);
        r->uploaded = nullptr;
    }
    cudaEventDestroy(b.finished);
    S->slot_busy[(size_t)b.slot] = false;
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &r : b.reqs) {
        if (r->status == CCL_OK) r->status = st;    // an error from the launch stays
        r->t_done = now;
        r->done = true;
        S->held -= r->dev_bytes;
        S->held_req -= r->dev_bytes;
        S->completed++;
        S->sites_completed += r->n;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        const Clock::time_point tp[5] = {r->t_submit, r->t_admit, r->t_ready, r->t_launch, now};
        for (int k = 0; k < 4; ++k)
            S->phase_ms[k].push_back(std::chrono::duration<double, std::milli>(tp[k + 1] - tp[k]).count());
        r->v_row_ptr.clear(); r->v_row_ptr.shrink_to_fit();
        r->v_col_idx.clear(); r->v_col_idx.shrink_to_fit();
        r->v_bits.clear(); r->v_bits.shrink_to_fit();
    }
    S->t_last = now;
    S->batches++;
    S->cv_done.notify_all();
    S->cv_upload.notify_one();       // device memory was freed
}

// uploads one admitted request on stream `up`; returns false if the pool is exhausted
bool start_upload(ccl_server *S, const std::shared_ptr<Req> &r, cudaStream_t up) {
    const HostLayout lay(r->n, r->nnz);
    void *mem = nullptr;
    if (cudaMallocFromPoolAsync(&mem, lay.total, S->pool, up) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    r->d_mem = (char *)mem;
    if (r->h && !r->ext_rp) {   // one contiguous pinned block: one copy
        cudaMemcpyAsync(r->d_mem, r->h, lay.lab, cudaMemcpyHostToDevice, up);
    } else {
        cudaMemcpyAsync(r->d_mem, h_row_ptr(*r), (size_t)(r->n + 1) * 4, cudaMemcpyHostToDevice, up);
        if (r->nnz > 0) {
            cudaMemcpyAsync(r->d_mem + lay.ci, h_col_idx(*r), (size_t)r->nnz * 4, cudaMemcpyHostToDevice,
                            up);
            cudaMemcpyAsync(r->d_mem + lay.bits, h_bits(*r), (size_t)((r->nnz + 31) / 32) * 4,
                            cudaMemcpyHostToDevice, up);
        }
    }
    cudaEventCreateWithFlags(&r->uploaded, cudaEventDisableTiming);
    cudaEventRecord(r->uploaded, up);
    return true;
}

void launch_batch(ccl_server *S, int slot, std::vector<std::shared_ptr<Req>> reqs) {
    cudaStream_t s = S->streams[(size_t)slot];
    const auto t_launch = Clock::now();
    for (auto &r : reqs) r->t_launch = t_launch;
    std::vector<ccl::Inst> table;
    table.reserve(reqs.size());
    for (auto &r : reqs) {
        cudaStreamWaitEvent(s, r->uploaded, 0);
        const HostLayout lay(r->n, r->nnz);
        ccl::Inst I{};
        I.row_ptr = (const int32_t *)r->d_mem;
        I.col_idx = (const int32_t *)(r->d_mem + lay.ci);
        I.bits = (const uint32_t *)(r->d_mem + lay.bits);
        I.labels = (int32_t *)(r->d_mem + lay.lab);
        I.rp_lo = r->d_mem;
        I.rp_hi = r->d_mem + lay.total;     // one allocation holds all four arrays
        I.ci_lo = I.rp_lo;
        I.ci_hi = I.rp_hi;
        I.bits_lo = I.rp_lo;
        I.bits_hi = I.rp_hi;
        I.bit_off = 0;
        I.n = r->n;
        I.nnz = (int32_t)r->nnz;
        table.push_back(I);
    }
    ccl_context *ctx = S->ctxs[(size_t)slot];
    const int64_t ws_before = ccl::workspace_bytes(ctx);
    ccl_status st = CCL_OK;
    if (S->fail_batch > 0 && ++S->launches == S->fail_batch) {
        st = CCL_ERR_OUT_OF_MEMORY;     // test hook: as if the workspace could not be allocated
    } else {
        st = ccl::label_instances(ctx, table, s);
        if (st == CCL_ERR_OUT_OF_MEMORY) {
            // the pool may keep freed request buffers that the workspace's
            // cudaMalloc cannot use: hand them back and try once more
            cudaMemPoolTrimTo(S->pool, 0);
            (void)cudaGetLastError();
            st = ccl::label_instances(ctx, table, s);
        }
    }
    {
        // the batch's workspace shares are released; the context now keeps
        // ws_after bytes of workspace (at most the shares it was granted)
        const int64_t ws_after = ccl::workspace_bytes(ctx);
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &r : reqs) { S->held -= r->ws_bytes; r->ws_bytes = 0; }
        S->held += ws_after - ws_before;
        S->ws_slot[(size_t)slot] = ws_after;
    }
    for (size_t t = 0; t < reqs.size(); ++t) {
        auto &r = reqs[t];
        if (pinned_labels(*r) && r->n > 0)
            cudaMemcpyAsync(h_labels(*r), table[t].labels, (size_t)r->n * 4, cudaMemcpyDeviceToHost, s);
        if (st != CCL_OK) r->status = st;
    }
    Batch b;
    b.reqs = std::move(reqs);
    b.slot = slot;
    cudaEventCreateWithFlags(&b.finished, cudaEventDisableTiming);
    cudaEventRecord(b.finished, s);
    S->slot_busy[(size_t)slot] = true;
    S->inflight.push_back(std::move(b));
}

void server_loop(ccl_server *S) {
    cudaSetDevice(S->cfg.device);
    for (;;) {
        bool progressed = false;
        // 1. collect every request whose upload has finished, in any order (a
        //    large upload still in flight does not hold back the small ones
        //    behind it; admission and uploads run on the uploader threads)
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stop) break;
            for (auto it = S->uploading.begin(); it != S->uploading.end();) {
                auto &r = *it;
                const cudaError_t e = cudaEventQuery(r->uploaded);
                if (e == cudaErrorNotReady) { ++it; continue; }
                if (e != cudaSuccess) { (void)cudaGetLastError(); r->status = CCL_ERR_CUDA; }
                r->t_ready = Clock::now();
                S->ready.push_back(r);
                it = S->uploading.erase(it);
                progressed = true;
            }
        }
        // 2. free the workspace idle contexts keep, when it blocks admission
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->trim_ws) {
                S->trim_ws = false;
                for (size_t slot = 0; slot < S->ctxs.size(); ++slot) {
                    if (S->slot_busy[slot] || S->ws_slot[slot] == 0) continue;
                    const int64_t ws = S->ws_slot[slot];
                    lk.unlock();
                    ccl::release_workspace(S->ctxs[slot]);
                    lk.lock();
                    S->held -= ws;
                    S->ws_slot[slot] = 0;
                }
                S->cv_upload.notify_all();
                progressed = true;
            }
        }
        // 3. launch on a free compute stream
        if (!S->ready.empty()) {
            for (size_t slot = 0; slot < S->streams.size() && !S->ready.empty(); ++slot) {
                if (S->slot_busy[slot]) continue;
                const size_t take = std::min<size_t>(S->ready.size(), (size_t)S->cfg.max_batch);
                std::vector<std::shared_ptr<Req>> reqs(S->ready.begin(), S->ready.begin() + (long)take);
                S->ready.erase(S->ready.begin(), S->ready.begin() + (long)take);
                launch_batch(S, (int)slot, std::move(reqs));
                progressed = true;
            }
        }
        // 4. retire finished batches
        for (size_t b = 0; b < S->inflight.size();) {
            const cudaError_t e = cudaEventQuery(S->inflight[b].finished);
            if (e == cudaErrorNotReady) { ++b; continue; }
            if (e != cudaSuccess) (void)cudaGetLastError();
            retire(S, S->inflight[b]);
            S->inflight.erase(S->inflight.begin() + (long)b);
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            const bool idle = S->pending.empty() && S->uploading.empty() && S->ready.empty() &&
                              S->inflight.empty();
            S->cv_work.wait_for(lk, idle ? std::chrono::milliseconds(5) : std::chrono::microseconds(50));
        }
    }
    // drain what is on the device before tearing down (after the uploader has stopped)
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_upload.notify_all();
        S->cv_done.wait(lk, [&] { return S->uploaders_running == 0; });
    }
    for (auto &b : S->inflight) {
        cudaEventSynchronize(b.finished);
        retire(S, b);
    }
    S->inflight.clear();
    for (auto &r : S->uploading) {
        cudaEventSynchronize(r->uploaded);
        if (r->d_mem) cudaFreeAsync(r->d_mem, S->upload);
        cudaEventDestroy(r->uploaded);
    }
    for (auto &r : S->ready) {
        if (r->d_mem) cudaFreeAsync(r->d_mem, S->upload);
        if (r->uploaded) cudaEventDestroy(r->uploaded);
    }
    for (auto us : S->upload_streams) cudaStreamSynchronize(us);
}

// Admits pending requests while their device bytes fit the budget and uploads
// them on the upload stream. Copies from pageable memory block the calling
// thread while the driver stages them, so they run here, apart from the
// launch/retire loop.
void upload_loop(ccl_server *S, cudaStream_t up) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (S->pending.empty()) {
            S->cv_upload.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        auto r = S->pending.front();
        if (S->held + r->dev_bytes + r->ws_bytes > S->budget && S->held > 0) {
            // wait for memory to free up; if only the workspace kept by idle
            // contexts stands in the way, ask the server thread to free it
            if (S->held_req == 0) { S->trim_ws = true; S->cv_work.notify_one(); }
            S->cv_upload.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        S->pending.pop_front();
        S->held += r->dev_bytes + r->ws_bytes;
        S->held_req += r->dev_bytes;
        r->t_admit = Clock::now();
        lk.unlock();
        const bool ok = start_upload(S, r, up);
        lk.lock();
        if (!ok) {
            // the pool cannot allocate right now (other work holds the
            // memory): retry later; once the server holds nothing for other
            // requests and this has lasted kAllocGiveUp, the request fails
            S->held -= r->dev_bytes + r->ws_bytes;
            S->held_req -= r->dev_bytes;
            const auto now = Clock::now();
            if (!r->alloc_failing) { r->alloc_failing = true; r->t_alloc_fail = now; }
            const bool alone = S->held_req == 0;
            if (alone && now - r->t_alloc_fail > kAllocGiveUp) {
                r->status = CCL_ERR_OUT_OF_MEMORY;
                r->t_done = now;
                r->done = true;
                S->completed++;
                S->cv_done.notify_all();
                continue;
            }
            if (alone) { S->trim_ws = true; S->cv_work.notify_one(); }
            S->pending.push_front(r);
            S->cv_upload.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        r->alloc_failing = false;
        S->uploading.push_back(r);
        S->cv_work.notify_one();
    }
    S->uploaders_running--;
    S->cv_done.notify_all();
}

}  // namespace

extern "C" {

ccl_status ccl_server_create(ccl_server **out, const ccl_server_config *cfg_in) {
    if (!out) return CCL_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    ccl_server_config cfg{};
    cfg.device = 0;
    cfg.n_streams = 2;
    cfg.hbm_reserve = (int64_t)2 << 30;
    cfg.hbm_budget = 0;
    cfg.max_batch = 1024;
    cfg.max_pending = 1 << 20;
    cfg.host_staging_bytes = (int64_t)1 << 30;
    if (cfg_in) {
        if (cfg_in->host_staging_bytes != 0) cfg.host_staging_bytes = std::max<int64_t>(0, cfg_in->host_staging_bytes);
        cfg.device = cfg_in->device;
        if (cfg_in->n_streams > 0) cfg.n_streams = cfg_in->n_streams;
        if (cfg_in->hbm_reserve > 0) cfg.hbm_reserve = cfg_in->hbm_reserve;
        if (cfg_in->hbm_budget > 0) cfg.hbm_budget = cfg_in->hbm_budget;
        if (cfg_in->max_batch > 0) cfg.max_batch = cfg_in->max_batch;
        if (cfg_in->max_pending > 0) cfg.max_pending = cfg_in->max_pending;
    }
    if (cfg.n_streams > 16) return CCL_ERR_INVALID_ARGUMENT;
    if (cudaSetDevice(cfg.device) != cudaSuccess) { (void)cudaGetLastError(); return CCL_ERR_INVALID_ARGUMENT; }
    auto S = new ccl_server();
    S->cfg = cfg;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { (void)cudaGetLastError(); delete S; return CCL_ERR_CUDA; }
    S->budget = (int64_t)free_b - cfg.hbm_reserve;
    if (cfg.hbm_budget > 0) S->budget = std::min(S->budget, cfg.hbm_budget);
    if (S->budget <= 0) { delete S; return CCL_ERR_OUT_OF_MEMORY; }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = cfg.device;
    e = cudaMemPoolCreate(&S->pool, &props);
    if (e == cudaSuccess) {
        uint64_t thr = UINT64_MAX;   // keep freed memory in the pool
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    for (int u = 0; u < kUploaders && e == cudaSuccess; ++u) {
        cudaStream_t us = nullptr;
        e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->upload_streams.push_back(us);
    }
    if (e == cudaSuccess) S->upload = S->upload_streams[0];
    if (e == cudaSuccess && cfg.host_staging_bytes > 0) {
        e = cudaMallocHost(&S->h_stage, (size_t)cfg.host_staging_bytes);
        if (e == cudaSuccess) S->arena.init(S->h_stage, (size_t)cfg.host_staging_bytes);
    }
    for (int i = 0; i < cfg.n_streams && e == cudaSuccess; ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        S->streams.push_back(s);
        ccl_context *c = nullptr;
        if (ccl_context_create(&c, cfg.device) != CCL_OK) { e = cudaErrorUnknown; break; }
        ccl_set_option(c, CCL_OPT_USE_GRAPHS, 0);
        // batches of varying size: grow the workspace twofold, so it is
        // reallocated (a device-wide synchronisation) a few times, not at
        // every new largest batch
        ccl::set_workspace_growth(c, 2.0);
        S->ctxs.push_back(c);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        for (auto c : S->ctxs) ccl_context_destroy(c);
        for (auto s : S->streams) cudaStreamDestroy(s);
        for (auto us : S->upload_streams) cudaStreamDestroy(us);
        if (S->pool) cudaMemPoolDestroy(S->pool);
        if (S->h_stage) cudaFreeHost(S->h_stage);
        delete S;
        return CCL_ERR_CUDA;
    }
    S->slot_busy.assign(S->streams.size(), false);
    S->ws_slot.assign(S->streams.size(), 0);
    // test hook: CCL_SERVER_FAIL_BATCH=k makes the k-th batch launch report
    // CCL_ERR_OUT_OF_MEMORY without running, as a failed workspace allocation would
    if (const char *env = getenv("CCL_SERVER_FAIL_BATCH")) S->fail_batch = std::max(0, atoi(env));
    {
        // copy threads: CCL_SERVER_COPY_THREADS, else three quarters of the host's cores, at most 12
        const unsigned hw = std::max(2u, std::thread::hardware_concurrency());
        int nt = (int)std::min(12u, hw * 3 / 4);
        if (const char *env = getenv("CCL_SERVER_COPY_THREADS")) nt = std::max(0, std::min(64, atoi(env)));
        S->copier.reset(new CopyPool(nt));
    }
    S->uploaders_running = (int)S->upload_streams.size();
    S->th = std::thread(server_loop, S);
    for (auto us : S->upload_streams) S->uploaders.emplace_back(upload_loop, S, us);
    *out = S;
    return CCL_OK;
}

}  // extern "C"

namespace {
ccl_status server_submit(ccl_server *S, const ccl_request *req, uint64_t *ticket, bool copy) {
    if (!S || !req || !ticket) return CCL_ERR_INVALID_ARGUMENT;
    if (req->n_sites < 0 || req->n_sites > CCL_MAX_SITES || req->nnz < 0 || req->nnz > INT32_MAX)
        return CCL_ERR_INVALID_ARGUMENT;
    if (!req->row_ptr || (req->nnz > 0 && (!req->col_idx || !req->open_bits)))
        return CCL_ERR_INVALID_ARGUMENT;
    auto r = std::make_shared<Req>();
    r->n = req->n_sites;
    r->nnz = req->nnz;
    // device bytes: inputs + labels + the request's share of the labelling
    // workspace of a batched launch (a residual-pair slot of 8 B and its
    // instance id of 4 B per CSR entry)
    const HostLayout lay(r->n, r->nnz);
    r->dev_bytes = (int64_t)lay.total;
    r->ws_bytes = 12 * r->nnz;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (r->dev_bytes + r->ws_bytes > S->budget || (int64_t)S->pending.size() >= S->cfg.max_pending) {
            S->rejected++;
            return CCL_ERR_REJECTED;
        }
    }
    r->t_submit = Clock::now();
    if (!copy) {
        r->ext_rp = req->row_ptr;
        r->ext_ci = req->nnz > 0 ? req->col_idx : req->row_ptr;
        r->ext_bits = req->nnz > 0 ? req->open_bits : (const uint32_t *)req->row_ptr;
        std::lock_guard<std::mutex> lk(S->mu);
        r->lab_h = (int32_t *)S->arena.alloc((size_t)r->n * 4 + 4);
        if (r->lab_h) r->lab_bytes = (size_t)r->n * 4 + 4;
        else S->arena_misses++;
    } else {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->h = S->arena.alloc(lay.total);
            if (r->h) r->h_bytes = lay.total;
            else S->arena_misses++;
        }
        if (r->h) {
            S->copier->copy(r->h, req->row_ptr, (size_t)(r->n + 1) * 4);
            if (r->nnz > 0) {
                S->copier->copy(r->h + lay.ci, req->col_idx, (size_t)r->nnz * 4);
                S->copier->copy(r->h + lay.bits, req->open_bits, (size_t)((r->nnz + 31) / 32) * 4);
            }
        } else {
            r->v_row_ptr.assign(req->row_ptr, req->row_ptr + r->n + 1);
            r->v_col_idx.assign(req->col_idx, req->col_idx + r->nnz);
            r->v_bits.assign(req->open_bits, req->open_bits + (r->nnz + 31) / 32);
            if (r->v_bits.empty()) r->v_bits.push_back(0);
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        S->tickets[r->ticket] = r;
        S->pending.push_back(r);
        S->submitted++;
        if (!S->have_first) { S->have_first = true; S->t_first = r->t_submit; }
        *ticket = r->ticket;
    }
    S->cv_upload.notify_one();
    return CCL_OK;
}
}  // namespace

extern "C" {

ccl_status ccl_server_submit(ccl_server *S, const ccl_request *req, uint64_t *ticket) {
    return server_submit(S, req, ticket, true);
}

ccl_status ccl_server_submit_nocopy(ccl_server *S, const ccl_request *req, uint64_t *ticket) {
    return server_submit(S, req, ticket, false);
}

ccl_status ccl_server_wait(ccl_server *S, uint64_t ticket, int32_t *labels_host, int64_t timeout_ms) {
    if (!S) return CCL_ERR_INVALID_ARGUMENT;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return CCL_ERR_NOT_FOUND;
    auto r = it->second;
    // counted while inside, so that ccl_server_destroy frees nothing under a waiter
    ++S->waiters;
    struct Leave {
        ccl_server *S;
        std::unique_lock<std::mutex> &lk;
        ~Leave() {
            if (!lk.owns_lock()) lk.lock();
            if (--S->waiters == 0) S->cv_done.notify_all();
        }
    } leave{S, lk};
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return CCL_ERR_TIMEOUT;
    if (r->dropped) {
        S->tickets.erase(ticket);
        return r->status;
    }
    if (labels_host && r->n > 0) {
        // copy outside the lock: the request is done and only this waiter owns it now
        S->tickets.erase(ticket);
        lk.unlock();
        S->copier->copy(labels_host, h_labels(*r), (size_t)r->n * 4);
        lk.lock();
    } else {
        S->tickets.erase(ticket);
    }
    if (r->h) { S->arena.release(r->h, r->h_bytes); r->h = nullptr; }
    if (r->lab_h) { S->arena.release((char *)r->lab_h, r->lab_bytes); r->lab_h = nullptr; }
    r->v_labels.clear();
    r->v_labels.shrink_to_fit();
    return r->status;
}

ccl_status ccl_server_stats_get(ccl_server *S, ccl_server_stats *out) {
    if (!S || !out) return CCL_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->batches = S->batches;
    out->sites_completed = S->sites_completed;
    out->waiting = S->waiters;
    out->arena_misses = S->arena_misses;
    for (int k = 0; k < 4; ++k) {
        if (S->phase_ms[k].empty()) continue;
        std::vector<double> v = S->phase_ms[k];
        std::sort(v.begin(), v.end());
        out->phase_p50_ms[k] = v[std::min(v.size() - 1, (size_t)(0.5 * (double)(v.size() - 1) + 0.5))];
        out->phase_p99_ms[k] = v[std::min(v.size() - 1, (size_t)(0.99 * (double)(v.size() - 1) + 0.5))];
    }
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    if (S->have_first && S->completed > 0) {
        out->busy_seconds = std::chrono::duration<double>(S->t_last - S->t_first).count();
        if (out->busy_seconds > 0) out->sites_per_second = (double)S->sites_completed / out->busy_seconds;
    }
    return CCL_OK;
}

void ccl_server_destroy(ccl_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_upload.notify_all();
    for (auto &u : S->uploaders)
        if (u.joinable()) u.join();
    if (S->th.joinable()) S->th.join();
    {
        // requests that were never labelled end as CCL_ERR_REJECTED; waiters
        // blocked on them return, and every waiter leaves before anything is freed
        std::unique_lock<std::mutex> lk(S->mu);
        for (auto &kv : S->tickets) {
            Req &r = *kv.second;
            if (r.done) continue;
            r.dropped = true;
            r.status = CCL_ERR_REJECTED;
            r.done = true;
        }
        S->cv_done.notify_all();
        S->cv_done.wait(lk, [&] { return S->waiters == 0; });
    }
    S->copier.reset();
    cudaSetDevice(S->cfg.device);
    for (auto c : S->ctxs) ccl_context_destroy(c);
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto us : S->upload_streams) cudaStreamDestroy(us);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->h_stage) cudaFreeHost(S->h_stage);
    (void)cudaGetLastError();
    delete S;
}

}  // extern "C"
