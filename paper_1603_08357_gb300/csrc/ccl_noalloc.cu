// ccl_label_noalloc: the single-instance labelling of ccl_label for callers
// that cannot allocate device memory at run time.
//
// Some host programs must not call cudaMalloc once they are running: a
// latency-bound loop cannot afford the device-wide synchronisation that
// cudaMalloc and cudaFree may cause, and a process whose device memory is
// already handed out by another allocator (a framework's caching pool, a fixed
// arena) may have nothing left for a library to take. This entry point uses
// no context and allocates nothing. The few bytes of working memory the
// labelling needs (the latched error word, counters, per-CTA pair records) and
// the residual-pair queue live in one file-scope device array of fixed size,
// which every GPU that loads this library holds until the process exits.
//
// The array's name is not a device address on the host: its address is taken
// with cudaGetSymbolAddress once per device, on that device's first call.
#include <ccl.h>

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#define CCL_NO_VALIDATE_KERNEL
#include "ccl_device.cuh"

using namespace ccl;

namespace {

constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 21;   // CSR entries (residual-pair slots)
constexpr size_t kOffErr = 0;                               // unsigned error word
constexpr size_t kOffCounters = 256;                        // 4 x u64 counters
constexpr size_t kOffBand = 512;                            // kMaxBands BandRec
constexpr size_t kOffQueue = kOffBand + sizeof(BandRec) * kMaxBands;
constexpr size_t kScratchBytes = kOffQueue + sizeof(int2) * (size_t)kNoAllocMaxEntries;

static_assert(kOffQueue % 256 == 0, "queue must stay 256-byte aligned");

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of the array
    int num_sms = 0;
    int init_per_sm = 1, ana_per_sm = 1, red_per_sm = 1;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Per-device set-up on the device's first call, with that device current:
// the scratch address, the SM count, the kernels' occupancy and the opt-in
// shared memory of step (i). None of it allocates.
ccl_status setup_device(int dev, DeviceSetup **out) {
    if (dev < 0 || dev >= kMaxDevices) return CCL_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_init<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInitSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.init_per_sm, k_init<false>, kInitThreads, kInitSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.ana_per_sm, k_analysis<false, true>, 256, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.red_per_sm, k_reduce<false, true>, 256, 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? CCL_ERR_OUT_OF_MEMORY : CCL_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char *>(ptr);
        d.init_per_sm = std::max(d.init_per_sm, 1);
        d.ana_per_sm = std::max(d.ana_per_sm, 1);
        d.red_per_sm = std::max(d.red_per_sm, 1);
        d.ready = true;
    }
    *out = &d;
    return CCL_OK;
}

}  // namespace

extern "C" ccl_status ccl_label_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                        const int32_t *col_idx, const uint32_t *bits, int32_t *labels,
                                        void *stream) {
    if (n < 0 || n > CCL_MAX_SITES || nnz < 0) return CCL_ERR_INVALID_ARGUMENT;
    if (nnz > kNoAllocMaxEntries) return CCL_ERR_INVALID_ARGUMENT;   // beyond the fixed scratch
    if (n == 0) return CCL_OK;
    if (!row_ptr || !labels || (nnz > 0 && (!col_idx || !bits))) return CCL_ERR_INVALID_ARGUMENT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return CCL_ERR_CUDA; }
    DeviceSetup *d = nullptr;
    ccl_status st = setup_device(dev, &d);
    if (st != CCL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    Params P;
    memset(&P, 0, sizeof(P));
    P.K = 1;
    P.link_mode = 0;
    P.n_chunks = ((int64_t)n + kChunk - 1) / kChunk;
    P.n_tiles = ((int64_t)n + kTileSites - 1) / kTileSites;
    P.err = reinterpret_cast<unsigned *>(d->scratch + kOffErr);
    P.counters = reinterpret_cast<unsigned long long *>(d->scratch + kOffCounters);
    P.band = reinterpret_cast<BandRec *>(d->scratch + kOffBand);
    P.q = reinterpret_cast<int2 *>(d->scratch + kOffQueue);
    P.qk = nullptr;
    P.q_cap = kNoAllocMaxEntries;
    Inst &I = P.one;
    I.row_ptr = row_ptr;
    I.col_idx = col_idx;
    I.bits = bits;
    I.labels = labels;
    I.rp_lo = row_ptr;
    I.rp_hi = row_ptr + (int64_t)n + 1;
    I.ci_lo = col_idx;
    I.ci_hi = col_idx ? col_idx + nnz : col_idx;
    I.bits_lo = bits;
    I.bits_hi = bits ? bits + (nnz + 31) / 32 : bits;
    I.bit_off = 0;
    I.q_off = 0;
    I.chunk_begin = 0;
    I.tile_begin = 0;
    I.n = n;
    I.nnz = (int32_t)nnz;

    // step (i) bands: one CTA per non-empty band (as in ccl_label)
    int64_t g = std::min<int64_t>((int64_t)d->num_sms * d->init_per_sm, std::min<int64_t>(P.n_tiles, kMaxBands));
    g = std::max<int64_t>(g, 1);
    const int64_t per = (P.n_tiles + g - 1) / g;
    const int64_t g_init = (P.n_tiles + per - 1) / per;
    P.n_bands = (int32_t)g_init;
    const int64_t ana_warps = (P.n_chunks + kAnaChunks - 1) / kAnaChunks;
    const int64_t g_ana = std::max<int64_t>(1, std::min<int64_t>((int64_t)d->num_sms * d->ana_per_sm, (ana_warps + 7) / 8));
    const int64_t g_red = (int64_t)d->num_sms * d->red_per_sm;

    // the array keeps the previous call's contents: clear the error word, the
    // counters and the band records that must start at zero
    cudaError_t e = cudaMemsetAsync(d->scratch, 0, kOffBand + sizeof(BandRec) * (size_t)g_init, s);
    if (e == cudaSuccess) {
        k_init<false><<<(unsigned)g_init, kInitThreads, kInitSmem, s>>>(P);
        k_analysis<false, true><<<(unsigned)g_ana, 256, 0, s>>>(P);
        k_reduce<false, true><<<(unsigned)g_red, 256, 0, s>>>(P);
        k_analysis<false, true><<<(unsigned)g_ana, 256, 0, s>>>(P);
        e = cudaGetLastError();
    }
    // the error word comes back on the call's own stream (no wait on other
    // streams of the device), then the call waits for that stream
    unsigned err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err, d->scratch + kOffErr, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return CCL_ERR_CUDA;
    }
    if (err & kErrIndex) return CCL_ERR_INDEX_OUT_OF_RANGE;
    if (err & kErrShape) return CCL_ERR_INVALID_ARGUMENT;
    if (err & kErrNonconv) return CCL_ERR_NONCONVERGED;
    return CCL_OK;
}
