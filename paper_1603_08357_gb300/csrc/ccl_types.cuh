// Data layout shared by the labelling kernels and the host code: the
// per-instance descriptor, the per-chunk record and the kernel parameters.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kChunk = 32;                 // sites per chunk (one warp's worth)
constexpr unsigned kFull = 0xffffffffu;

// step (i): one CTA = kInitConsumers consumer warps + 1 producer warp; the
// producer streams tiles of kTileSites sites through kStages shared-memory
// stages with bulk asynchronous copies
constexpr int kTileSites = 1024;
constexpr int kInitConsumers = 16;
constexpr int kInitThreads = 32 * (kInitConsumers + 1);
constexpr int kChunksPerConsumer = kTileSites / kChunk / kInitConsumers;
constexpr int kStages = 3;
constexpr int kColCap = 7168;              // column entries a stage holds (7 per site)
constexpr int kRpBuf = kTileSites + 8;     // row pointers of a tile, + 16-byte rounding
constexpr int kColBuf = kColCap + 8;
constexpr int kBitBuf = kColCap / 32 + 12;
constexpr int kRowRegs = 8;                // rows up to this degree are scanned in registers

// steps (ii)/(iv): chunks a warp walks at once
#ifndef CCL_ANA_CHUNKS
#define CCL_ANA_CHUNKS 2
#endif
constexpr int kAnaChunks = CCL_ANA_CHUNKS;
#ifndef CCL_ANA_CHUNKS_BATCHED
#define CCL_ANA_CHUNKS_BATCHED 4
#endif
constexpr int kAnaChunksBatched = CCL_ANA_CHUNKS_BATCHED;

// step (iii): pairs a lane carries at once; pairs a warp drains per window;
// most step-(i) CTAs (bands)
#ifndef CCL_RED_SLOTS
#define CCL_RED_SLOTS 6
#endif
constexpr int kRedSlots = CCL_RED_SLOTS;
constexpr int kRedWindowMax = 2048;   // default most pairs per warp window (fewer for small queues)
constexpr int kMaxBands = 1024;

// latched device error bits
constexpr unsigned kErrIndex = 1u;         // col_idx or row_ptr out of range
constexpr unsigned kErrNonconv = 2u;       // iteration cap hit, or a bounded wait expired
constexpr unsigned kErrShape = 4u;         // row_ptr[0] != 0 or row_ptr[n] != nnz
constexpr unsigned kErrAsym = 8u;          // validate: missing mirror entry

// One instance as the kernels see it.
struct Inst {
    const int32_t *row_ptr;    // n+1 local entry numbers
    const int32_t *col_idx;    // local entry -> local site
    const uint32_t *bits;      // bit words; local entry e is bit bit_off + e
    int32_t *labels;           // n outputs
    // readable memory around each input array: bulk copies round their
    // ranges outward to 16 bytes but never leave [lo, hi)
    const void *rp_lo, *rp_hi, *ci_lo, *ci_hi, *bits_lo, *bits_hi;
    int64_t bit_off;
    int64_t q_off;             // queue slot of local entry 0
    int64_t chunk_begin;       // first global chunk of the instance
    int64_t tile_begin;        // first global tile of the instance
    int32_t n;
    int32_t nnz;
};

// Residual pairs of one step-(i) CTA: they are packed from queue slot qbase
// on (inside the slot range of the band's CSR entries, so bands never overlap).
struct __align__(16) BandRec {
    int64_t qbase;
    unsigned long long cnt;
};

struct Params {
    const Inst *insts;         // device table, K entries (K > 1)
    Inst one;                  // the instance when K == 1
    int32_t K;
    int32_t link_mode;         // step (iii): 0 root to root, 1 root to the other chain's node
    int64_t n_chunks;          // over all instances
    int64_t n_tiles;           // over all instances
    int32_t n_bands;           // CTAs of step (i)
    int32_t dense;             // 1: step (i) reads the dense neighbour list nn
    BandRec *band;             // [n_bands]
    int2 *q;                   // residual pairs (i, j); slots indexed by global CSR entry
    int32_t *qk;               // instance of each pair (K > 1 only)
    int64_t q_cap;             // slots of q (and qk)
    uint64_t gen_seed;         // bonds drawn on the device: SplitMix64 state ...
    uint64_t gen_thr;          // ... and threshold (bond open iff output >> 11 < gen_thr)
    const int32_t *nn;         // dense neighbour list (slot k of site i at nn[i + k*n]), or null
    int64_t nn_width;          // slots per site of the dense list
    int64_t tile_off;          // step (i) on part of the tiles: its first tile ...
    int32_t band_off;          // ... and its first band record
    int32_t iter_cap;          // > 0: steps (ii)-(iv) give up after this many iterations (test option)
    int32_t red_window;        // step (iii): most pairs per warp window (0: kRedWindowMax)
    int32_t ana_group;         // steps (ii)/(iv), contiguous order: > 0 visit the sites in super-chunks
                               // (every warp takes its next ana_group chunk groups of each), 0 one range per warp
    unsigned *err;
    unsigned long long *counters;   // [0] residual pairs
};

// Shared-memory stage of step (i).
struct __align__(16) StageHdr {
    int64_t w_lo, w_hi;        // bit words present: [w_lo, w_hi) relative to Inst::bits
    int32_t k, s0, ts, e0, e1; // instance, first site, sites, entry range of the tile
    int32_t rp_lo, rp_hi;      // row pointers present (indices relative to Inst::row_ptr)
    int32_t ci_lo, ci_hi;      // column entries present (relative to Inst::col_idx)
    int32_t status;            // 0 valid, 1 corrupt row pointers
    int32_t pad_;
    int64_t qband;             // first queue slot of this CTA's band
    // the fields of the tile's instance the consumers use (batched calls read
    // them here instead of from the instance table in global memory)
    const int32_t *i_rp, *i_ci;
    const uint32_t *i_bits;
    int32_t *i_lab;
    int64_t i_bit_off, i_tile_begin;
    int32_t i_n, i_nnz;
    // per-tile values every consumer warp needs, computed once by the producer:
    // stage-relative bit index of local entry 0, bits present, whether the
    // stage holds the tile's whole entry range, and the instance-local tiles
    // [vis_lo, vis_hi] of the band whose labels are final and visible
    int32_t t_rb0, t_nbits, t_staged, t_vis_lo, t_vis_hi, pad2_;
};

// the consumers load {k, s0, ts, e0}, {e1, rp_lo, rp_hi, ci_lo} and {t_rb0,
// t_nbits, t_staged, t_vis_lo} as one 16-byte word each
static_assert(offsetof(StageHdr, k) % 16 == 0 && offsetof(StageHdr, s0) == offsetof(StageHdr, k) + 4 &&
                  offsetof(StageHdr, ts) == offsetof(StageHdr, k) + 8 &&
                  offsetof(StageHdr, e0) == offsetof(StageHdr, k) + 12 &&
                  offsetof(StageHdr, e1) == offsetof(StageHdr, k) + 16 &&
                  offsetof(StageHdr, rp_lo) == offsetof(StageHdr, k) + 20 &&
                  offsetof(StageHdr, rp_hi) == offsetof(StageHdr, k) + 24 &&
                  offsetof(StageHdr, ci_lo) == offsetof(StageHdr, k) + 28,
              "stage header words read as int4");
static_assert(offsetof(StageHdr, t_rb0) % 16 == 0 && offsetof(StageHdr, t_nbits) == offsetof(StageHdr, t_rb0) + 4 &&
                  offsetof(StageHdr, t_staged) == offsetof(StageHdr, t_rb0) + 8 &&
                  offsetof(StageHdr, t_vis_lo) == offsetof(StageHdr, t_rb0) + 12,
              "stage header tile words read as int4");

struct __align__(16) Stage {
    StageHdr h;
    int32_t rp[kRpBuf];
    int32_t ci[kColBuf];
    uint32_t bw[kBitBuf];
};

constexpr size_t kInitSmem = 64 + sizeof(Stage) * kStages;

}  // namespace ccl
