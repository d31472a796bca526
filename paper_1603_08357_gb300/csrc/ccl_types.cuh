// Data layout shared by the labelling kernels and the host code: the
// per-instance descriptor, the per-chunk record and the kernel parameters.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kChunk = 32;                 // sites per chunk (one warp)
constexpr int kStageEntries = 256;         // CSR entries a warp can stage (8 per site)
constexpr int kStageWords = kStageEntries / 32 + 2;
constexpr unsigned kFull = 0xffffffffu;

// latched device error bits
constexpr unsigned kErrIndex = 1u;         // col_idx or row_ptr out of range
constexpr unsigned kErrNonconv = 2u;       // iteration cap hit
constexpr unsigned kErrShape = 4u;         // row_ptr[0] != 0 or row_ptr[n] != nnz
constexpr unsigned kErrAsym = 8u;          // validate: missing mirror entry

// One instance as the kernels see it.
struct Inst {
    const int32_t *row_ptr;    // n+1 local entry numbers
    const int32_t *col_idx;    // local entry -> local site
    const uint32_t *bits;      // bit words; local entry e is bit bit_off + e
    int32_t *labels;           // n outputs
    int64_t bit_off;
    int64_t q_off;             // queue slot of local entry 0
    int64_t chunk_begin;       // first global chunk of the instance
    int32_t n;
    int32_t nnz;
};

// Per-chunk record written by step (i) and read by step (iii).
struct __align__(16) ChunkRec {
    int64_t qbeg;              // first queue slot of the chunk's pairs
    int32_t cnt;               // residual pairs of the chunk
    int32_t inst;              // instance of the chunk
};

struct Params {
    const Inst *insts;         // device table, K entries (K > 1)
    Inst one;                  // the instance when K == 1
    int32_t K;
    int32_t dedup;
    int64_t n_chunks;          // over all instances
    ChunkRec *rec;             // [n_chunks]
    int2 *q;                   // residual pairs (i, j), slots indexed by global entry
    unsigned *err;
    unsigned long long *counters;   // [0] residual pairs
};

}  // namespace ccl
