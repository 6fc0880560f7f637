// Library-internal definitions of the opaque C ABI handles, shared by the
// translation units that implement entry points.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace fastid {
// One NVTX range per C-ABI call, named after the entry point, so that a
// profiler or tracer attributes every kernel to the call that launched it
// (e.g. ncu --nvtx --nvtx-include "fastid_topk/").  Without a tool attached
// the push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace fastid
#define FASTID_RANGE() ::fastid::NvtxRange fastid_nvtx_range_(__func__)

struct fastid_ctx {
    int device = 0;
    int form = FASTID_FORM_AUTO;
    int sms = 0;
    cudaMemPool_t pool = nullptr;
    uint32_t *dev_status = nullptr;  // [8]: the live word [0..3], a snapshot [4..7] (fastid_sync_status)
    int grid_topk = 0, grid_hits = 0, grid_scores = 0, grid_tensor = 0;
    int pair_clusters = 0;  // resident 2-CTA clusters of the paired tensor kernel (0: never pair)
    std::string last_error;
    // profiling (fastid_profile)
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t events_used = 0;
    int64_t launches = 0;
    int64_t pool_allocs = 0;  // stream-ordered scratch allocations from `pool` (fastid_memory_info)
};

struct fastid_refdb {
    int64_t n_refs = 0;
    int64_t n_pad = 0;
    int32_t n_loci = 0;
    int32_t n_words64 = 0;
    int64_t ld64 = 0;
    uint32_t flags = 0;
    uint64_t *packed = nullptr;  // [n_pad][ld64]
    uint32_t *norms = nullptr;   // [n_pad]
    uint8_t *fp8 = nullptr;      // [n_pad][kpad] e4m3 0/1 operand (FASTID_REFS_TENSOR)
    int32_t kpad = 0;            // loci padded to the tensor form's K stage
    uint8_t *fp4 = nullptr;      // [n_pad][kbytes4] e2m1 0/1 operand (FASTID_REFS_FP4)
    int32_t kbytes4 = 0;         // its row bytes: loci padded to 256, two per byte
    CUtensorMap map_b;           // TMA map over fp8 (boxes of K-stage x reference tile)
    CUtensorMap map_b_half;      // same, boxes of half a reference tile (paired launches)
    CUtensorMap map_p;           // TMA map over packed (boxes of 2 words x 256 refs, packed-operand launches)
    CUtensorMap map_b4;          // TMA map over fp4 (boxes of 128 bytes x 224 refs)
    CUtensorMap map_b4_half;     // same, boxes of 112 refs (paired FP4 launches)
    CUtensorMap map_p4;          // TMA map over packed (boxes of 4 words x 224 refs, packed FP4 launches)
    int64_t bytes = 0;
    int device = 0;
    bool view = false;           // fastid_refs_view: rows of another database, memory not owned
};

namespace fastid {
// Operand of a comparison call.
enum Operand : int {
    OP_PLAIN = 0,       // plain form (packed words, AND + POPC)
    OP_FP8 = 1,         // tensor form over the database's FP8 copy
    OP_FP8_PACKED = 2,  // tensor form over the packed rows, expanded to FP8 on chip
    OP_FP4 = 3,         // tensor form over the database's FP4 copy
    OP_FP4_PACKED = 4,  // tensor form over the packed rows, expanded to FP4 on chip
};
__host__ __device__ inline bool op_tensor(int op) { return op != OP_PLAIN; }
__host__ __device__ inline bool op_packed(int op) { return op == OP_FP8_PACKED || op == OP_FP4_PACKED; }
__host__ __device__ inline bool op_f4(int op) { return op == OP_FP4 || op == OP_FP4_PACKED; }
// FASTID_FORM_AUTO takes FP4 operands: the database's FP4 copy above
// AUTO_FP4_PACKED_MAX_Q queries, else (and whenever there is no FP4 copy)
// the packed rows expanded to FP4 on chip.  Measured with fastid_topk on 20M
// references at N = 2048 (ms, k = 16 / k = 32):
//   queries      FP4 copy    FP4 packed   FP8 copy    FP8 packed
//   32-128       2.94/2.94   1.97/2.55    5.76/5.76   3.23/4.07
//   256          3.58/3.58   3.75/4.99    6.68/6.69   6.25/8.04
//   512          6.01/5.99   7.31/9.92    10.6/10.6   12.3/16.1
//   2048         24.1/24.6   29.7/40.8    40.6/40.6   50.3/65.2
// so the FP4 packed rows are never slower than an FP8 operand, and the FP4
// copy wins from two query tiles on.
constexpr int64_t AUTO_FP4_PACKED_MAX_Q = 128;
int pick_operand(int form, bool has_fp8, bool has_fp4, int64_t n_q, bool slots16 = true);

// Argument checks of the top-k entry points (fastid_topk, fastid_topk_noalloc,
// fastid_topk_accumulate): the shared query arguments, k, and the two output
// buffers.  Sets ctx->last_error and returns EINVAL on a bad argument.
fastid_status check_topk_args(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *q, int64_t ld_q, int64_t n_q,
                              const uint8_t *modes, int32_t k, const void *out_scores, const void *out_idx);

// Events around one main compare kernel on stream `st`, recorded only while
// profiling is on (fastid_profile); no device memory is allocated.
struct MainTimer {
    fastid_ctx *ctx;
    cudaStream_t s;
    cudaEvent_t e1 = nullptr;
    MainTimer(fastid_ctx *c, cudaStream_t st);
    void done();
};

// The hit-list half of fastid_compare: every (q, r) with score <= threshold of
// this call is appended at atomicAdd(count) (stored while < capacity),
// reference indices relative to db.  No sort, no reset of the count.
fastid_status compare_append(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev, int64_t ld_q,
                             int64_t n_q, const uint8_t *modes_dev, uint32_t threshold, int64_t capacity,
                             int64_t *hit_q_dev, int64_t *hit_r_dev, uint32_t *hit_score_dev,
                             unsigned long long *count, cudaStream_t s);
// Bytes of a hit call's counter (at 0) and sort scratch (at 256).
size_t hits_aux_bytes(int64_t capacity);
// Kernel launches of launch_hits_finish for this capacity.
int64_t hits_finish_launches(int64_t capacity);
// Streamed blocks, hit lists: snaps[b] = *count, then hits appended by block
// b (since snaps[b - 1]) get r0 added to their reference index (2 launches,
// or 1 when r0 == 0).  In reduce.cu.
cudaError_t launch_hits_block_offset(const unsigned long long *count, unsigned long long *snaps, int64_t b,
                                     int64_t capacity, int64_t *hit_r, int64_t r0, int grid, cudaStream_t s);
}  // namespace fastid
