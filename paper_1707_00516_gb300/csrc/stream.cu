// fastid_topk_streamed: top-k over host-resident references, copied to the
// device block by block (the blocked transfer of the known profiles in
// Sec. III-C), with each block's loading overlapping the previous block's
// comparison and the k-lists folded on the device.
//
// Two slots, each a device staging buffer (the block as copied, host row
// stride dropped) and a block database (padded rows + norms, and the FP8
// operand with its TMA maps).  Block b uses slot s = b % 2 on three streams:
//   copy:    wait expanded[s] (block b - 2 done with staging) -> H2D copy into
//            staging[s] -> record copied[s]
//   expand:  wait copied[s], compared[s] (block b - 2 done with the database)
//            -> rows + norms (+ FP8 operand) of db[s] -> record expanded[s]
//   compute: wait expanded[s] -> top-k of db[s] -> fold -> record compared[s]
// so block b + 1's copy and expansion, and block b + 2's copy, run while
// block b is compared.  Block sizes ramp up from an eighth of block_refs so
// that little loading is exposed before the first comparison.  All device
// memory comes from the context's stream-ordered pool and is released in
// stream order: nothing waits on the host.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace fastid;

namespace {

fastid_status sfail(fastid_ctx *ctx, fastid_status st, const char *msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

fastid_status scuda(fastid_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();
    if (ctx) ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA;
}

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Slot {
    uint64_t *staging = nullptr;  // [block][n_words64]
    fastid_refdb db;              // capacity rows; n_refs / n_pad set per block
};

// Everything one call holds: freed in stream order by the destructor.
struct StreamState {
    fastid_ctx *ctx;
    cudaStream_t s;                 // compute (the caller's stream)
    cudaStream_t copy = nullptr;    // host-to-device copies
    cudaStream_t expand = nullptr;  // block rows and operands
    cudaEvent_t ready = nullptr;    // pool allocations done (compute stream)
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t expanded[2] = {nullptr, nullptr};
    cudaEvent_t compared[2] = {nullptr, nullptr};
    cudaEvent_t tail[2] = {nullptr, nullptr};  // ends of the copy and expand streams
    Slot slot[2];
    std::vector<void *> extra;  // the entry point's own buffers
    StreamState(fastid_ctx *c, cudaStream_t st) : ctx(c), s(st) {}
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&expand, cudaStreamNonBlocking);
        cudaEvent_t *evs[] = {&ready, &copied[0], &copied[1], &expanded[0], &expanded[1],
                              &compared[0], &compared[1], &tail[0], &tail[1]};
        for (cudaEvent_t *ev : evs)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        return e;
    }
    void *take(size_t bytes, cudaError_t &e) {
        void *p = nullptr;
        if (e == cudaSuccess) {
            ++ctx->pool_allocs;
            e = cudaMallocFromPoolAsync(&p, bytes < 256 ? 256 : bytes, ctx->pool, s);
        }
        return e == cudaSuccess ? p : nullptr;
    }
    void *take_extra(size_t bytes, cudaError_t &e) {
        void *p = take(bytes, e);
        if (p) extra.push_back(p);
        return p;
    }
    ~StreamState() {
        // Frees are ordered after everything already enqueued on the copy and
        // expand streams (also on an early error return), then after the
        // compute stream's own work.
        cudaStream_t side[2] = {copy, expand};
        for (int i = 0; i < 2; ++i)
            if (side[i] && tail[i] && cudaEventRecord(tail[i], side[i]) == cudaSuccess)
                cudaStreamWaitEvent(s, tail[i], 0);
        for (Slot &sl : slot) {
            if (sl.staging) cudaFreeAsync(sl.staging, s);
            if (sl.db.packed) cudaFreeAsync(sl.db.packed, s);
            if (sl.db.norms) cudaFreeAsync(sl.db.norms, s);
            if (sl.db.fp8) cudaFreeAsync(sl.db.fp8, s);
        }
        for (void *p : extra) cudaFreeAsync(p, s);
        cudaEvent_t evs[] = {ready, copied[0], copied[1], expanded[0], expanded[1],
                             compared[0], compared[1], tail[0], tail[1]};
        for (cudaEvent_t ev : evs)
            if (ev) cudaEventDestroy(ev);
        if (copy) cudaStreamDestroy(copy);  // released once their work completes
        if (expand) cudaStreamDestroy(expand);
    }
};

// Arguments of the reference side of a streamed call.
struct StreamRefs {
    const uint64_t *host;
    int64_t n_refs;
    int32_t n_loci;
    int64_t ld_words;
    uint32_t flags;
    int64_t block_refs;
};

fastid_status check_refs(fastid_ctx *ctx, const StreamRefs &r) {
    if (!r.host) return sfail(ctx, FASTID_EINVAL, "refs_host is NULL");
    if (r.n_refs < 1 || r.n_refs > 0x7fffffffll) return sfail(ctx, FASTID_EINVAL, "n_refs out of range");
    if (r.n_loci < 1 || r.n_loci > FASTID_MAX_LOCI) return sfail(ctx, FASTID_EINVAL, "n_loci out of range");
    if (r.ld_words < (r.n_loci + 63) / 64) return sfail(ctx, FASTID_EINVAL, "ld_words too small");
    if (r.flags & ~(uint32_t)FASTID_REFS_TENSOR) return sfail(ctx, FASTID_EINVAL, "unknown flags");
    if (r.block_refs < 1) return sfail(ctx, FASTID_EINVAL, "block_refs must be >= 1");
    return FASTID_OK;
}

// The block pipeline (see the top of this file).  `setup(st)` allocates the
// entry point's own buffers (take_extra) and enqueues its initial work on the
// caller's stream; `compare(b, db, r0)` enqueues block b's comparison of
// db (references r0 .. r0 + db.n_refs - 1) there.
template <class Setup, class Compare>
fastid_status stream_blocks(fastid_ctx *ctx, const StreamRefs &R, int64_t n_q, bool slots16, cudaStream_t s,
                            Setup setup, Compare compare) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return scuda(ctx, e, "cudaSetDevice");
    const int32_t n_words = (R.n_loci + 63) / 64;
    const int64_t block = std::min<int64_t>(R.block_refs, R.n_refs);
    const int64_t cap = rup(block, ROW_ALIGN);
    // The operand the per-block comparisons will take (as the comparison
    // calls pick it): the FP8 operand is built per block only for the tensor
    // form over the FP8 copy; the plain form and the tensor form over packed
    // rows read the padded rows.
    // An FP4 form takes the packed rows of each block, expanded on chip.
    const int op = pick_operand(ctx->form, (R.flags & FASTID_REFS_TENSOR) != 0, false, n_q, slots16);
    const bool tensor = op == OP_FP8;
    const bool rows = !tensor;

    StreamState st(ctx, s);
    if ((e = st.init()) != cudaSuccess) return scuda(ctx, e, "streams and events");

    const int64_t ld64 = rup(n_words, 8);
    const int32_t kpad = tensor_kpad(R.n_loci);
    for (Slot &sl : st.slot) {
        fastid_refdb &db = sl.db;
        db.device = ctx->device;
        db.n_loci = R.n_loci;
        db.n_words64 = n_words;
        db.ld64 = ld64;
        db.flags = R.flags;
        db.kpad = kpad;
        db.kbytes4 = tensor_kbytes4(R.n_loci);
        sl.staging = static_cast<uint64_t *>(st.take((size_t)block * n_words * 8, e));
        if (rows) {
            db.packed = static_cast<uint64_t *>(st.take((size_t)cap * ld64 * 8, e));
            db.norms = static_cast<uint32_t *>(st.take((size_t)cap * 4, e));
            if (e == cudaSuccess) e = make_packed_map(&db.map_p, db.packed, cap, ld64);
            if (e == cudaSuccess) e = make_packed_map(&db.map_p4, db.packed, cap, ld64, 4, tensor_tile_r4());
        }
        if (tensor) {
            db.fp8 = static_cast<uint8_t *>(st.take((size_t)cap * kpad, e));
            if (e == cudaSuccess) e = make_operand_map(&db.map_b, db.fp8, cap, kpad, tensor_tile_r());
            if (e == cudaSuccess) e = make_operand_map(&db.map_b_half, db.fp8, cap, kpad, tensor_tile_r() / 2);
        }
    }
    if (e != cudaSuccess) return scuda(ctx, e, "block buffers");
    fastid_status rs = setup(st);
    if (rs != FASTID_OK) return rs;
    // the side streams may touch the pool allocations only after they exist
    if ((e = cudaEventRecord(st.ready, s)) != cudaSuccess || (e = cudaStreamWaitEvent(st.copy, st.ready, 0)) ||
        (e = cudaStreamWaitEvent(st.expand, st.ready, 0)))
        return scuda(ctx, e, "stream ordering");

    int64_t r0 = 0, next = std::max<int64_t>(std::min<int64_t>(block, ROW_ALIGN), block / 8);
    for (int64_t b = 0; r0 < R.n_refs; ++b) {
        const int i = (int)(b & 1);
        Slot &sl = st.slot[i];
        fastid_refdb &db = sl.db;
        const int64_t n = std::min<int64_t>(next, R.n_refs - r0);
        next = std::min<int64_t>(block, 2 * next);
        // copy: staging[i] is free once block b - 2 was expanded from it
        if (b >= 2 && (e = cudaStreamWaitEvent(st.copy, st.expanded[i], 0))) return scuda(ctx, e, "wait");
        e = cudaMemcpy2DAsync(sl.staging, (size_t)n_words * 8, R.host + r0 * R.ld_words, (size_t)R.ld_words * 8,
                              (size_t)n_words * 8, (size_t)n, cudaMemcpyHostToDevice, st.copy);
        if (e == cudaSuccess) e = cudaEventRecord(st.copied[i], st.copy);
        if (e != cudaSuccess) return scuda(ctx, e, "reference block copy");
        // expand: db[i] is free once block b - 2 was compared
        if ((e = cudaStreamWaitEvent(st.expand, st.copied[i], 0))) return scuda(ctx, e, "wait");
        if (b >= 2 && (e = cudaStreamWaitEvent(st.expand, st.compared[i], 0))) return scuda(ctx, e, "wait");
        db.n_refs = n;
        db.n_pad = rup(n, ROW_ALIGN);
        if (rows) {
            e = launch_copy_rows(sl.staging, n, n_words, n_words, db.packed, db.n_pad, ld64, db.norms, st.expand);
            ctx->launches += 1;
        }
        // The FP8 operand straight from the staged rows, on a full grid: it
        // runs beside the previous block's comparison, and the sooner it is
        // done the less it slows it down.
        if (e == cudaSuccess && tensor) {
            e = launch_refs_e4m3(sl.staging, n_words, n, n_words, db.n_pad, kpad, db.fp8, ctx->grid_tensor * 32,
                                 st.expand);
            ctx->launches += 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(st.expanded[i], st.expand);
        if (e != cudaSuccess) return scuda(ctx, e, "reference block rows");
        // compute: the block's comparison
        if ((e = cudaStreamWaitEvent(s, st.expanded[i], 0))) return scuda(ctx, e, "wait");
        if ((rs = compare(b, db, r0)) != FASTID_OK) return rs;
        if ((e = cudaEventRecord(st.compared[i], s))) return scuda(ctx, e, "stream ordering");
        r0 += n;
    }
    return FASTID_OK;
}

}  // namespace

extern "C" {

fastid_status fastid_topk_streamed(fastid_ctx *ctx, const uint64_t *refs_host, int64_t n_refs, int32_t n_loci,
                                   int64_t ld_words, uint32_t flags, int64_t block_refs,
                                   const uint64_t *queries_dev, int64_t ld_q, int64_t n_q, const uint8_t *modes_dev,
                                   int32_t k, uint32_t threshold, uint32_t *out_scores_dev, int64_t *out_idx_dev,
                                   fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    const StreamRefs R{refs_host, n_refs, n_loci, ld_words, flags, block_refs};
    fastid_status rs = check_refs(ctx, R);
    if (rs != FASTID_OK) return rs;
    if (n_q < 0 || n_q > 0x7fffffffll) return sfail(ctx, FASTID_EINVAL, "n_q out of range");
    if (n_q > 0 && (!queries_dev || !modes_dev)) return sfail(ctx, FASTID_EINVAL, "queries or modes is NULL");
    if (ld_q < (n_loci + 63) / 64) return sfail(ctx, FASTID_EINVAL, "ld_q too small");
    if (k < 1 || k > FASTID_MAX_K) return sfail(ctx, FASTID_EINVAL, "k out of range");
    if (n_q > 0 && (!out_scores_dev || !out_idx_dev)) return sfail(ctx, FASTID_EINVAL, "output is NULL");
    if (n_q == 0) return FASTID_OK;
    const cudaStream_t s = (cudaStream_t)stream;
    uint32_t *blk_s = nullptr;  // one block's lists [n_q][k]
    int64_t *blk_i = nullptr;
    auto setup = [&](StreamState &st) -> fastid_status {
        cudaError_t e = cudaSuccess;
        blk_s = static_cast<uint32_t *>(st.take_extra((size_t)n_q * k * 4, e));
        blk_i = static_cast<int64_t *>(st.take_extra((size_t)n_q * k * 8, e));
        return e == cudaSuccess ? FASTID_OK : scuda(ctx, e, "block lists");
    };
    // top-k of the block, folded into the running lists
    auto compare = [&](int64_t b, fastid_refdb &db, int64_t r0) -> fastid_status {
        uint32_t *os = b == 0 ? out_scores_dev : blk_s;
        int64_t *oi = b == 0 ? out_idx_dev : blk_i;
        fastid_status st = fastid_topk(ctx, &db, queries_dev, ld_q, n_q, modes_dev, k, threshold, os, oi, stream);
        if (st != FASTID_OK || b == 0) return st;
        cudaError_t e = launch_topk_fold(out_scores_dev, out_idx_dev, blk_s, blk_i, r0, n_q, k, s);
        if (e != cudaSuccess) return scuda(ctx, e, "fold");
        ctx->launches += 1;
        return FASTID_OK;
    };
    return stream_blocks(ctx, R, n_q, k <= 16, s, setup, compare);
}

fastid_status fastid_compare_streamed(fastid_ctx *ctx, const uint64_t *refs_host, int64_t n_refs, int32_t n_loci,
                                      int64_t ld_words, uint32_t flags, int64_t block_refs,
                                      const uint64_t *queries_dev, int64_t ld_q, int64_t n_q,
                                      const uint8_t *modes_dev, uint32_t threshold, int64_t capacity,
                                      int64_t *hit_q_dev, int64_t *hit_r_dev, uint32_t *hit_score_dev,
                                      int64_t *hit_count_dev, fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    const StreamRefs R{refs_host, n_refs, n_loci, ld_words, flags, block_refs};
    fastid_status rs = check_refs(ctx, R);
    if (rs != FASTID_OK) return rs;
    if (n_q < 0 || n_q > 0x7fffffffll) return sfail(ctx, FASTID_EINVAL, "n_q out of range");
    if (n_q > 0 && (!queries_dev || !modes_dev)) return sfail(ctx, FASTID_EINVAL, "queries or modes is NULL");
    if (ld_q < (n_loci + 63) / 64) return sfail(ctx, FASTID_EINVAL, "ld_q too small");
    if (capacity < 0) return sfail(ctx, FASTID_EINVAL, "capacity < 0");
    if (!hit_count_dev) return sfail(ctx, FASTID_EINVAL, "hit_count is NULL");
    if (capacity > 0 && (!hit_q_dev || !hit_r_dev || !hit_score_dev))
        return sfail(ctx, FASTID_EINVAL, "hit buffers are NULL");
    const cudaStream_t s = (cudaStream_t)stream;
    if (n_q == 0) {
        cudaError_t e = cudaMemsetAsync(hit_count_dev, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? FASTID_OK : scuda(ctx, e, "memset");
    }
    // blocks of the ramp: an upper bound for the count snapshots
    int64_t n_blocks = 0;
    {
        const int64_t block = std::min<int64_t>(block_refs, n_refs);
        int64_t r0 = 0, next = std::max<int64_t>(std::min<int64_t>(block, ROW_ALIGN), block / 8);
        for (; r0 < n_refs; ++n_blocks) {
            r0 += std::min<int64_t>(next, n_refs - r0);
            next = std::min<int64_t>(block, 2 * next);
        }
    }
    unsigned long long *count = nullptr, *snaps = nullptr;
    uint64_t *sort_tmp = nullptr;
    auto setup = [&](StreamState &st) -> fastid_status {
        cudaError_t e = cudaSuccess;
        uint8_t *aux = static_cast<uint8_t *>(st.take_extra(hits_aux_bytes(capacity), e));
        snaps = static_cast<unsigned long long *>(st.take_extra((size_t)n_blocks * 8, e));
        if (e == cudaSuccess) {
            count = reinterpret_cast<unsigned long long *>(aux);
            sort_tmp = reinterpret_cast<uint64_t *>(aux + 256);
            e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
        }
        return e == cudaSuccess ? FASTID_OK : scuda(ctx, e, "hit counters");
    };
    // hits of the block appended, then their reference indices made global
    auto compare = [&](int64_t b, fastid_refdb &db, int64_t r0) -> fastid_status {
        fastid_status st = compare_append(ctx, &db, queries_dev, ld_q, n_q, modes_dev, threshold, capacity,
                                          hit_q_dev, hit_r_dev, hit_score_dev, count, s);
        if (st != FASTID_OK) return st;
        cudaError_t e = launch_hits_block_offset(count, snaps, b, capacity, hit_r_dev, r0, ctx->grid_tensor * 4, s);
        if (e != cudaSuccess) return scuda(ctx, e, "hit offsets");
        ctx->launches += r0 != 0 && capacity > 0 ? 2 : 1;
        return FASTID_OK;
    };
    if ((rs = stream_blocks(ctx, R, n_q, true, s, setup, compare)) != FASTID_OK) return rs;
    cudaError_t e = launch_hits_finish(count, capacity, hit_q_dev, hit_r_dev, hit_score_dev, hit_count_dev, sort_tmp,
                                       ctx->dev_status, s);
    if (e != cudaSuccess) return scuda(ctx, e, "hit list finish");
    ctx->launches += hits_finish_launches(capacity);
    return FASTID_OK;
}

}  // extern "C"
