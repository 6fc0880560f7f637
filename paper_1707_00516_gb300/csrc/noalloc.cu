// fastid_topk_noalloc: the plain-form top-k with its scratch memory taken
// from one fixed array compiled into the library instead of from an
// allocator.
//
// For callers that may not allocate device memory once they are running:
// a process that reserves its whole HBM budget up front and must not fail
// later under memory pressure, a plug-in hosted by a runtime that owns every
// device allocation, or a latency-critical loop in which an allocator call
// (with its driver locks) is not acceptable.  They still pass their own
// inputs and outputs; only the library's scratch moves into the array.
//
// The array lives in this translation unit's device code.  Host code cannot
// use the symbol itself as a device address, so the first call on each device
// (with that device current) looks its address up with cudaGetSymbolAddress
// and keeps it; that lookup may also make CUDA load this file's device code on
// the device (lazy module loading), so the first call on a device should come
// before any stream capture.  The array then stays resident on every device that has
// used it until the process exits.  The kept address belongs to the device's
// primary context: after cudaDeviceReset (or anything else that destroys that
// context) it is stale, and later calls must not be made.
//
// All calls share the array and it keeps whatever the last call left in it.
// Nothing in it needs to start at zero: every word a call reads was written
// earlier in the same call.  Calls whose kernels overlap on the GPU (other
// streams, other host threads, other contexts of this process) race on the
// array; serialise them.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[FASTID_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

fastid_status set_error(fastid_ctx *ctx, fastid_status st, const std::string &msg) {
    ctx->last_error = msg;
    return st;
}

fastid_status cuda_error(fastid_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();
    return set_error(ctx, FASTID_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device address of the array on the current device (set-up on first use).
fastid_status scratch_address(fastid_ctx *ctx, uint8_t **out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return set_error(ctx, FASTID_EUNSUPPORTED, "fastid_topk_noalloc supports devices 0..63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(ctx, e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_addr[ctx->device] = p;
    }
    *out = static_cast<uint8_t *>(g_scratch_addr[ctx->device]);
    return FASTID_OK;
}

}  // namespace

extern "C" fastid_status fastid_topk_noalloc(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev,
                                             int64_t ld_q, int64_t n_q, const uint8_t *modes_dev, int32_t k,
                                             uint32_t threshold, uint32_t *out_scores_dev, int64_t *out_idx_dev,
                                             fastid_stream stream) {
    FASTID_RANGE();
    using namespace fastid;
    // the same argument checks and messages as fastid_topk
    fastid_status st0 = check_topk_args(ctx, db, queries_dev, ld_q, n_q, modes_dev, k, out_scores_dev, out_idx_dev);
    if (st0 != FASTID_OK) return st0;
    if (n_q == 0) return FASTID_OK;

    // Scratch layout: padded queries, coefficients, per-segment top-k lists.
    const int64_t ld32 = db->ld64 * 2;
    const int64_t n_q_pad = round_up(n_q, PL_TQ);
    Partition part = make_partition((int32_t)(n_q_pad / PL_TQ), db->n_pad / PL_TR, ctx->grid_topk);
    const int64_t off_q = 0;
    const int64_t off_c = round_up(off_q + n_q_pad * ld32 * (int64_t)sizeof(uint32_t), 256);
    const int64_t off_p = round_up(off_c + n_q_pad * (int64_t)sizeof(QueryCoef), 256);
    const int64_t need = off_p + (int64_t)part.grid * part.max_seg * PL_TQ * k * (int64_t)sizeof(uint64_t);
    if (need > (int64_t)FASTID_NOALLOC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "fastid_topk_noalloc: this request needs %lld bytes of scratch, more than the fixed %u bytes "
                 "(FASTID_NOALLOC_SCRATCH_BYTES); use fewer queries, a smaller k, or fastid_topk",
                 (long long)need, (unsigned)FASTID_NOALLOC_SCRATCH_BYTES);
        return set_error(ctx, FASTID_EINVAL, buf);
    }

    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaSetDevice");
    uint8_t *scr = nullptr;
    fastid_status st = scratch_address(ctx, &scr);
    if (st != FASTID_OK) return st;
    uint32_t *q32 = reinterpret_cast<uint32_t *>(scr + off_q);
    QueryCoef *coef = reinterpret_cast<QueryCoef *>(scr + off_c);
    uint64_t *partial = reinterpret_cast<uint64_t *>(scr + off_p);
    cudaStream_t s = (cudaStream_t)stream;

    e = launch_query_prep(queries_dev, ld_q, n_q, db->n_words64, modes_dev, q32, n_q_pad, ld32, coef, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "query preparation");
    MainTimer tm(ctx, s);  // profiling events, as around fastid_topk's compare kernel
    e = launch_plain(EPI_TOPK, (const uint32_t *)db->packed, db->norms, db->n_refs, ld32, db->n_words64 * 2, q32,
                     coef, n_q, threshold, k, nullptr, 0, 0, nullptr, nullptr, nullptr, nullptr, partial, part,
                     ctx->dev_status, s);
    tm.done();
    if (e != cudaSuccess) return cuda_error(ctx, e, "plain compare kernel");
    e = launch_topk_merge(partial, part, n_q, k, out_scores_dev, out_idx_dev, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "top-k merge");
    ctx->launches += 3;
    return FASTID_OK;
}
