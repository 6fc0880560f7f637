// C ABI of the library (declared in include/fastid.h): argument checks,
// context and database ownership, scratch memory, and launch sequencing.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

using namespace fastid;

#include "internal.h"

namespace {

fastid_status fail(fastid_ctx *ctx, fastid_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

fastid_status cuda_fail(fastid_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error of this thread
    return fail(ctx, e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define FASTID_CUDA(ctx, call)                              \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Stream-ordered scratch from the context's pool.
struct Scratch {
    fastid_ctx *ctx;
    cudaStream_t s;
    void *p = nullptr;
    Scratch(fastid_ctx *c, cudaStream_t st) : ctx(c), s(st) {}
    cudaError_t alloc(size_t bytes) {
        ++ctx->pool_allocs;
        return cudaMallocFromPoolAsync(&p, bytes < 256 ? 256 : bytes, ctx->pool, s);
    }
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

// Carves aligned sub-buffers out of one allocation.
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        off = (off + 255) & ~size_t(255);
        size_t at = off;
        off += count * sizeof(T);
        return at;
    }
};

template <class T>
T *at(void *base, size_t off) {
    return reinterpret_cast<T *>(static_cast<uint8_t *>(base) + off);
}

fastid_status check_query_args(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *q, int64_t ld_q,
                               int64_t n_q, const uint8_t *modes) {
    if (!ctx) return FASTID_EINVAL;
    if (!db) return fail(ctx, FASTID_EINVAL, "database is NULL");
    if (n_q < 0 || n_q > 0x7fffffffll) return fail(ctx, FASTID_EINVAL, "n_q out of range: %lld", (long long)n_q);
    if (n_q > 0 && (!q || !modes)) return fail(ctx, FASTID_EINVAL, "queries or modes is NULL");
    if (ld_q < db->n_words64) return fail(ctx, FASTID_EINVAL, "ld_q %lld < %d words", (long long)ld_q, db->n_words64);
    if (db->device != ctx->device) return fail(ctx, FASTID_EINVAL, "database belongs to another device");
    return FASTID_OK;
}

void count_launches(fastid_ctx *ctx, int64_t n) { ctx->launches += n; }

// Pads the queries into the plain layout and computes per-query coefficients.
struct PreparedQueries {
    uint32_t *q32;
    QueryCoef *coef;
    int64_t n_q_pad;
};

}  // namespace

extern "C" {

int32_t fastid_version(void) { return 100; }

const char *fastid_status_string(fastid_status s) {
    switch (s) {
        case FASTID_OK: return "FASTID_OK";
        case FASTID_EINVAL: return "FASTID_EINVAL";
        case FASTID_ENOMEM: return "FASTID_ENOMEM";
        case FASTID_ECUDA: return "FASTID_ECUDA";
        case FASTID_EOVERFLOW: return "FASTID_EOVERFLOW";
        case FASTID_ETIMEOUT: return "FASTID_ETIMEOUT";
        case FASTID_EUNSUPPORTED: return "FASTID_EUNSUPPORTED";
        case FASTID_EDEVICE: return "FASTID_EDEVICE";
    }
    return "FASTID_UNKNOWN";
}

fastid_status fastid_create(fastid_ctx **out, int32_t device) {
    if (!out) return FASTID_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return FASTID_ECUDA;
    }
    if (device < 0 || device >= n) return FASTID_EINVAL;
    fastid_ctx *ctx = new (std::nothrow) fastid_ctx();
    if (!ctx) return FASTID_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&ctx->pool, &props);
    }
    if (e == cudaSuccess) {
        uint64_t keep = ~0ull;  // keep freed scratch cached in the pool
        e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dev_status, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->dev_status, 0, 8 * sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->dev_status) cudaFree(ctx->dev_status);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA;
    }
    ctx->grid_topk = plain_grid_target(EPI_TOPK, device);
    ctx->grid_hits = plain_grid_target(EPI_HITS, device);
    ctx->grid_scores = plain_grid_target(EPI_SCORES32, device);
    ctx->grid_tensor = tensor_grid_target(device);
    ctx->pair_clusters = tensor_pair_clusters(device);
    *out = ctx;
    return FASTID_OK;
}

fastid_status fastid_destroy(fastid_ctx *ctx) {
    if (!ctx) return FASTID_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    for (auto &pr : ctx->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    delete ctx;
    return FASTID_OK;
}

fastid_status fastid_profile(fastid_ctx *ctx, int32_t enable) {
    if (!ctx) return FASTID_EINVAL;
    ctx->profile = enable != 0;
    return FASTID_OK;
}

fastid_status fastid_profile_read(fastid_ctx *ctx, double *main_ms, int64_t *main_launches, int64_t *all_launches,
                                  int32_t reset) {
    if (!ctx) return FASTID_EINVAL;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    double ms = 0.0;
    for (size_t i = 0; i < ctx->events_used; ++i) {
        FASTID_CUDA(ctx, cudaEventSynchronize(ctx->events[i].second));
        float t = 0.f;
        FASTID_CUDA(ctx, cudaEventElapsedTime(&t, ctx->events[i].first, ctx->events[i].second));
        ms += t;
    }
    if (main_ms) *main_ms = ms;
    if (main_launches) *main_launches = (int64_t)ctx->events_used;
    if (all_launches) *all_launches = ctx->launches;
    if (reset) {
        ctx->events_used = 0;
        ctx->launches = 0;
    }
    return FASTID_OK;
}

const char *fastid_last_error(const fastid_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

fastid_status fastid_memory_info(fastid_ctx *ctx, int64_t *pool_allocs, int64_t *pool_used_bytes,
                                 int64_t *pool_reserved_bytes) {
    if (!ctx) return FASTID_EINVAL;
    if (pool_allocs) *pool_allocs = ctx->pool_allocs;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    uint64_t used = 0, reserved = 0;
    FASTID_CUDA(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used));
    FASTID_CUDA(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    if (pool_used_bytes) *pool_used_bytes = (int64_t)used;
    if (pool_reserved_bytes) *pool_reserved_bytes = (int64_t)reserved;
    return FASTID_OK;
}

fastid_status fastid_set_form(fastid_ctx *ctx, int32_t form) {
    if (!ctx) return FASTID_EINVAL;
    if (form != FASTID_FORM_AUTO && form != FASTID_FORM_PLAIN && form != FASTID_FORM_TENSOR &&
        form != FASTID_FORM_TENSOR_PACKED && form != FASTID_FORM_TENSOR_FP4 && form != FASTID_FORM_TENSOR_FP4_PACKED)
        return fail(ctx, FASTID_EINVAL, "unknown form %d", form);
    ctx->form = form;
    return FASTID_OK;
}

fastid_status fastid_sync_status(fastid_ctx *ctx, fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    uint32_t host[4];
    // read and clear in one atomic step per word, then copy the snapshot
    FASTID_CUDA(ctx, launch_status_take(ctx->dev_status, ctx->dev_status + 4, s));
    FASTID_CUDA(ctx, cudaMemcpyAsync(host, ctx->dev_status + 4, sizeof host, cudaMemcpyDeviceToHost, s));
    FASTID_CUDA(ctx, cudaStreamSynchronize(s));
    if (host[0] & ST_DEVICE) return fail(ctx, FASTID_EDEVICE, "device-side check failed (detail %u)", host[1]);
    if (host[0] & ST_TIMEOUT) return fail(ctx, FASTID_ETIMEOUT, "bounded device wait ran out (site %u)", host[1]);
    if (host[0] & ST_OVERFLOW) return fail(ctx, FASTID_EOVERFLOW, "hit list overflow");
    return FASTID_OK;
}

fastid_status fastid_pack(fastid_ctx *ctx, const uint8_t *alleles_dev, int64_t n, int32_t n_loci,
                          int64_t ld_alleles, uint64_t *packed_dev, int64_t ld_words, uint32_t *norms_dev,
                          fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (n < 0) return fail(ctx, FASTID_EINVAL, "n < 0");
    if (n_loci < 1 || n_loci > FASTID_MAX_LOCI) return fail(ctx, FASTID_EINVAL, "n_loci out of range: %d", n_loci);
    if (ld_alleles < n_loci) return fail(ctx, FASTID_EINVAL, "ld_alleles < n_loci");
    if (ld_words < (n_loci + 63) / 64) return fail(ctx, FASTID_EINVAL, "ld_words too small");
    if (n > 0 && (!alleles_dev || !packed_dev)) return fail(ctx, FASTID_EINVAL, "NULL buffer");
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    FASTID_CUDA(ctx, launch_pack(alleles_dev, n, n_loci, ld_alleles, packed_dev, ld_words, norms_dev,
                                 (cudaStream_t)stream));
    count_launches(ctx, n > 0);
    return FASTID_OK;
}

fastid_status fastid_mix(fastid_ctx *ctx, const uint64_t *src_dev, int64_t ld_src, int32_t n_words,
                         const int32_t *offsets_dev, int64_t n_mix, uint64_t *out_dev, int64_t ld_out,
                         uint32_t *norms_dev, fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (n_mix < 0) return fail(ctx, FASTID_EINVAL, "n_mix < 0");
    if (n_words < 1 || ld_src < n_words || ld_out < n_words)
        return fail(ctx, FASTID_EINVAL, "bad word counts (n_words %d, ld_src %lld, ld_out %lld)", n_words,
                    (long long)ld_src, (long long)ld_out);
    if (n_mix > 0 && (!src_dev || !offsets_dev || !out_dev)) return fail(ctx, FASTID_EINVAL, "NULL buffer");
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    FASTID_CUDA(ctx, launch_mix(src_dev, ld_src, n_words, offsets_dev, n_mix, out_dev, ld_out, norms_dev,
                                (cudaStream_t)stream));
    count_launches(ctx, n_mix > 0);
    return FASTID_OK;
}

fastid_status fastid_load_refs(fastid_ctx *ctx, const uint64_t *packed_dev, int64_t n_refs, int32_t n_loci,
                               int64_t ld_words, uint32_t flags, fastid_refdb **out, fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!out) return fail(ctx, FASTID_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_refs < 1 || n_refs > 0x7fffffffll) return fail(ctx, FASTID_EINVAL, "n_refs out of range");
    if (n_loci < 1 || n_loci > FASTID_MAX_LOCI) return fail(ctx, FASTID_EINVAL, "n_loci out of range");
    if (ld_words < (n_loci + 63) / 64) return fail(ctx, FASTID_EINVAL, "ld_words too small");
    if (!packed_dev) return fail(ctx, FASTID_EINVAL, "packed is NULL");
    if (flags & ~(uint32_t)(FASTID_REFS_TENSOR | FASTID_REFS_FP4)) return fail(ctx, FASTID_EINVAL, "unknown flags");
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    fastid_refdb *db = new (std::nothrow) fastid_refdb();
    if (!db) return fail(ctx, FASTID_ENOMEM, "host allocation");
    db->device = ctx->device;
    db->n_refs = n_refs;
    db->n_loci = n_loci;
    db->n_words64 = (n_loci + 63) / 64;
    db->ld64 = round_up(db->n_words64, 8);
    db->n_pad = round_up(n_refs, ROW_ALIGN);
    db->flags = flags;
    size_t pbytes = (size_t)db->n_pad * db->ld64 * 8, nbytes = (size_t)db->n_pad * 4;
    cudaError_t e = cudaMalloc(&db->packed, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&db->norms, nbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (db->packed) cudaFree(db->packed);
        delete db;
        return fail(ctx, e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA,
                    "database allocation (%zu bytes): %s", pbytes + nbytes, cudaGetErrorString(e));
    }
    db->bytes = (int64_t)(pbytes + nbytes);
    e = launch_copy_rows(packed_dev, n_refs, ld_words, db->n_words64, db->packed, db->n_pad, db->ld64, db->norms,
                         (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaFree(db->packed);
        cudaFree(db->norms);
        delete db;
        return cuda_fail(ctx, e, "copy rows");
    }
    count_launches(ctx, 1);
    db->kpad = tensor_kpad(n_loci);
    db->kbytes4 = tensor_kbytes4(n_loci);
    e = make_packed_map(&db->map_p, db->packed, db->n_pad, db->ld64);
    if (e == cudaSuccess) e = make_packed_map(&db->map_p4, db->packed, db->n_pad, db->ld64, 4, tensor_tile_r4());
    if (e != cudaSuccess) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(db->packed);
        cudaFree(db->norms);
        delete db;
        return cuda_fail(ctx, e, "packed operand map");
    }
    if (flags & FASTID_REFS_TENSOR) {
        const size_t fbytes = (size_t)db->n_pad * db->kpad;
        e = cudaMalloc(&db->fp8, fbytes);
        if (e == cudaSuccess)
            e = launch_refs_e4m3(db->packed, db->ld64, db->n_pad, (int32_t)db->ld64, db->n_pad, db->kpad, db->fp8,
                                 ctx->grid_tensor * 32, (cudaStream_t)stream);
        if (e == cudaSuccess) e = make_operand_map(&db->map_b, db->fp8, db->n_pad, db->kpad, tensor_tile_r());
        if (e == cudaSuccess)
            e = make_operand_map(&db->map_b_half, db->fp8, db->n_pad, db->kpad, tensor_tile_r() / 2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize((cudaStream_t)stream);
            if (db->fp8) cudaFree(db->fp8);
            cudaFree(db->packed);
            cudaFree(db->norms);
            delete db;
            return fail(ctx, e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA,
                        "tensor operand copy (%zu bytes): %s", fbytes, cudaGetErrorString(e));
        }
        db->bytes += (int64_t)fbytes;
        count_launches(ctx, 1);
    }
    if (flags & FASTID_REFS_FP4) {
        const size_t fbytes = (size_t)db->n_pad * db->kbytes4;
        e = cudaMalloc(&db->fp4, fbytes);
        if (e == cudaSuccess)
            e = launch_refs_e2m1(db->packed, db->ld64, db->n_pad, (int32_t)db->ld64, db->n_pad, db->kbytes4, db->fp4,
                                 ctx->grid_tensor * 32, (cudaStream_t)stream);
        if (e == cudaSuccess) e = make_operand_map(&db->map_b4, db->fp4, db->n_pad, db->kbytes4, tensor_tile_r4());
        if (e == cudaSuccess)
            e = make_operand_map(&db->map_b4_half, db->fp4, db->n_pad, db->kbytes4, tensor_tile_r4() / 2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize((cudaStream_t)stream);
            if (db->fp4) cudaFree(db->fp4);
            if (db->fp8) cudaFree(db->fp8);
            cudaFree(db->packed);
            cudaFree(db->norms);
            delete db;
            return fail(ctx, e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA,
                        "FP4 operand copy (%zu bytes): %s", fbytes, cudaGetErrorString(e));
        }
        db->bytes += (int64_t)fbytes;
        count_launches(ctx, 1);
    }
    *out = db;
    return FASTID_OK;
}

fastid_status fastid_free_refs(fastid_ctx *ctx, fastid_refdb *db) {
    if (!db) return FASTID_OK;
    if (db->view) {  // the parent owns the memory
        delete db;
        return FASTID_OK;
    }
    cudaSetDevice(db->device);
    cudaDeviceSynchronize();
    cudaFree(db->packed);
    cudaFree(db->norms);
    if (db->fp8) cudaFree(db->fp8);
    if (db->fp4) cudaFree(db->fp4);
    delete db;
    (void)ctx;
    return FASTID_OK;
}

fastid_status fastid_refs_view(fastid_ctx *ctx, const fastid_refdb *db, int64_t r_begin, int64_t n_refs,
                               fastid_refdb **out) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!out) return fail(ctx, FASTID_EINVAL, "out is NULL");
    *out = nullptr;
    if (!db) return fail(ctx, FASTID_EINVAL, "database is NULL");
    if (db->device != ctx->device) return fail(ctx, FASTID_EINVAL, "database belongs to another device");
    if (r_begin < 0 || r_begin % FASTID_VIEW_ALIGN != 0)
        return fail(ctx, FASTID_EINVAL, "r_begin %lld is not a multiple of %d", (long long)r_begin, FASTID_VIEW_ALIGN);
    if (n_refs < 1 || r_begin + n_refs > db->n_refs)
        return fail(ctx, FASTID_EINVAL, "rows [%lld, %lld) outside the database's %lld", (long long)r_begin,
                    (long long)(r_begin + n_refs), (long long)db->n_refs);
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    fastid_refdb *v = new (std::nothrow) fastid_refdb(*db);
    if (!v) return fail(ctx, FASTID_ENOMEM, "host allocation");
    v->view = true;
    v->bytes = 0;
    v->n_refs = n_refs;
    // rows up to n_pad exist in the parent (its rows are padded to ROW_ALIGN
    // and r_begin is a multiple of it); the kernels mask rows >= n_refs
    v->n_pad = round_up(n_refs, ROW_ALIGN);
    v->packed = db->packed + r_begin * db->ld64;
    v->norms = db->norms + r_begin;
    cudaError_t e = make_packed_map(&v->map_p, v->packed, v->n_pad, v->ld64);
    if (e == cudaSuccess) e = make_packed_map(&v->map_p4, v->packed, v->n_pad, v->ld64, 4, tensor_tile_r4());
    if (e == cudaSuccess && db->fp8) {
        v->fp8 = db->fp8 + r_begin * (int64_t)db->kpad;
        e = make_operand_map(&v->map_b, v->fp8, v->n_pad, v->kpad, tensor_tile_r());
        if (e == cudaSuccess) e = make_operand_map(&v->map_b_half, v->fp8, v->n_pad, v->kpad, tensor_tile_r() / 2);
    }
    if (e == cudaSuccess && db->fp4) {
        v->fp4 = db->fp4 + r_begin * (int64_t)db->kbytes4;
        e = make_operand_map(&v->map_b4, v->fp4, v->n_pad, v->kbytes4, tensor_tile_r4());
        if (e == cudaSuccess)
            e = make_operand_map(&v->map_b4_half, v->fp4, v->n_pad, v->kbytes4, tensor_tile_r4() / 2);
    }
    if (e != cudaSuccess) {
        delete v;
        return cuda_fail(ctx, e, "view operand maps");
    }
    *out = v;
    return FASTID_OK;
}

fastid_status fastid_topk_fold(fastid_ctx *ctx, uint32_t *run_scores_dev, int64_t *run_idx_dev,
                               const uint32_t *blk_scores_dev, const int64_t *blk_idx_dev, int64_t ref_offset,
                               int64_t n_q, int32_t k, fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (n_q < 0 || n_q > 0x7fffffffll) return fail(ctx, FASTID_EINVAL, "n_q out of range: %lld", (long long)n_q);
    if (k < 1 || k > FASTID_MAX_K) return fail(ctx, FASTID_EINVAL, "k out of range: %d", k);
    if (ref_offset < 0 || ref_offset > 0x7fffffffll)
        return fail(ctx, FASTID_EINVAL, "ref_offset out of range: %lld", (long long)ref_offset);
    if (n_q > 0 && (!run_scores_dev || !run_idx_dev || !blk_scores_dev || !blk_idx_dev))
        return fail(ctx, FASTID_EINVAL, "list buffer is NULL");
    if (n_q == 0) return FASTID_OK;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    FASTID_CUDA(ctx, launch_topk_fold(run_scores_dev, run_idx_dev, blk_scores_dev, blk_idx_dev, ref_offset, n_q, k,
                                      (cudaStream_t)stream));
    count_launches(ctx, 1);
    return FASTID_OK;
}

fastid_status fastid_refs_info(const fastid_refdb *db, int64_t *n_refs, int32_t *n_loci, uint32_t *flags,
                               int64_t *device_bytes) {
    if (!db) return FASTID_EINVAL;
    if (n_refs) *n_refs = db->n_refs;
    if (n_loci) *n_loci = db->n_loci;
    if (flags) *flags = db->flags;
    if (device_bytes) *device_bytes = db->bytes;
    return FASTID_OK;
}

}  // extern "C"

namespace {

// Shared front half of the comparison calls: scratch for the padded queries
// and coefficients (+ `extra` bytes), query preparation.
fastid_status prepare(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *q, int64_t ld_q, int64_t n_q,
                      const uint8_t *modes, cudaStream_t s, Scratch &scr, size_t extra, size_t *extra_off,
                      PreparedQueries *pq) {
    const int64_t ld32 = db->ld64 * 2;
    pq->n_q_pad = round_up(n_q, PL_TQ);
    Carver cv;
    size_t o_q = cv.take<uint32_t>((size_t)pq->n_q_pad * ld32);
    size_t o_c = cv.take<QueryCoef>((size_t)pq->n_q_pad);
    *extra_off = cv.take<uint8_t>(extra);
    FASTID_CUDA(ctx, scr.alloc(cv.off));
    pq->q32 = at<uint32_t>(scr.p, o_q);
    pq->coef = at<QueryCoef>(scr.p, o_c);
    FASTID_CUDA(ctx, launch_query_prep(q, ld_q, n_q, db->n_words64, modes, pq->q32, pq->n_q_pad, ld32, pq->coef, s));
    count_launches(ctx, 1);
    return FASTID_OK;
}

// The call's operand (fastid::Operand).  slots16: the launch keeps 16-slot
// lists (k <= 16, or no top-k).
fastid_status pick_form(fastid_ctx *ctx, const fastid_refdb *db, int64_t n_q, int *op, bool slots16 = true) {
    *op = fastid::pick_operand(ctx->form, db->fp8 != nullptr, db->fp4 != nullptr, n_q, slots16);
    return FASTID_OK;
}

// Tensor-form front half: e4m3 query operand + c_q in scratch, its TMA map,
// and the partition over (128-query tile, 256-reference tile) units.
// Paired launches (2-CTA clusters sharing reference stages) from two query
// tiles on.  The two CTAs of a pair consume every reference tile together, so
// it leaves DRAM once; single-tile groups that share a slice only through L2
// drift apart and re-read it.  Measured on 20M references at N = 2048: 200
// queries 6.7 ms paired against 8.7 ms unpaired, 300 queries (padded to four
// tiles) 13.5 ms against 25 ms.
constexpr int PAIR_MIN_TILES = 2;

// Tensor-form front half of a call: schedule, scratch (e4m3 query operand,
// c_q, and `extra` bytes computed from the schedule), operand encoding and
// the launch description for one panel.
struct TensorPrep {
    TcLaunch L;
    int64_t n_ctas;
};

enum ExtraKind { EXTRA_NONE, EXTRA_TOPK, EXTRA_HITS };

// op (an operand other than OP_PLAIN): FP8 or FP4 operands; packed rows
// expanded on chip are unpaired, and their FP8 queries are encoded at half
// scale to match the expanded 2.0.
fastid_status prepare_tensor(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *q, int64_t ld_q, int64_t n_q,
                             const uint8_t *modes, cudaStream_t s, Scratch &scr, ExtraKind ek, int64_t karg,
                             size_t *extra_off, TensorPrep *tp, int op) {
    TcLaunch &L = tp->L;
    memset(&L, 0, sizeof L);
    const bool pk = op_packed(op), f4 = op_f4(op);
    const int64_t n_qt = round_up(n_q, tensor_tile_q()) / tensor_tile_q();
    L.pk = pk ? 1 : 0;
    L.f4 = f4 ? 1 : 0;
    L.pair = (!pk && ctx->pair_clusters > 0 && n_qt >= PAIR_MIN_TILES) ? 1 : 0;
    // multicast pairs: on 2048 x 20M at N = 2048 they took 24.6 (FP4) / 41.3 (FP8)
    // ms against 25.4 / 46.5 ms as 2-SM MMAs (which batched plans may choose)
    L.cg2 = 0;
    const int64_t n_q_pad = round_up(n_q, (int64_t)tensor_tile_q() * (L.pair ? 2 : 1));
    const int64_t n_qq = n_q_pad / tensor_tile_q() / (L.pair ? 2 : 1);
    const int64_t tile_r = f4 ? tensor_tile_r4() : tensor_tile_r();
    const int64_t n_rt = (db->n_pad + tile_r - 1) / tile_r;
    const int32_t kbytes = f4 ? db->kbytes4 : db->kpad;  // operand row bytes
    const int64_t tile_bytes = tile_r * (pk ? db->ld64 * 8 : kbytes);
    L.n_groups = make_tensor_schedule(1, &n_qq, &n_rt, &tile_bytes, L.pair ? ctx->pair_clusters : ctx->grid_tensor,
                                      L.pair ? 2 : 1, L.sched, L.order, &L.n_slots);
    if (L.n_groups == -2) return fail(ctx, FASTID_EDEVICE, "schedule self-check failed (debug build)");
    if (L.n_groups < 0) return fail(ctx, FASTID_EINVAL, "too many query tiles (top-k slots)");
    tp->n_ctas = (int64_t)L.n_groups * (L.pair ? 2 : 1);
    size_t extra = 0;
    if (ek == EXTRA_TOPK) extra = (size_t)L.n_slots * tensor_tile_q() * (size_t)karg * 8;
    if (ek == EXTRA_HITS) extra = 256 + (size_t)(2 + hits_sort_elems(karg) * 3 / 2 + 1) * 8;
    Carver cv;
    size_t o_a = cv.take<uint8_t>((size_t)n_q_pad * kbytes);
    size_t o_c = cv.take<float>((size_t)n_q_pad);
    *extra_off = cv.take<uint8_t>(extra);
    FASTID_CUDA(ctx, scr.alloc(cv.off));
    uint8_t *a = at<uint8_t>(scr.p, o_a);
    float *qconst = at<float>(scr.p, o_c);
    // spread the input queries over every tile of the operand (see
    // spread_row_to_query)
    const int64_t spread = n_q_pad / tensor_tile_q();
    if (f4)
        FASTID_CUDA(ctx, launch_queries_e2m1(q, ld_q, n_q, db->n_words64, db->n_loci, modes, n_q_pad, kbytes, a,
                                             qconst, spread, s));
    else
        FASTID_CUDA(ctx, launch_queries_e4m3(q, ld_q, n_q, db->n_words64, db->n_loci, modes, n_q_pad, kbytes, a,
                                             qconst, pk, spread, s));
    count_launches(ctx, 1);
    FASTID_CUDA(ctx, make_operand_map(&L.map_a[0], a, n_q_pad, kbytes, tensor_tile_q()));
    L.n_panels = 1;
    if (f4)
        L.map_b[0] = pk ? db->map_p4 : L.pair ? db->map_b4_half : db->map_b4;
    else
        L.map_b[0] = pk ? db->map_p : L.pair ? db->map_b_half : db->map_b;
    L.n_refs[0] = db->n_refs;
    L.n_q[0] = n_q;
    L.n_rt[0] = n_rt;
    L.kpad[0] = kbytes;
    L.qconst[0] = qconst;
    L.qspread[0] = (int32_t)spread;
    L.status = ctx->dev_status;
    return FASTID_OK;
}

uint32_t clamp_threshold(uint32_t t, int32_t n_loci) {
    if (t == 0xFFFFFFFFu) return t;
    return t > (uint32_t)n_loci ? (uint32_t)n_loci : t;
}

}  // namespace

extern "C" {

fastid_status fastid_scores(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev, int64_t ld_q,
                            int64_t n_q, const uint8_t *modes_dev, void *out_dev, int32_t out_bytes,
                            int64_t ld_out, fastid_stream stream) {
    FASTID_RANGE();
    fastid_status st = check_query_args(ctx, db, queries_dev, ld_q, n_q, modes_dev);
    if (st) return st;
    if (out_bytes != 2 && out_bytes != 4) return fail(ctx, FASTID_EINVAL, "out_bytes must be 2 or 4");
    if (out_bytes == 2 && db->n_loci > 65535) return fail(ctx, FASTID_EINVAL, "uint16 scores need n_loci <= 65535");
    if (ld_out < db->n_refs) return fail(ctx, FASTID_EINVAL, "ld_out < n_refs");
    if (n_q > 0 && !out_dev) return fail(ctx, FASTID_EINVAL, "out is NULL");
    int tensor;
    if ((st = pick_form(ctx, db, n_q, &tensor))) return st;
    if (n_q == 0) return FASTID_OK;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scr(ctx, s);
    size_t xo;
    if (tensor) {
        TensorPrep tp;
        if ((st = prepare_tensor(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, EXTRA_NONE, 0, &xo, &tp,
                                 tensor)))
            return st;
        tp.L.epi = out_bytes == 2 ? EPI_SCORES16 : EPI_SCORES32;
        tp.L.threshold = 0xFFFFFFFFu;
        tp.L.k = 1;
        tp.L.out = out_dev;
        tp.L.ld_out = ld_out;
        MainTimer tm(ctx, s);
        FASTID_CUDA(ctx, launch_tensor_multi(256, tp.L, s));
        tm.done();
        count_launches(ctx, 1);
        return FASTID_OK;
    }
    PreparedQueries pq;
    if ((st = prepare(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, 0, &xo, &pq))) return st;
    Partition part = make_partition((int32_t)(pq.n_q_pad / PL_TQ), db->n_pad / PL_TR, ctx->grid_scores);
    MainTimer tm(ctx, s);
    FASTID_CUDA(ctx, launch_plain(out_bytes == 2 ? EPI_SCORES16 : EPI_SCORES32, (const uint32_t *)db->packed,
                                  db->norms, db->n_refs, db->ld64 * 2, db->n_words64 * 2, pq.q32, pq.coef, n_q,
                                  0xFFFFFFFFu, 1, out_dev, ld_out, 0, nullptr, nullptr, nullptr, nullptr,
                                  nullptr, part, ctx->dev_status, s));
    tm.done();
    count_launches(ctx, 1);
    return FASTID_OK;
}

fastid_status fastid_topk(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev, int64_t ld_q,
                          int64_t n_q, const uint8_t *modes_dev, int32_t k, uint32_t threshold,
                          uint32_t *out_scores_dev, int64_t *out_idx_dev, fastid_stream stream) {
    FASTID_RANGE();
    fastid_status st = fastid::check_topk_args(ctx, db, queries_dev, ld_q, n_q, modes_dev, k, out_scores_dev,
                                               out_idx_dev);
    if (st) return st;
    int tensor;
    if ((st = pick_form(ctx, db, n_q, &tensor, k <= 16))) return st;
    if (n_q == 0) return FASTID_OK;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scr(ctx, s);
    if (tensor) {
        TensorPrep tp;
        size_t xo;
        if ((st = prepare_tensor(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, EXTRA_TOPK, k, &xo, &tp,
                                 tensor)))
            return st;
        uint64_t *partial = at<uint64_t>(scr.p, xo);
        tp.L.epi = EPI_TOPK;
        tp.L.threshold = clamp_threshold(threshold, db->n_loci);
        tp.L.k = k;
        tp.L.partial = partial;
        MainTimer tm(ctx, s);
        FASTID_CUDA(ctx, launch_tensor_multi(256, tp.L, s));
        tm.done();
        FASTID_CUDA(ctx, launch_merge_sched(partial, tp.L, nullptr, n_q, out_scores_dev, out_idx_dev, s));
        count_launches(ctx, 2);
        return FASTID_OK;
    }
    const int64_t n_q_pad = round_up(n_q, PL_TQ);
    Partition part = make_partition((int32_t)(n_q_pad / PL_TQ), db->n_pad / PL_TR, ctx->grid_topk);
    const size_t partial_elems = (size_t)part.grid * part.max_seg * PL_TQ * k;
    PreparedQueries pq;
    size_t xo;
    if ((st = prepare(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, partial_elems * 8, &xo, &pq))) return st;
    uint64_t *partial = at<uint64_t>(scr.p, xo);
    MainTimer tm(ctx, s);
    FASTID_CUDA(ctx, launch_plain(EPI_TOPK, (const uint32_t *)db->packed, db->norms, db->n_refs, db->ld64 * 2,
                                  db->n_words64 * 2, pq.q32, pq.coef, n_q, threshold, k, nullptr, 0, 0, nullptr,
                                  nullptr, nullptr, nullptr, partial, part, ctx->dev_status, s));
    tm.done();
    FASTID_CUDA(ctx, launch_topk_merge(partial, part, n_q, k, out_scores_dev, out_idx_dev, s));
    count_launches(ctx, 2);
    return FASTID_OK;
}

fastid_status fastid_topk_accumulate(fastid_ctx *ctx, const fastid_refdb *db, int64_t ref_offset,
                                     const uint64_t *queries_dev, int64_t ld_q, int64_t n_q, const uint8_t *modes_dev,
                                     int32_t k, uint32_t threshold, uint32_t *run_scores_dev, int64_t *run_idx_dev,
                                     fastid_stream stream) {
    FASTID_RANGE();
    fastid_status st = fastid::check_topk_args(ctx, db, queries_dev, ld_q, n_q, modes_dev, k, run_scores_dev,
                                               run_idx_dev);
    if (st) return st;
    if (ref_offset < 0 || ref_offset + db->n_refs > 0x7fffffffll)
        return fail(ctx, FASTID_EINVAL, "ref_offset out of range: %lld", (long long)ref_offset);
    int op;
    if ((st = pick_form(ctx, db, n_q, &op, k <= 16))) return st;
    if (n_q == 0) return FASTID_OK;
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scr(ctx, s);
    if (op) {
        TensorPrep tp;
        size_t xo;
        if ((st = prepare_tensor(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, EXTRA_TOPK, k, &xo, &tp, op)))
            return st;
        uint64_t *partial = at<uint64_t>(scr.p, xo);
        tp.L.epi = EPI_TOPK;
        tp.L.threshold = clamp_threshold(threshold, db->n_loci);
        tp.L.k = k;
        tp.L.partial = partial;
        MainTimer tm(ctx, s);
        FASTID_CUDA(ctx, launch_tensor_multi(256, tp.L, s));
        tm.done();
        FASTID_CUDA(ctx, launch_merge_sched(partial, tp.L, nullptr, n_q, run_scores_dev, run_idx_dev, s, true,
                                            ref_offset));
        count_launches(ctx, 2);
        return FASTID_OK;
    }
    // plain form: the call's lists in scratch, then folded
    const int64_t n_q_pad = round_up(n_q, PL_TQ);
    Partition part = make_partition((int32_t)(n_q_pad / PL_TQ), db->n_pad / PL_TR, ctx->grid_topk);
    const size_t partial_elems = (size_t)part.grid * part.max_seg * PL_TQ * k;
    PreparedQueries pq;
    size_t xo;
    if ((st = prepare(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, partial_elems * 8 + (size_t)n_q * k * 12 + 512,
                      &xo, &pq)))
        return st;
    uint64_t *partial = at<uint64_t>(scr.p, xo);
    uint8_t *lists = reinterpret_cast<uint8_t *>(partial + partial_elems);
    lists += (256 - reinterpret_cast<uintptr_t>(lists) % 256) % 256;
    uint32_t *blk_s = reinterpret_cast<uint32_t *>(lists);
    int64_t *blk_i = reinterpret_cast<int64_t *>(lists + (((size_t)n_q * k * 4 + 255) & ~size_t(255)));
    MainTimer tm(ctx, s);
    FASTID_CUDA(ctx, launch_plain(EPI_TOPK, (const uint32_t *)db->packed, db->norms, db->n_refs, db->ld64 * 2,
                                  db->n_words64 * 2, pq.q32, pq.coef, n_q, threshold, k, nullptr, 0, 0, nullptr,
                                  nullptr, nullptr, nullptr, partial, part, ctx->dev_status, s));
    tm.done();
    FASTID_CUDA(ctx, launch_topk_merge(partial, part, n_q, k, blk_s, blk_i, s));
    FASTID_CUDA(ctx, launch_topk_fold(run_scores_dev, run_idx_dev, blk_s, blk_i, ref_offset, n_q, k, s));
    count_launches(ctx, 3);
    return FASTID_OK;
}

fastid_status fastid_compare(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev, int64_t ld_q,
                             int64_t n_q, const uint8_t *modes_dev, uint32_t threshold, int64_t capacity,
                             int64_t *hit_q_dev, int64_t *hit_r_dev, uint32_t *hit_score_dev,
                             int64_t *hit_count_dev, fastid_stream stream) {
    FASTID_RANGE();
    fastid_status st = check_query_args(ctx, db, queries_dev, ld_q, n_q, modes_dev);
    if (st) return st;
    if (capacity < 0) return fail(ctx, FASTID_EINVAL, "capacity < 0");
    if (!hit_count_dev) return fail(ctx, FASTID_EINVAL, "hit_count is NULL");
    if (capacity > 0 && (!hit_q_dev || !hit_r_dev || !hit_score_dev))
        return fail(ctx, FASTID_EINVAL, "hit buffers are NULL");
    FASTID_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (n_q == 0) {
        FASTID_CUDA(ctx, cudaMemsetAsync(hit_count_dev, 0, sizeof(int64_t), s));
        return FASTID_OK;
    }
    // device hit counter and the sort's scratch
    Scratch aux(ctx, s);
    FASTID_CUDA(ctx, aux.alloc(fastid::hits_aux_bytes(capacity)));
    unsigned long long *count = at<unsigned long long>(aux.p, 0);
    uint64_t *sort_tmp = at<uint64_t>(aux.p, 256);
    FASTID_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    if ((st = fastid::compare_append(ctx, db, queries_dev, ld_q, n_q, modes_dev, threshold, capacity, hit_q_dev,
                                     hit_r_dev, hit_score_dev, count, s)))
        return st;
    FASTID_CUDA(ctx, launch_hits_finish(count, capacity, hit_q_dev, hit_r_dev, hit_score_dev, hit_count_dev, sort_tmp,
                                        ctx->dev_status, s));
    count_launches(ctx, hits_finish_launches(capacity));
    return FASTID_OK;
}

}  // extern "C"

namespace fastid {

fastid_status check_topk_args(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *q, int64_t ld_q, int64_t n_q,
                              const uint8_t *modes, int32_t k, const void *out_scores, const void *out_idx) {
    fastid_status st = check_query_args(ctx, db, q, ld_q, n_q, modes);
    if (st) return st;
    if (k < 1 || k > FASTID_MAX_K) return fail(ctx, FASTID_EINVAL, "k out of range: %d", k);
    if (n_q > 0 && (!out_scores || !out_idx)) return fail(ctx, FASTID_EINVAL, "output is NULL");
    return FASTID_OK;
}

MainTimer::MainTimer(fastid_ctx *c, cudaStream_t st) : ctx(c), s(st) {
    if (!ctx->profile) return;
    if (ctx->events_used == ctx->events.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return;
        }
        ctx->events.emplace_back(a, b);
    }
    auto &pr = ctx->events[ctx->events_used++];
    cudaEventRecord(pr.first, s);
    e1 = pr.second;
}

void MainTimer::done() {
    if (e1) cudaEventRecord(e1, s);
    e1 = nullptr;
}

int pick_operand(int form, bool has_fp8, bool has_fp4, int64_t n_q, bool slots16) {
    (void)slots16;
    switch (form) {
        case FASTID_FORM_PLAIN:
            return OP_PLAIN;
        case FASTID_FORM_TENSOR_PACKED:
            return OP_FP8_PACKED;
        case FASTID_FORM_TENSOR:
            return has_fp8 ? OP_FP8 : OP_FP8_PACKED;
        case FASTID_FORM_TENSOR_FP4:
            return has_fp4 ? OP_FP4 : OP_FP4_PACKED;
        case FASTID_FORM_TENSOR_FP4_PACKED:
            return OP_FP4_PACKED;
        default:  // AUTO: see AUTO_FP4_PACKED_MAX_Q
            return has_fp4 && n_q > AUTO_FP4_PACKED_MAX_Q ? OP_FP4 : OP_FP4_PACKED;
    }
}

size_t hits_aux_bytes(int64_t capacity) {
    return 256 + (size_t)(2 + hits_sort_elems(capacity) * 3 / 2 + 1) * 8;
}

fastid_status compare_append(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev, int64_t ld_q,
                             int64_t n_q, const uint8_t *modes_dev, uint32_t threshold, int64_t capacity,
                             int64_t *hit_q_dev, int64_t *hit_r_dev, uint32_t *hit_score_dev,
                             unsigned long long *count, cudaStream_t s) {
    int tensor;
    fastid_status st;
    if ((st = pick_form(ctx, db, n_q, &tensor))) return st;
    Scratch scr(ctx, s);
    if (tensor) {
        TensorPrep tp;
        size_t xo;
        if ((st = prepare_tensor(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, EXTRA_NONE, 0, &xo, &tp,
                                 tensor)))
            return st;
        tp.L.epi = EPI_HITS;
        tp.L.threshold = clamp_threshold(threshold, db->n_loci);
        tp.L.k = 1;
        tp.L.capacity = capacity;
        tp.L.hit_q = hit_q_dev;
        tp.L.hit_r = hit_r_dev;
        tp.L.hit_score = hit_score_dev;
        tp.L.hit_count = count;
        MainTimer tm(ctx, s);
        FASTID_CUDA(ctx, launch_tensor_multi(256, tp.L, s));
        tm.done();
        count_launches(ctx, 1);
        return FASTID_OK;
    }
    PreparedQueries pq;
    size_t xo;
    if ((st = prepare(ctx, db, queries_dev, ld_q, n_q, modes_dev, s, scr, 0, &xo, &pq))) return st;
    Partition part = make_partition((int32_t)(pq.n_q_pad / PL_TQ), db->n_pad / PL_TR, ctx->grid_hits);
    MainTimer tm(ctx, s);
    FASTID_CUDA(ctx, launch_plain(EPI_HITS, (const uint32_t *)db->packed, db->norms, db->n_refs, db->ld64 * 2,
                                  db->n_words64 * 2, pq.q32, pq.coef, n_q, threshold, 1, nullptr, 0, capacity,
                                  hit_q_dev, hit_r_dev, hit_score_dev, count, nullptr, part, ctx->dev_status, s));
    tm.done();
    count_launches(ctx, 1);
    return FASTID_OK;
}

int64_t hits_finish_launches(int64_t capacity) {
    if (capacity == 0) return 1;
    int64_t P = hits_sort_elems(capacity), n = 4;  // prep, keys, first smem sort, unpack
    for (int64_t size = 2 * 2048; size <= P; size <<= 1) {
        for (int64_t j = size >> 1; j >= 2048; j >>= 1) ++n;
        ++n;
    }
    return n;
}

}  // namespace fastid
