// Reference databases on disk: fastid_save_refs writes a database's packed
// rows behind a small header, fastid_load_refs_file reads them back into a
// new database (building the FP8 copy if asked), so a service restarts from
// the file instead of regenerating or re-packing its references.
//
// File layout (little-endian):
//   bytes  0..7    magic "FASTIDDB"
//   bytes  8..11   format version (1)
//   bytes 12..15   n_loci
//   bytes 16..23   n_refs
//   bytes 24..27   words per row (ceil(n_loci / 64))
//   bytes 28..31   reserved (0)
//   then n_refs rows of `words` uint64, locus l at bit l % 64 of word l / 64
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

using namespace fastid;

namespace {

constexpr char MAGIC[8] = {'F', 'A', 'S', 'T', 'I', 'D', 'D', 'B'};
constexpr uint32_t VERSION = 1;
constexpr int64_t CHUNK_ROWS = 1 << 18;  // rows per host <-> device transfer

struct Header {
    char magic[8];
    uint32_t version;
    int32_t n_loci;
    int64_t n_refs;
    int32_t words;
    uint32_t reserved;
};
static_assert(sizeof(Header) == 32, "file header is 32 bytes");

fastid_status ffail(fastid_ctx *ctx, fastid_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

struct HostBuf {
    void *p = nullptr;
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace

extern "C" {

fastid_status fastid_save_refs(fastid_ctx *ctx, const fastid_refdb *db, const char *path) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!db || !path) return ffail(ctx, FASTID_EINVAL, "database or path is NULL");
    cudaError_t e = cudaSetDevice(db->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the rows are final (any stream)
    if (e != cudaSuccess) return ffail(ctx, FASTID_ECUDA, std::string("device: ") + cudaGetErrorString(e));
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return ffail(ctx, FASTID_EINVAL, std::string("cannot open for writing: ") + path);
    Header h;
    memcpy(h.magic, MAGIC, 8);
    h.version = VERSION;
    h.n_loci = db->n_loci;
    h.n_refs = db->n_refs;
    h.words = db->n_words64;
    h.reserved = 0;
    if (fwrite(&h, sizeof h, 1, out.f) != 1) return ffail(ctx, FASTID_EINVAL, "write failed");
    const int64_t rows = std::min<int64_t>(CHUNK_ROWS, db->n_refs);
    HostBuf buf;
    if ((e = cudaMallocHost(&buf.p, (size_t)rows * db->n_words64 * 8)) != cudaSuccess)
        return ffail(ctx, FASTID_ENOMEM, "pinned buffer");
    // the database's rows sit at stride ld64; the file keeps n_words64 of them
    for (int64_t r0 = 0; r0 < db->n_refs; r0 += rows) {
        const int64_t n = std::min<int64_t>(rows, db->n_refs - r0);
        e = cudaMemcpy2D(buf.p, (size_t)db->n_words64 * 8, db->packed + r0 * db->ld64, (size_t)db->ld64 * 8,
                         (size_t)db->n_words64 * 8, (size_t)n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return ffail(ctx, FASTID_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
        if (fwrite(buf.p, (size_t)db->n_words64 * 8, (size_t)n, out.f) != (size_t)n)
            return ffail(ctx, FASTID_EINVAL, "write failed");
    }
    if (fflush(out.f) != 0) return ffail(ctx, FASTID_EINVAL, "write failed");
    return FASTID_OK;
}

fastid_status fastid_load_refs_file(fastid_ctx *ctx, const char *path, uint32_t flags, fastid_refdb **out,
                                    fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!path || !out) return ffail(ctx, FASTID_EINVAL, "path or out is NULL");
    *out = nullptr;
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return ffail(ctx, FASTID_EINVAL, std::string("cannot open: ") + path);
    Header h;
    if (fread(&h, sizeof h, 1, in.f) != 1 || memcmp(h.magic, MAGIC, 8) != 0)
        return ffail(ctx, FASTID_EINVAL, "not a database file");
    if (h.version != VERSION) return ffail(ctx, FASTID_EINVAL, "unknown database file version");
    if (h.n_loci < 1 || h.n_loci > FASTID_MAX_LOCI || h.n_refs < 1 || h.n_refs > 0x7fffffffll ||
        h.words != (h.n_loci + 63) / 64)
        return ffail(ctx, FASTID_EINVAL, "inconsistent database file header");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return ffail(ctx, FASTID_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    const cudaStream_t s = (cudaStream_t)stream;
    // the rows on the device (as the caller of fastid_load_refs would hold
    // them), then the ordinary load
    uint64_t *dev = nullptr;
    if ((e = cudaMalloc(&dev, (size_t)h.n_refs * h.words * 8)) != cudaSuccess) {
        cudaGetLastError();
        return ffail(ctx, FASTID_ENOMEM, "device buffer for the file's rows");
    }
    const int64_t rows = std::min<int64_t>(CHUNK_ROWS, h.n_refs);
    HostBuf buf;
    fastid_status st = FASTID_OK;
    if ((e = cudaMallocHost(&buf.p, (size_t)rows * h.words * 8)) != cudaSuccess) {
        st = ffail(ctx, FASTID_ENOMEM, "pinned buffer");
    } else {
        for (int64_t r0 = 0; r0 < h.n_refs && st == FASTID_OK; r0 += rows) {
            const int64_t n = std::min<int64_t>(rows, h.n_refs - r0);
            if (fread(buf.p, (size_t)h.words * 8, (size_t)n, in.f) != (size_t)n) {
                st = ffail(ctx, FASTID_EINVAL, "database file is truncated");
            } else if ((e = cudaMemcpyAsync(dev + r0 * h.words, buf.p, (size_t)n * h.words * 8,
                                            cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                       (e = cudaStreamSynchronize(s)) != cudaSuccess) {  // the bounce buffer is reused
                st = ffail(ctx, FASTID_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
            }
        }
    }
    if (st == FASTID_OK) st = fastid_load_refs(ctx, dev, h.n_refs, h.n_loci, h.words, flags, out, stream);
    cudaStreamSynchronize(s);  // the load has read the rows
    cudaFree(dev);
    return st;
}

}  // extern "C"
