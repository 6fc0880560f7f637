// Batched top-k over several reference databases ("panels", e.g. loci
// panels of different sizes) in one persistent tensor-form launch.
//
// A plan fixes the panels, the batches (each a set of queries against one
// panel, with its own output buffers), k and the threshold.  Creating it
// allocates and fills every table the launches need; running it enqueues
// three kernels -- operand preparation for every batch row, one persistent
// compare launch that walks the units (panel, 128-query tile, reference tile)
// of all panels, and the merge that writes each batch's results -- with no
// allocation and no host synchronisation, so a run can be captured once into
// a CUDA graph (fastid_plan_capture) and replayed (fastid_plan_replay) with
// new query contents in the same buffers.
//
// Work balance: panels get work groups in proportion to their cost (query
// tiles x reference tiles x K stages) and each panel's groups follow the
// aligned tile-group x reference-slice schedule (TcSched).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace fastid;

struct fastid_plan {
    fastid_ctx *ctx = nullptr;
    int32_t n_panels = 0;
    int32_t bn = 256;
    int32_t variant = FASTID_VARIANT_TENSOR_N256;  // as resolved from AUTO
    int32_t k = 0;
    uint32_t threshold = 0;
    int64_t n_queries = 0;
    int64_t n_jobs_prep = 0;
    int64_t n_jobs_merge = 0;
    int64_t n_ctas = 0;
    TcLaunch launch;
    void *work = nullptr;  // one device allocation for every table and operand
    int64_t work_bytes = 0;
    PrepJob *prep = nullptr;
    MergeJob *merge = nullptr;
    uint64_t *partial = nullptr;
    unsigned int *arrive = nullptr;  // panel-entry counters of the compare launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace {

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

fastid_status perr(fastid_ctx *ctx, fastid_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

fastid_status pcuda(fastid_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();
    return perr(ctx, e == cudaErrorMemoryAllocation ? FASTID_ENOMEM : FASTID_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

void free_plan(fastid_plan *p) {
    if (!p) return;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->work) cudaFree(p->work);
    delete p;
}

}  // namespace

extern "C" {

fastid_status fastid_plan_create(fastid_ctx *ctx, const fastid_refdb *const *dbs, int32_t n_panels,
                                 const fastid_batch *batches, int32_t n_batches, int32_t k, uint32_t threshold,
                                 int32_t variant, fastid_plan **out) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!out) return perr(ctx, FASTID_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dbs || n_panels < 1 || n_panels > TC_MAXP)
        return perr(ctx, FASTID_EINVAL, "n_panels must be in 1..8 with a database per panel");
    if (n_batches < 0 || (n_batches > 0 && !batches)) return perr(ctx, FASTID_EINVAL, "bad batch list");
    if (k < 1 || k > FASTID_MAX_K) return perr(ctx, FASTID_EINVAL, "k out of range");
    if (variant < FASTID_VARIANT_AUTO || variant > FASTID_VARIANT_TENSOR_FP4_PAIR_2SM)
        return perr(ctx, FASTID_EINVAL, "unknown variant");
    bool all_fp8 = true, all_fp4 = true;
    for (int p = 0; p < n_panels; ++p) {
        if (!dbs[p]) return perr(ctx, FASTID_EINVAL, "database is NULL");
        if (dbs[p]->device != ctx->device) return perr(ctx, FASTID_EINVAL, "database belongs to another device");
        all_fp8 = all_fp8 && dbs[p]->fp8;
        all_fp4 = all_fp4 && dbs[p]->fp4;
    }
    if (variant == FASTID_VARIANT_AUTO)  // the FP4 copies when every panel has one, paired when clusters run
        variant = all_fp4 ? (ctx->pair_clusters > 0 ? FASTID_VARIANT_TENSOR_FP4_PAIR : FASTID_VARIANT_TENSOR_FP4)
                          : FASTID_VARIANT_TENSOR_N256;
    const bool f4 = variant == FASTID_VARIANT_TENSOR_FP4 || variant == FASTID_VARIANT_TENSOR_FP4_PAIR ||
                    variant == FASTID_VARIANT_TENSOR_FP4_PAIR_2SM;
    const bool paired = variant == FASTID_VARIANT_TENSOR_PAIR || variant == FASTID_VARIANT_TENSOR_FP4_PAIR ||
                        variant == FASTID_VARIANT_TENSOR_PAIR_2SM || variant == FASTID_VARIANT_TENSOR_FP4_PAIR_2SM;
    if (paired && ctx->pair_clusters < 1)
        return perr(ctx, FASTID_EUNSUPPORTED, "paired launches need 2-CTA clusters");
    if (f4 && !all_fp4)
        return perr(ctx, FASTID_EUNSUPPORTED, "FP4 plan variants read the FP4 copy: load every panel with "
                                              "FASTID_REFS_FP4");
    if (!f4 && !all_fp8)
        return perr(ctx, FASTID_EUNSUPPORTED, "FP8 plan variants read the FP8 copy: load every panel with "
                                              "FASTID_REFS_TENSOR");
    for (int b = 0; b < n_batches; ++b) {
        const fastid_batch &B = batches[b];
        if (B.panel < 0 || B.panel >= n_panels) return perr(ctx, FASTID_EINVAL, "batch panel out of range");
        if (B.n_q < 0 || B.n_q > 0x7fffffffll) return perr(ctx, FASTID_EINVAL, "batch n_q out of range");
        if (B.n_q > 0 && (!B.queries_dev || !B.modes_dev || !B.out_scores_dev || !B.out_idx_dev))
            return perr(ctx, FASTID_EINVAL, "batch buffer is NULL");
        if (B.ld_q < dbs[B.panel]->n_words64) return perr(ctx, FASTID_EINVAL, "batch ld_q too small");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return pcuda(ctx, e, "cudaSetDevice");

    fastid_plan *P = new (std::nothrow) fastid_plan();
    if (!P) return perr(ctx, FASTID_ENOMEM, "host allocation");
    P->ctx = ctx;
    P->n_panels = n_panels;
    P->bn = f4 ? tensor_tile_r4() : variant == FASTID_VARIANT_TENSOR_N128 ? 128 : 256;
    P->variant = variant;
    P->k = k;
    P->threshold = threshold;
    const int BN = P->bn;
    const int pair = paired ? 1 : 0;
    // operand row bytes of each panel (FP8: a byte per locus; FP4: two loci a byte)
    auto kbytes = [&](int p) { return (int64_t)(f4 ? dbs[p]->kbytes4 : dbs[p]->kpad); };
    const int64_t tq = (int64_t)TC_TILE_Q * (pair ? 2 : 1);  // operand rows per tile (pair)

    // Rows of each panel's operand: its batches' queries, in batch order.
    std::vector<int64_t> rows(n_panels, 0);
    for (int b = 0; b < n_batches; ++b) rows[batches[b].panel] += batches[b].n_q;
    std::vector<int64_t> rows_pad(n_panels), n_qq(n_panels), n_rt(n_panels), tile_bytes(n_panels);
    for (int p = 0; p < n_panels; ++p) {
        rows_pad[p] = rup(std::max<int64_t>(rows[p], 1), tq);
        n_qq[p] = rows[p] > 0 ? rows_pad[p] / tq : 0;
        n_rt[p] = (dbs[p]->n_pad + BN - 1) / BN;
        tile_bytes[p] = (int64_t)BN * kbytes(p);
        P->n_queries += rows[p];
    }
    TcLaunch &L = P->launch;
    memset(&L, 0, sizeof L);
    L.pair = pair;
    L.cg2 = variant == FASTID_VARIANT_TENSOR_PAIR_2SM || variant == FASTID_VARIANT_TENSOR_FP4_PAIR_2SM ? 1 : 0;
    L.f4 = f4 ? 1 : 0;
    L.n_groups = make_tensor_schedule(n_panels, n_qq.data(), n_rt.data(), tile_bytes.data(),
                                      pair ? ctx->pair_clusters : ctx->grid_tensor, pair ? 2 : 1, L.sched,
                                      L.order, &L.n_slots);
    if (L.n_groups < 0) {
        free_plan(P);
        if (L.n_groups == -2) return perr(ctx, FASTID_EDEVICE, "schedule self-check failed (debug build)");
        return perr(ctx, FASTID_EINVAL, "plan too large (top-k slots)");
    }
    P->n_ctas = (int64_t)L.n_groups * (pair ? 2 : 1);

    // Workspace layout.
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        size_t at = off;
        off += bytes;
        return at;
    };
    std::vector<size_t> o_a(n_panels), o_qc(n_panels);
    int64_t n_prep = 0;
    for (int p = 0; p < n_panels; ++p) {
        o_a[p] = take((size_t)rows_pad[p] * kbytes(p));
        o_qc[p] = take((size_t)rows_pad[p] * sizeof(float));
        n_prep += rows_pad[p];
    }
    const size_t o_prep = take((size_t)n_prep * sizeof(PrepJob));
    const size_t o_merge = take((size_t)std::max<int64_t>(P->n_queries, 1) * sizeof(MergeJob));
    const size_t o_part = take((size_t)std::max<int32_t>(L.n_slots, 1) * TC_TILE_Q * k * sizeof(uint64_t));
    const size_t o_arrive = take(TC_MAXP * sizeof(unsigned int));
    e = cudaMalloc(&P->work, off);
    if (e != cudaSuccess) {
        free_plan(P);
        return pcuda(ctx, e, "plan workspace");
    }
    P->work_bytes = (int64_t)off;
    uint8_t *W = static_cast<uint8_t *>(P->work);
    P->prep = reinterpret_cast<PrepJob *>(W + o_prep);
    P->merge = reinterpret_cast<MergeJob *>(W + o_merge);
    P->partial = reinterpret_cast<uint64_t *>(W + o_part);
    P->arrive = reinterpret_cast<unsigned int *>(W + o_arrive);

    // Host tables.
    std::vector<PrepJob> prep(n_prep);
    std::vector<MergeJob> merge;
    merge.reserve(P->n_queries);
    {
        std::vector<int64_t> fill(n_panels, 0);
        std::vector<int64_t> prep_base(n_panels, 0);
        for (int p = 1; p < n_panels; ++p) prep_base[p] = prep_base[p - 1] + rows_pad[p - 1];
        for (int p = 0; p < n_panels; ++p)
            for (int64_t r = 0; r < rows_pad[p]; ++r) {
                PrepJob &j = prep[prep_base[p] + r];
                j.src = nullptr;
                j.mode = nullptr;
                j.dst = W + o_a[p] + (size_t)r * kbytes(p);
                j.qc = reinterpret_cast<float *>(W + o_qc[p]) + r;
                j.n_words = dbs[p]->n_words64;
                j.n_loci = dbs[p]->n_loci;
                j.kpad = (int32_t)kbytes(p);
                j.f4 = f4 ? 1 : 0;
            }
        for (int b = 0; b < n_batches; ++b) {
            const fastid_batch &B = batches[b];
            const int p = B.panel;
            for (int64_t i = 0; i < B.n_q; ++i) {
                // the panel's queries, in batch order, spread over its tiles
                const int64_t r = spread_query_to_row(fill[p]++, rows_pad[p] / TC_TILE_Q);
                PrepJob &j = prep[prep_base[p] + r];
                j.src = B.queries_dev + i * B.ld_q;
                j.mode = B.modes_dev + i;
                MergeJob m;
                m.out_s = B.out_scores_dev + i * k;
                m.out_i = B.out_idx_dev + i * k;
                m.panel = p;
                m.q = (int32_t)r;
                merge.push_back(m);
            }
        }
    }
    P->n_jobs_prep = n_prep;
    P->n_jobs_merge = (int64_t)merge.size();
    e = cudaMemcpy(P->prep, prep.data(), prep.size() * sizeof(PrepJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !merge.empty())
        e = cudaMemcpy(P->merge, merge.data(), merge.size() * sizeof(MergeJob), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_plan(P);
        return pcuda(ctx, e, "plan tables");
    }

    // Launch description.
    L.n_panels = n_panels;
    for (int p = 0; p < n_panels; ++p) {
        e = make_operand_map(&L.map_a[p], W + o_a[p], rows_pad[p], (int32_t)kbytes(p), TC_TILE_Q);
        if (e == cudaSuccess)
            e = make_operand_map(&L.map_b[p], f4 ? dbs[p]->fp4 : dbs[p]->fp8, dbs[p]->n_pad, (int32_t)kbytes(p),
                                 pair ? BN / 2 : BN);
        if (e != cudaSuccess) {
            free_plan(P);
            return pcuda(ctx, e, "tensor maps");
        }
        L.n_refs[p] = dbs[p]->n_refs;
        L.n_q[p] = rows[p];
        L.n_rt[p] = n_rt[p];
        L.kpad[p] = (int32_t)kbytes(p);
        L.qconst[p] = reinterpret_cast<const float *>(W + o_qc[p]);
        L.qspread[p] = (int32_t)(rows_pad[p] / TC_TILE_Q);  // see the prep jobs
    }
    L.k = k;
    L.epi = EPI_TOPK;
    L.partial = P->partial;
    L.status = ctx->dev_status;
    int busy = 0;
    for (int p = 0; p < n_panels; ++p) busy += n_qq[p] > 0;
    L.arrive = busy > 1 ? P->arrive : nullptr;
    // Scores never exceed a panel's loci count; clamp so T + 1 stays exact in FP32.
    L.threshold = threshold;
    if (threshold != 0xFFFFFFFFu) {
        int32_t nmax = 0;
        for (int p = 0; p < n_panels; ++p) nmax = std::max(nmax, dbs[p]->n_loci);
        L.threshold = threshold > (uint32_t)nmax ? (uint32_t)nmax : threshold;
    }
    *out = P;
    return FASTID_OK;
}

fastid_status fastid_plan_run(fastid_plan *plan, fastid_stream stream) {
    FASTID_RANGE();
    if (!plan) return FASTID_EINVAL;
    fastid_ctx *ctx = plan->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return pcuda(ctx, e, "cudaSetDevice");
    if (plan->n_queries == 0) return FASTID_OK;
    e = launch_prep_jobs(plan->prep, plan->n_jobs_prep, s);
    if (e != cudaSuccess) return pcuda(ctx, e, "batched operand preparation");
    if (plan->launch.arrive) {
        e = cudaMemsetAsync(plan->launch.arrive, 0, TC_MAXP * sizeof(unsigned int), s);
        if (e != cudaSuccess) return pcuda(ctx, e, "panel counters");
    }
    e = launch_tensor_multi(plan->bn, plan->launch, s);
    if (e != cudaSuccess) return pcuda(ctx, e, "batched compare launch");
    e = launch_merge_sched(plan->partial, plan->launch, plan->merge, plan->n_jobs_merge, nullptr, nullptr, s);
    if (e != cudaSuccess) return pcuda(ctx, e, "batched merge");
    ctx->launches += 3;
    return FASTID_OK;
}

fastid_status fastid_plan_capture(fastid_plan *plan, fastid_stream stream) {
    FASTID_RANGE();
    if (!plan) return FASTID_EINVAL;
    fastid_ctx *ctx = plan->ctx;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return pcuda(ctx, e, "cudaSetDevice");
    if (plan->graph_exec) {
        cudaGraphExecDestroy(plan->graph_exec);
        plan->graph_exec = nullptr;
    }
    if (plan->graph) {
        cudaGraphDestroy(plan->graph);
        plan->graph = nullptr;
    }
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return pcuda(ctx, e, "capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return pcuda(ctx, e, "begin capture");
    }
    const int64_t launches_before = ctx->launches;
    fastid_status st = fastid_plan_run(plan, cs);
    ctx->launches = launches_before;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != FASTID_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return pcuda(ctx, e, "end capture");
    plan->graph = g;
    e = cudaGraphInstantiate(&plan->graph_exec, g, 0);
    if (e != cudaSuccess) return pcuda(ctx, e, "graph instantiate");
    (void)stream;
    return FASTID_OK;
}

fastid_status fastid_plan_replay(fastid_plan *plan, fastid_stream stream) {
    FASTID_RANGE();
    if (!plan) return FASTID_EINVAL;
    fastid_ctx *ctx = plan->ctx;
    if (!plan->graph_exec) return perr(ctx, FASTID_EINVAL, "plan has no captured graph: call fastid_plan_capture");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaGraphLaunch(plan->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return pcuda(ctx, e, "graph launch");
    if (plan->n_queries > 0) ctx->launches += 3;
    return FASTID_OK;
}

fastid_status fastid_plan_info(const fastid_plan *plan, int64_t *n_queries, int64_t *n_units, int32_t *grid,
                               int32_t *variant, int64_t *workspace_bytes) {
    if (!plan) return FASTID_EINVAL;
    if (n_queries) *n_queries = plan->n_queries;
    if (n_units) {
        int64_t u = 0;
        for (int p = 0; p < plan->launch.n_panels; ++p)
            u += (int64_t)plan->launch.sched[p].n_qq * plan->launch.n_rt[p];
        *n_units = u;
    }
    if (grid) *grid = (int32_t)plan->n_ctas;
    if (variant) *variant = plan->variant;
    if (workspace_bytes) *workspace_bytes = plan->work_bytes;
    return FASTID_OK;
}

fastid_status fastid_plan_destroy(fastid_plan *plan) {
    if (!plan) return FASTID_OK;
    cudaSetDevice(plan->ctx->device);
    cudaDeviceSynchronize();
    free_plan(plan);
    return FASTID_OK;
}

}  // extern "C"
