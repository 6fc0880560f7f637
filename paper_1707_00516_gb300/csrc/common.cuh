// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastid.h"

namespace fastid {

// Device status word bits (ctx->dev_status[0]); detail in dev_status[1..].
enum : uint32_t {
    ST_OVERFLOW = 1u,  // hit list longer than its capacity
    ST_TIMEOUT = 2u,   // a bounded wait ran out
    ST_DEVICE = 4u,    // a device-side consistency check failed
};

// Plain-form tile: 128 references x 128 queries per CTA, K staged in chunks of
// KC 32-bit words.
constexpr int PL_TR = 128;       // references per tile
constexpr int PL_TQ = 128;       // queries per tile
constexpr int PL_KC = 16;        // u32 words per K stage
constexpr int PL_THREADS = 256;  // 16 x 16 threads, 8 x 8 outputs each
constexpr int ROW_ALIGN = 256;   // database rows are padded to this multiple (both forms' tiles)
constexpr int WORD_ALIGN32 = 32; // database row stride (u32 words) is a multiple of this

// Epilogue kinds of the comparison kernels.
enum Epi : int { EPI_SCORES16 = 0, EPI_SCORES32 = 1, EPI_HITS = 2, EPI_TOPK = 3 };

// Per-query coefficients for the plain form: score = |R| + b - a * G, where
// G = popc(R AND Q):  mode 0 (XOR): a = 2, b = |Q|;  mode 1 (Eq. 1): a = 1, b = 0.
struct QueryCoef {
    uint32_t a;
    uint32_t b;
};

// Work partition of a persistent launch over units = query tiles x reference
// tiles in query-tile-major order; CTA c takes units [c*U/G, (c+1)*U/G).
struct Partition {
    int64_t n_units;   // QT * RT
    int32_t n_qt;      // query tiles
    int64_t n_rt;      // reference tiles
    int32_t grid;      // G
    int32_t max_seg;   // max query-tile segments per CTA
};

__host__ __device__ inline int64_t part_begin(const Partition &p, int64_t c) {
    return (c * p.n_units) / p.grid;
}

__host__ inline Partition make_partition(int32_t n_qt, int64_t n_rt, int32_t grid_target) {
    Partition p;
    p.n_qt = n_qt;
    p.n_rt = n_rt;
    p.n_units = (int64_t)n_qt * n_rt;
    int64_t g = grid_target < 1 ? 1 : grid_target;
    if (g > p.n_units) g = p.n_units;
    if (g < 1) g = 1;
    p.grid = (int32_t)g;
    int64_t span = (p.n_units + g - 1) / g;
    p.max_seg = (int32_t)((span + n_rt - 1) / n_rt + 1);
    return p;
}

// Panels (databases) one tensor-form launch can walk, and the tensor form's
// query-tile height (TMEM lanes).
constexpr int TC_MAXP = 8;
constexpr int TC_TILE_Q = 128;

// Batched form: one operand row to encode (src == nullptr: padding row).
struct PrepJob {
    const uint64_t *src;   // packed query row
    const uint8_t *mode;   // its mode byte
    uint8_t *dst;          // operand row [kpad bytes]: e4m3, or e2m1 when f4
    float *qc;             // its c_q
    int32_t n_words;
    int32_t n_loci;
    int32_t kpad;          // operand row bytes
    int32_t f4;            // 1: FP4 (e2m1) operand
};

// Batched form: one query's merge of per-slot lists into its output row.
struct MergeJob {
    uint32_t *out_s;  // [k]
    int64_t *out_i;   // [k]
    int32_t panel;
    int32_t q;        // row of the panel's query operand
};

// Tensor-form schedule of one panel.  The panel's work groups (CTAs, or
// 2-CTA clusters when paired) form an a x b grid: tile group x owns query
// tiles (pairs) [x tpx, (x+1) tpx), reference slice y owns reference tiles
// [y n_rt / b, (y+1) n_rt / b).  A group walks its slice in chunks of
// `chunk` tiles and, inside a chunk, each of its query tiles in turn, so the
// groups of a slice read the same reference chunk at about the same time (it
// is fetched from DRAM once and served from L2 to the others).  Each (CTA,
// query tile) keeps its running top-k in a slot of the partial buffer, saved
// after every chunk and resumed at the next; the panel's slots start at
// slot0 and CTA c's tile i is slot slot0 + c tpx + i.
// Panels run one after another: every panel's grid is laid over the same
// work groups (group g of panel p is group g of the launch), and each group
// walks its share of every panel in the launch's panel order (largest first),
// so the L2 serves one panel's working set at a time.
struct TcSched {
    int32_t n_qq;   // query tiles, or tile pairs when paired
    int32_t slot0;  // first top-k slot of the panel
    int32_t a, b;   // tile groups x reference slices
    int32_t tpx;    // query tiles (pairs) per tile group
    int32_t chunk;  // reference tiles per chunk
    int32_t pf;     // 1: prefetch the next reference tile into L2 (tpx == 1 only)
    // Tail: groups a*b .. a*b + t_groups - 1 (otherwise idle) take reference
    // tiles [r_main, n_rt) for t_tpx query tiles (pairs) each, in chunks of
    // t_chunk; the a x b grid covers [0, r_main).  t_groups == 0: no tail,
    // r_main == n_rt.
    int32_t r_main;
    int32_t t_groups, t_tpx, t_chunk;
};

// Host-side description of one tensor-form launch over up to TC_MAXP panels.
// Query spreading.  The work of a query tile depends on its queries (a
// mixture under Eq. 1 keeps beating its current k-th best for longer than an
// individual under the mismatch count, and its tile's epilogue competes with
// the MMA issuer for the SM), and callers often pass queries grouped by kind,
// which left whole tiles -- and the groups that own them -- slower than the
// rest.  So a tensor call spreads the input queries over the operand's s tiles
// with stride s: operand row r (tile r / 128, lane r % 128) holds input query
// (r % 128) s + r / 128, and input query q sits at row (q % s) 128 + q / s.
// s <= 1 is the identity.  A bijection on [0, 128 s); rows whose query is
// >= n_q are padding.  (2048 x 20M, top-32: FP4 20.4 -> 18.9 ms, FP8 40.8 ->
// 38.2 ms with the C3 queries, individuals first and mixtures after.)
__host__ __device__ __forceinline__ int64_t spread_row_to_query(int64_t r, int64_t s) {
    return s <= 1 ? r : (r % TC_TILE_Q) * s + r / TC_TILE_Q;
}
__host__ __device__ __forceinline__ int64_t spread_query_to_row(int64_t q, int64_t s) {
    return s <= 1 ? q : (q % s) * TC_TILE_Q + q / s;
}

struct TcLaunch {
    int32_t n_panels;
    int32_t pair;  // 2-CTA clusters sharing reference stages (groups are clusters, tiles are pairs)
    int32_t pk;    // packed references expanded on chip (map_b over the packed rows; FP8 queries at half scale)
    int32_t f4;    // block-scaled FP4 operands (224-reference tiles); else FP8
    int32_t cg2;   // paired launches: one 2-SM MMA per pair (cta_group::2); else multicast stages
    CUtensorMap map_a[TC_MAXP];
    CUtensorMap map_b[TC_MAXP];
    int64_t n_refs[TC_MAXP];
    int64_t n_q[TC_MAXP];
    int64_t n_rt[TC_MAXP];
    int32_t kpad[TC_MAXP];  // operand row bytes (a multiple of 128)
    const float *qconst[TC_MAXP];
    // Query spreading (see spread_row_to_query): the panel's operand tiles
    // (0 or 1: operand row r holds input query r).  Batched plans spread each
    // panel's queries in batch order and give the merge their rows.
    int32_t qspread[TC_MAXP];
    TcSched sched[TC_MAXP];
    int32_t order[TC_MAXP];  // panel order of every group's walk
    int32_t n_groups;  // work groups of the launch: max of a * b over panels
    int32_t n_slots;   // top-k slots over all panels
    uint32_t threshold;
    int32_t k;
    int32_t epi;
    void *out;
    int64_t ld_out;
    int64_t capacity;
    int64_t *hit_q;
    int64_t *hit_r;
    uint32_t *hit_score;
    unsigned long long *hit_count;
    uint64_t *partial;  // EPI_TOPK: [n_slots][k][128]
    uint32_t *status;
    // Panel-entry counters, one per position of the panel order (zero before
    // the launch), or nullptr: see the rendezvous in the tensor kernel.
    unsigned int *arrive;
};

// Fills sched[] and order[] for n panels, each over (up to) G work groups of
// `ctas_per_group` CTAs; returns the number of groups the launch needs (max
// of a * b + t_groups; -1: too many top-k slots; -2, debug builds only: the
// schedule's self-check failed) and sets *n_slots.  tile_bytes: bytes of one
// reference tile of the operand.
int32_t make_tensor_schedule(int n, const int64_t *n_qq, const int64_t *n_rt, const int64_t *tile_bytes,
                             int32_t G, int32_t ctas_per_group, TcSched *sched, int32_t *order,
                             int32_t *n_slots);

// Top-k keys: (score << 32) | ref, so that ordering keys orders by score then
// by reference index.  An empty slot holds KEY_EMPTY.
constexpr uint64_t KEY_EMPTY = ~0ull;

__host__ __device__ inline uint64_t make_key(uint32_t score, uint32_t ref) {
    return ((uint64_t)score << 32) | ref;
}

// Initial cutoff: keys strictly below it may enter a list that is not full.
__host__ __device__ inline uint64_t initial_cut(uint32_t threshold) {
    return threshold == 0xFFFFFFFFu ? KEY_EMPTY : ((uint64_t)(threshold + 1u) << 32);
}

}  // namespace fastid

// Launchers implemented in the .cu files (all enqueue on `s`, no sync).
namespace fastid {
cudaError_t launch_pack(const uint8_t *alleles, int64_t n, int32_t n_loci, int64_t ld_alleles,
                        uint64_t *packed, int64_t ld_words, uint32_t *norms, cudaStream_t s);
cudaError_t launch_mix(const uint64_t *src, int64_t ld_src, int32_t n_words, const int32_t *offsets,
                       int64_t n_mix, uint64_t *out, int64_t ld_out, uint32_t *norms,
                       cudaStream_t s);
cudaError_t launch_copy_rows(const uint64_t *src, int64_t n, int64_t ld_src, int32_t n_words,
                             uint64_t *dst, int64_t n_pad, int64_t ld_dst, uint32_t *norms,
                             cudaStream_t s);
cudaError_t launch_query_prep(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words,
                              const uint8_t *modes, uint32_t *q32, int64_t n_q_pad, int64_t ld32,
                              QueryCoef *coef, cudaStream_t s);
cudaError_t launch_plain(int epi, const uint32_t *refs32, const uint32_t *ref_norms, int64_t n_refs,
                         int64_t ld32, int32_t k_words32, const uint32_t *q32,
                         const QueryCoef *coef, int64_t n_q, uint32_t threshold, int32_t k,
                         void *out, int64_t ld_out, int64_t capacity, int64_t *hit_q,
                         int64_t *hit_r, uint32_t *hit_score, unsigned long long *hit_count,
                         uint64_t *partial, const Partition &part, uint32_t *status,
                         cudaStream_t s);
int plain_grid_target(int epi, int device);
cudaError_t launch_topk_merge(const uint64_t *partial, const Partition &part, int64_t n_q,
                              int32_t k, uint32_t *out_scores, int64_t *out_idx, cudaStream_t s);
cudaError_t launch_topk_merge_tile(const uint64_t *partial, const Partition &part, int32_t tile_q, int32_t pair,
                                   int64_t n_q, int32_t k, uint32_t *out_scores, int64_t *out_idx, cudaStream_t s);
int64_t hits_sort_elems(int64_t capacity);
// tensor form (tensor.cu)
cudaError_t make_operand_map(CUtensorMap *map, const uint8_t *base, int64_t rows, int32_t kpad, int box_rows);
int tensor_tile_q();
int tensor_tile_r();
int tensor_kpad(int32_t n_loci);
int tensor_grid_target(int device);
int tensor_pair_clusters(int device);
// FP8 reference operand [n_rows][kpad] from packed rows (n_src rows of n_words
// words exist at stride ld64; zero elsewhere), on at most max_blocks CTAs.
cudaError_t launch_refs_e4m3(const uint64_t *packed, int64_t ld64, int64_t n_src, int32_t n_words, int64_t n_rows,
                             int32_t kpad, uint8_t *out, int max_blocks, cudaStream_t s);
cudaError_t launch_queries_e4m3(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words, int32_t n_loci,
                                const uint8_t *modes, int64_t n_q_pad, int32_t kpad, uint8_t *out, float *qconst,
                                bool half, int64_t spread, cudaStream_t s);
// TMA map over packed rows for packed-reference (PK) launches: boxes of 2
// words x 256 rows (FP8 stages) or 4 words x 224 rows (FP4 stages).
cudaError_t make_packed_map(CUtensorMap *map, const uint64_t *packed, int64_t rows, int64_t ld64, int box_words = 2,
                            int box_rows = 256);
// FP4 form: reference tile (224), operand row bytes of n_loci (loci padded to
// 256, two per byte), the database's FP4 copy and the query operand.
int tensor_tile_r4();
int tensor_kbytes4(int32_t n_loci);
cudaError_t launch_refs_e2m1(const uint64_t *packed, int64_t ld64, int64_t n_src, int32_t n_words, int64_t n_rows,
                             int32_t kbytes, uint8_t *out, int max_blocks, cudaStream_t s);
cudaError_t launch_queries_e2m1(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words, int32_t n_loci,
                                const uint8_t *modes, int64_t n_q_pad, int32_t kbytes, uint8_t *out, float *qconst,
                                int64_t spread, cudaStream_t s);

cudaError_t launch_tensor_multi(int bn, const TcLaunch &L, cudaStream_t s);
cudaError_t launch_prep_jobs(const PrepJob *jobs, int64_t n_jobs, cudaStream_t s);
// snap[0..3] = status[0..3], status cleared, atomically per word (diag.cu).
cudaError_t launch_status_take(uint32_t *status, uint32_t *snap, cudaStream_t s);
// Merge of per-slot lists for the queries of a tensor launch (jobs == nullptr:
// one panel, query q's output is out_scores/out_idx row q).  accumulate:
// merge into the output lists (reference indices + ref_offset) instead of
// overwriting them.
cudaError_t launch_merge_sched(const uint64_t *partial, const TcLaunch &L, const MergeJob *jobs, int64_t n_jobs,
                               uint32_t *out_scores, int64_t *out_idx, cudaStream_t s, bool accumulate = false,
                               int64_t ref_offset = 0);
// Fold one streamed block's [n_q][k] lists (indices + offset) into the
// running [n_q][k] lists.
cudaError_t launch_topk_fold(uint32_t *run_s, int64_t *run_i, const uint32_t *blk_s, const int64_t *blk_i,
                             int64_t offset, int64_t n_q, int32_t k, cudaStream_t s);
cudaError_t launch_hits_finish(unsigned long long *count, int64_t capacity, int64_t *hit_q,
                               int64_t *hit_r, uint32_t *hit_score, int64_t *count_out,
                               uint64_t *sort_tmp, uint32_t *status, cudaStream_t s);
}  // namespace fastid
