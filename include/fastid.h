/*
 * fastid.h -- C ABI of the GB300 FastID all-pairs comparison library.
 *
 * Method: Samsi et al., "A Linear Algebra Approach to Fast DNA Mixture
 * Analysis Using GPUs" (arXiv:1707.00516).  Every unknown profile Q_q is
 * compared with every known (reference) profile R_r over N SNP loci, as an
 * overloaded matrix multiply (Sec. II-B), giving one of two integer scores per
 * pair (Sec. II-A):
 *
 *   mode 0  FASTID_MODE_MISMATCH     popcount(R_r XOR Q_q)
 *                                    (every minor-allele difference; used to
 *                                    compare two individuals)
 *   mode 1  FASTID_MODE_UNEXPLAINED  popcount(AND(XOR(R_r, Q_q), R_r))
 *                                    = popcount(R_r AND NOT Q_q)      (Eq. 1;
 *                                    reference alleles the query -- usually a
 *                                    mixture -- does not explain)
 *
 * The score matrix is reduced on the device (the reduction Sec. IV proposes):
 * per-query top-k (fastid_topk) or the list of pairs under a threshold
 * (fastid_compare).  fastid_scores writes the full matrix for small problems.
 *
 * Conventions shared by every call:
 *  - Profiles are packed bit vectors: locus l is bit (l mod 64) of 64-bit word
 *    l / 64, least significant bit first (Sec. II-A's conversion to unsigned
 *    words; the bit order is this library's reading).  A row has ld_words >=
 *    ceil(N / 64) words; bits at loci >= N must be zero.
 *  - "_dev" pointers are device memory of the context's device, owned by the
 *    caller.  fastid_ctx and fastid_refdb are owned by the library.
 *  - Every call is asynchronous on the given stream (a cudaStream_t; NULL is
 *    the legacy default stream) and performs no host synchronisation, except
 *    fastid_sync_status and fastid_destroy / fastid_free_refs (which
 *    synchronise the device before freeing).
 *  - Argument errors are returned synchronously (FASTID_EINVAL,
 *    FASTID_EUNSUPPORTED) and nothing is enqueued.  Conditions found on the
 *    device (hit-list overflow, a bounded wait that ran out) are recorded in
 *    the context's status word and returned by fastid_sync_status.
 *  - fastid_last_error returns a message for the last failing call of the
 *    context (thread-local to the context, not to the caller).
 *  - A context may be used from one host thread at a time.  Calls on
 *    different streams may overlap on the device; each call uses its own
 *    scratch memory, allocated stream-ordered on its stream.
 */
#ifndef FASTID_H
#define FASTID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fastid_ctx fastid_ctx;
typedef struct fastid_refdb fastid_refdb;
typedef void *fastid_stream; /* cudaStream_t */

typedef enum {
    FASTID_OK = 0,
    FASTID_EINVAL = 1,       /* bad argument                                   */
    FASTID_ENOMEM = 2,       /* device or host allocation failed               */
    FASTID_ECUDA = 3,        /* a CUDA runtime/driver call failed              */
    FASTID_EOVERFLOW = 4,    /* hit list longer than its capacity              */
    FASTID_ETIMEOUT = 5,     /* a bounded device-side wait ran out             */
    FASTID_EUNSUPPORTED = 6, /* valid request the library or device cannot serve */
    FASTID_EDEVICE = 7       /* a device-side consistency check failed         */
} fastid_status;

enum { FASTID_MODE_MISMATCH = 0, FASTID_MODE_UNEXPLAINED = 1 };

/* Compute form used by the comparison calls. */
enum {
    FASTID_FORM_AUTO = 0,          /* see below                                              */
    FASTID_FORM_PLAIN = 1,         /* packed words, AND + POPC on the integer pipes          */
    FASTID_FORM_TENSOR = 2,        /* 0/1 and +-1 operands in FP8 e4m3 on tcgen05, FP32 accum,
                                      the reference operand read from the database's FP8 copy
                                      (FASTID_REFS_TENSOR), else from its packed rows      */
    FASTID_FORM_TENSOR_PACKED = 3, /* the tensor form with the reference operand always read
                                      as packed bits and expanded to FP8 on chip (1/8 of the
                                      bytes; no FP8 copy needed)                          */
    FASTID_FORM_TENSOR_FP4 = 4,    /* 0/1 and +-1 operands as block-scaled FP4 (e2m1 with unit
                                      scale factors, tcgen05 kind::mxf4), FP32 accum: twice
                                      the FP8 rate per clock; the reference operand read from
                                      the database's FP4 copy (FASTID_REFS_FP4), else from its
                                      packed rows expanded to FP4 on chip                 */
    FASTID_FORM_TENSOR_FP4_PACKED = 5 /* the FP4 tensor form with the reference operand always
                                      read as packed bits and expanded on chip            */
};
/* FASTID_FORM_AUTO: the FP4 tensor form; its reference operand is the FP4 copy
 * when the database has one and the call has more than 128 queries (one query
 * tile), else the packed rows expanded on chip.  (Measured on GB300, the FP4
 * packed rows are never slower than either FP8 operand.) */

/* fastid_load_refs flags */
enum {
    FASTID_REFS_TENSOR = 1u, /* also build the FP8 operand copy used by the tensor form  */
    FASTID_REFS_FP4 = 2u     /* also build the FP4 operand copy (half a byte per locus)  */
};

#define FASTID_MAX_K 32          /* largest k accepted by fastid_topk          */
#define FASTID_MAX_LOCI 65536    /* largest N accepted                         */

/* ---------------------------------------------------------------- context */

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
int32_t fastid_version(void);

/* Human-readable name of a status code (static storage). */
const char *fastid_status_string(fastid_status s);

/* Create a context on CUDA device `device` (makes it current for the calling
 * thread).  *out receives the context.  Errors: EINVAL (out NULL, bad
 * device), ECUDA, ENOMEM. */
fastid_status fastid_create(fastid_ctx **out, int32_t device);

/* Synchronise the device and free the context.  NULL is accepted. */
fastid_status fastid_destroy(fastid_ctx *ctx);

/* Message describing the last failure on ctx ("" if none). */
const char *fastid_last_error(const fastid_ctx *ctx);

/* Device memory the context's calls take: the number of stream-ordered
 * scratch allocations made from its memory pool since creation, and the
 * pool's bytes in use and reserved now (any output may be NULL).  A
 * diagnostic: it shows, for instance, that fastid_topk_noalloc takes none.
 * Errors: EINVAL, ECUDA. */
fastid_status fastid_memory_info(fastid_ctx *ctx, int64_t *pool_allocs, int64_t *pool_used_bytes,
                                 int64_t *pool_reserved_bytes);

/* Choose the compute form for later comparison calls (FASTID_FORM_*). */
fastid_status fastid_set_form(fastid_ctx *ctx, int32_t form);

/* Synchronise `stream`, read and clear the context's device status word (one
 * atomic read-and-clear on the device, ordered on `stream`, so a condition
 * recorded meanwhile by a kernel on another stream is kept for the next call).
 * Returns FASTID_OK, FASTID_EOVERFLOW, FASTID_ETIMEOUT or FASTID_EDEVICE
 * (the most severe condition recorded since the last call), or ECUDA. */
fastid_status fastid_sync_status(fastid_ctx *ctx, fastid_stream stream);

/* Kernel timing and launch counting (off by default).  While enabled, each
 * comparison call records CUDA events around its main compare kernel on the
 * call's stream, and every kernel the library launches is counted.
 * fastid_profile_read synchronises those events, returns the summed duration
 * of the main kernels (ms), the number of main-kernel launches and the total
 * number of kernels launched since the last reset (any output may be NULL),
 * and with reset != 0 clears the counters. */
fastid_status fastid_profile(fastid_ctx *ctx, int32_t enable);
fastid_status fastid_profile_read(fastid_ctx *ctx, double *main_ms, int64_t *main_launches,
                                  int64_t *all_launches, int32_t reset);

/* ------------------------------------------------------------- profiles */

/*
 * Pack 0/1 alleles into bit vectors (Sec. II-A; conversion of alleles to an
 * array of unsigned integers, 512 SNPs -> 16 uint32 = 8 uint64 words).
 *  alleles_dev  uint8 [n][ld_alleles]; entry (i, l) for l < n_loci is the
 *               allele indicator of locus l (any nonzero byte counts as 1).
 *  packed_dev   uint64 [n][ld_words], ld_words >= ceil(n_loci / 64); bits at
 *               loci >= n_loci and words >= ceil(n_loci / 64) are written 0.
 *  norms_dev    optional uint32 [n]: popcount of each packed row.
 * Errors: EINVAL on NULL buffers, n < 0, n_loci outside [1, FASTID_MAX_LOCI],
 * ld_alleles < n_loci or ld_words too small.
 */
fastid_status fastid_pack(fastid_ctx *ctx, const uint8_t *alleles_dev, int64_t n, int32_t n_loci,
                          int64_t ld_alleles, uint64_t *packed_dev, int64_t ld_words,
                          uint32_t *norms_dev, fastid_stream stream);

/*
 * Build mixtures: out[m] = OR of src rows offsets[m] .. offsets[m+1]-1 (a
 * mixture carries every minor allele of its contributors, Sec. I and II-A).
 * An individual is a group of one row.
 *  src_dev      uint64 [*][ld_src] packed rows.
 *  offsets_dev  int32 [n_mix + 1], non-decreasing, offsets[0] >= 0; rows
 *               offsets[m] .. offsets[m+1]-1 must exist in src.  An empty group
 *               gives an all-zero profile.
 *  out_dev      uint64 [n_mix][ld_out]; words >= n_words are written 0.
 *  norms_dev    optional uint32 [n_mix] popcounts of the mixtures.
 * Offsets are read on the device and are not validated on the host.
 */
fastid_status fastid_mix(fastid_ctx *ctx, const uint64_t *src_dev, int64_t ld_src, int32_t n_words,
                         const int32_t *offsets_dev, int64_t n_mix, uint64_t *out_dev,
                         int64_t ld_out, uint32_t *norms_dev, fastid_stream stream);

/* ------------------------------------------------------ reference database */

/*
 * Copy n_refs packed reference profiles into a device-resident database
 * owned by the library (the known profiles of Sec. II-B, matrix A), compute
 * their popcounts, with FASTID_REFS_TENSOR also build the FP8 operand copy
 * (1 byte per locus) used by the tensor form, and with FASTID_REFS_FP4 the FP4
 * operand copy (loci padded to 256, half a byte each) used by
 * FASTID_FORM_TENSOR_FP4.  The caller's buffer may be
 * freed once the stream has passed this call.
 *  packed_dev  uint64 [n_refs][ld_words], bits at loci >= n_loci zero.
 *  n_refs      1 .. 2^31 - 1;  n_loci 1 .. FASTID_MAX_LOCI.
 * Errors: EINVAL, ENOMEM (database does not fit), ECUDA.
 */
fastid_status fastid_load_refs(fastid_ctx *ctx, const uint64_t *packed_dev, int64_t n_refs,
                               int32_t n_loci, int64_t ld_words, uint32_t flags,
                               fastid_refdb **out, fastid_stream stream);

/*
 * Write a database's packed rows to a file (a 32-byte header -- magic
 * "FASTIDDB", version, N, row count, words per row -- then the rows, locus l
 * at bit l % 64 of word l / 64), after synchronising the device.  A database
 * file is the restart point of a service: fastid_load_refs_file reads it back
 * into a new database, with its FP8 copy if flags asks for one.
 * Errors: EINVAL (I/O, or a file that is not a consistent database file),
 * ENOMEM, ECUDA.
 */
fastid_status fastid_save_refs(fastid_ctx *ctx, const fastid_refdb *db, const char *path);
fastid_status fastid_load_refs_file(fastid_ctx *ctx, const char *path, uint32_t flags,
                                    fastid_refdb **out, fastid_stream stream);

/* Synchronise the device and free a database.  NULL is accepted.  For a view
 * (fastid_refs_view) only the handle is freed. */
fastid_status fastid_free_refs(fastid_ctx *ctx, fastid_refdb *db);

/*
 * A database handle over rows [r_begin, r_begin + n_refs) of db, sharing db's
 * memory (nothing is copied or allocated on the device): every comparison
 * call on the view sees those references as indices 0 .. n_refs - 1, with
 * the operand copies db has.  Together with fastid_topk_fold this splits one
 * pass over a database into parts that may run in any order (the paper's
 * blocked comparison of known profiles, Sec. III-C, over resident blocks);
 * the serving layer uses it to let query batches join a running pass at any
 * part boundary.  r_begin must be a multiple of FASTID_VIEW_ALIGN.  Free the
 * view (fastid_free_refs) before db; db's rows must not change meanwhile.
 * Errors: EINVAL (range, alignment, NULL), ENOMEM (host), ECUDA.
 */
#define FASTID_VIEW_ALIGN 256
fastid_status fastid_refs_view(fastid_ctx *ctx, const fastid_refdb *db, int64_t r_begin, int64_t n_refs,
                               fastid_refdb **out);

/* Shape and footprint of a database; any output pointer may be NULL. */
fastid_status fastid_refs_info(const fastid_refdb *db, int64_t *n_refs, int32_t *n_loci,
                               uint32_t *flags, int64_t *device_bytes);

/* ---------------------------------------------------------- comparisons */
/*
 * Shared arguments:
 *  queries_dev  uint64 [n_q][ld_q] packed unknown profiles (matrix B of
 *               Sec. II-B, one row per unknown), same n_loci as the database.
 *  modes_dev    uint8 [n_q]: FASTID_MODE_MISMATCH or FASTID_MODE_UNEXPLAINED
 *               per query (any other value is treated as UNEXPLAINED).
 *  n_q          0 .. 2^31 - 1 (0 is a no-op).
 */

/*
 * Full score matrix (Algorithm 2's P_QR): out[q * ld_out + r] for r < n_refs.
 *  out_bytes  2 (uint16, needs n_loci <= 65535) or 4 (uint32);  ld_out >= n_refs.
 * Intended for small problems: it writes n_q * n_refs scores.
 */
fastid_status fastid_scores(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev,
                            int64_t ld_q, int64_t n_q, const uint8_t *modes_dev, void *out_dev,
                            int32_t out_bytes, int64_t ld_out, fastid_stream stream);

/*
 * Per-query top-k: the k smallest (score, reference index) pairs with
 * score <= threshold, ascending by score then by index (ties are broken by
 * the lower reference index, so the result does not depend on scheduling).
 * Unused slots get (0xFFFFFFFF, -1).  threshold 0xFFFFFFFF means none.
 *  k                1 .. FASTID_MAX_K.
 *  out_scores_dev   uint32 [n_q][k];  out_idx_dev  int64 [n_q][k].
 * The score matrix is never written to memory.
 */
fastid_status fastid_topk(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev,
                          int64_t ld_q, int64_t n_q, const uint8_t *modes_dev, int32_t k,
                          uint32_t threshold, uint32_t *out_scores_dev, int64_t *out_idx_dev,
                          fastid_stream stream);

/*
 * Hit list: every pair with score <= threshold, sorted by (q, r).
 *  hit_q_dev, hit_r_dev  int64 [capacity];  hit_score_dev  uint32 [capacity].
 *  hit_count_dev         int64 [1]: receives the true number of hits.
 * If the count exceeds capacity, the buffers hold `capacity` valid hits (not a
 * defined subset, sorted by (q, r)) and the next fastid_sync_status returns
 * FASTID_EOVERFLOW.  capacity may be 0 (count only).
 */
fastid_status fastid_compare(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev,
                             int64_t ld_q, int64_t n_q, const uint8_t *modes_dev,
                             uint32_t threshold, int64_t capacity, int64_t *hit_q_dev,
                             int64_t *hit_r_dev, uint32_t *hit_score_dev, int64_t *hit_count_dev,
                             fastid_stream stream);

/*
 * fastid_topk over a reference set that stays in HOST memory: the known
 * profiles are copied to the device block by block, each block is compared
 * against all queries and its top-k is folded into the running result.  This
 * is the blocked transfer of Sec. III-C ("Comparing Large Numbers of DNA
 * Mixtures": all unknowns resident, known profiles sent in blocks), for
 * databases larger than device memory; unlike the paper's scheme, block
 * i + 1's host-to-device copy runs on a second stream while block i is
 * compared, and only the k-lists (never the score block) stay on the device.
 * Results are identical to fastid_topk on the same references loaded whole.
 *  refs_host   uint64 [n_refs][ld_words] packed references in host memory,
 *              bits at loci >= n_loci zero.  Page-locked memory (cudaHostAlloc
 *              or cudaHostRegister) lets the copies overlap the comparisons;
 *              pageable memory works but serialises them.  It must stay valid
 *              and unchanged until the stream has passed this call.
 *  n_refs      1 .. 2^31 - 1;  flags: 0 or FASTID_REFS_TENSOR (expand each
 *              block to the FP8 operand, which FASTID_FORM_TENSOR then reads).
 *              Every other case reads each block's packed rows in the
 *              context's form: plain, or FP8 or FP4 expanded on chip
 *              (FASTID_FORM_AUTO: FP4).
 *  block_refs  largest block (>= 1; the first blocks are smaller, from
 *              block_refs / 8 doubling, so that the first comparison starts
 *              early).  Two blocks are on the device at once, each holding
 *              ceil(n_loci / 64) x 8 bytes per reference as copied plus, for
 *              the tensor form, its FP8 operand (n_loci rounded up to 128
 *              bytes per reference) or, for the plain form, padded rows and
 *              popcounts.
 *  The other arguments are those of fastid_topk.  Stream-ordered: the call
 *  enqueues the copies and kernels and returns without waiting for them.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
fastid_status fastid_topk_streamed(fastid_ctx *ctx, const uint64_t *refs_host, int64_t n_refs,
                                   int32_t n_loci, int64_t ld_words, uint32_t flags,
                                   int64_t block_refs, const uint64_t *queries_dev, int64_t ld_q,
                                   int64_t n_q, const uint8_t *modes_dev, int32_t k,
                                   uint32_t threshold, uint32_t *out_scores_dev,
                                   int64_t *out_idx_dev, fastid_stream stream);

/*
 * fastid_compare over a reference set in HOST memory: the hit list of
 * fastid_compare (every (q, r) with score <= threshold, sorted by (q, r), r the
 * index in refs_host), computed block by block as in fastid_topk_streamed.
 * Each block's hits are appended to the output buffers, their reference
 * indices made global, and the whole list is sorted once at the end.  The
 * reference arguments are those of fastid_topk_streamed, the others those of
 * fastid_compare (same overflow behaviour: hit_count receives the true count,
 * and FASTID_EOVERFLOW is reported by the next fastid_sync_status).
 */
fastid_status fastid_compare_streamed(fastid_ctx *ctx, const uint64_t *refs_host, int64_t n_refs,
                                      int32_t n_loci, int64_t ld_words, uint32_t flags,
                                      int64_t block_refs, const uint64_t *queries_dev, int64_t ld_q,
                                      int64_t n_q, const uint8_t *modes_dev, uint32_t threshold,
                                      int64_t capacity, int64_t *hit_q_dev, int64_t *hit_r_dev,
                                      uint32_t *hit_score_dev, int64_t *hit_count_dev,
                                      fastid_stream stream);

/*
 * Merge top-k lists of part of the references into running lists: for each
 * query q, run[q] becomes the k smallest (score, reference index) pairs of
 * run[q] and blk[q], blk's indices taken + ref_offset, ascending by score then
 * index; empty slots are (0xFFFFFFFF, -1) on input and output.  With views
 * over disjoint row ranges (fastid_refs_view) this reassembles fastid_topk
 * over the union from its parts, in any order, exactly.
 *  run_scores_dev  uint32 [n_q][k], run_idx_dev  int64 [n_q][k]  (in/out; an
 *                  all-empty list is every byte 0xFF)
 *  blk_scores_dev  uint32 [n_q][k], blk_idx_dev  int64 [n_q][k]  (as written
 *                  by fastid_topk with the same k)
 *  ref_offset      0 .. 2^31 - 1;  k 1 .. FASTID_MAX_K.
 * Errors: EINVAL, ECUDA.
 */
fastid_status fastid_topk_fold(fastid_ctx *ctx, uint32_t *run_scores_dev, int64_t *run_idx_dev,
                               const uint32_t *blk_scores_dev, const int64_t *blk_idx_dev, int64_t ref_offset,
                               int64_t n_q, int32_t k, fastid_stream stream);

/*
 * fastid_topk merged into running lists instead of written: for each query
 * q, run[q] becomes the k smallest (score, reference index) pairs of run[q]
 * and of this call's top-k against db, this call's indices taken + ref_offset
 * (fastid_topk then fastid_topk_fold in one call, without the intermediate
 * lists).  A pass over a database split into views (fastid_refs_view) is
 * this call once per view, in any order, into the same lists.
 *  ref_offset  0 .. 2^31 - 1 - db's reference count.
 *  run_scores_dev uint32 [n_q][k], run_idx_dev int64 [n_q][k]: in/out, empty
 *              slots (0xFFFFFFFF, -1) (an all-empty list is every byte 0xFF).
 *  The other arguments are fastid_topk's.  Errors: EINVAL, ENOMEM, ECUDA.
 */
fastid_status fastid_topk_accumulate(fastid_ctx *ctx, const fastid_refdb *db, int64_t ref_offset,
                                     const uint64_t *queries_dev, int64_t ld_q, int64_t n_q,
                                     const uint8_t *modes_dev, int32_t k, uint32_t threshold,
                                     uint32_t *run_scores_dev, int64_t *run_idx_dev, fastid_stream stream);

/* ------------------------------------------------------------- diagnostics */
/*
 * The library's bounded device wait, on a flag the caller owns: a one-thread
 * kernel waits until *flag_dev (uint32, device memory) is nonzero, for at
 * most wait_ms milliseconds (1 .. 10000).  If the limit runs out it records a
 * timeout in the context's status word -- the next fastid_sync_status returns
 * FASTID_ETIMEOUT -- exactly as the compare kernels do when one of their
 * pipeline waits runs out, and the context stays usable.  For testing the
 * failure path without faulting a GPU.  Errors: EINVAL, ECUDA.
 */
fastid_status fastid_wait_flag(fastid_ctx *ctx, const uint32_t *flag_dev, int32_t wait_ms,
                               fastid_stream stream);

/* ------------------------------------------------- batched persistent plans */
/*
 * Many query batches of uneven size against several reference databases
 * ("panels", e.g. loci panels of different N) in ONE persistent tensor-form
 * launch: the per-query top-k of fastid_topk for every batch.  (Batching is
 * not in the paper; it applies Eq. 1 / the XOR count exactly as fastid_topk.)
 *
 * A plan fixes panels, batches, k and threshold and owns all scratch memory,
 * so fastid_plan_run allocates nothing and never synchronises: it enqueues an
 * operand-preparation kernel, the persistent compare kernel over the units
 * (panel, 128-query tile, reference tile) of all panels -- each panel spread
 * over every work group, panels taken one after another, largest first --
 * and a merge kernel that writes each batch's outputs.  fastid_plan_capture records one run into a CUDA graph;
 * fastid_plan_replay launches that graph.  Between runs the caller may change
 * the contents (not the addresses or sizes) of the batch buffers.
 *
 * FP8 variants need every panel loaded with FASTID_REFS_TENSOR, FP4 variants
 * with FASTID_REFS_FP4 (EUNSUPPORTED otherwise); at most 8 panels.
 * Batch queries use the packed layout of fastid_topk; out_scores/out_idx are
 * [n_q][k] as in fastid_topk.  variant picks the operand encoding and the
 * reference-tile shape of the compare kernel (FASTID_VARIANT_*; the autotuner
 * in the Python package chooses it per workload).  fastid_plan_info reports
 * the variant AUTO resolved to.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA.
 */
typedef struct fastid_plan fastid_plan;

typedef struct {
    int32_t panel;               /* index into the plan's databases            */
    const uint64_t *queries_dev; /* [n_q][ld_q] packed queries                 */
    int64_t ld_q;
    int64_t n_q;                 /* 0 allowed                                  */
    const uint8_t *modes_dev;    /* [n_q] FASTID_MODE_*                        */
    uint32_t *out_scores_dev;    /* [n_q][k]                                   */
    int64_t *out_idx_dev;        /* [n_q][k]                                   */
} fastid_batch;

enum {
    FASTID_VARIANT_AUTO = 0,        /* FP4_PAIR when every panel has its FP4 copy,
                                       else N256                               */
    FASTID_VARIANT_TENSOR_N256 = 1, /* FP8, 128 x 256 tiles, 4-stage pipeline  */
    FASTID_VARIANT_TENSOR_N128 = 2, /* FP8, 128 x 128 tiles, 6-stage pipeline  */
    FASTID_VARIANT_TENSOR_PAIR = 3, /* FP8, 2-CTA clusters on tile pairs sharing reference stages */
    FASTID_VARIANT_TENSOR_FP4 = 4,  /* FP4 (block-scaled e2m1), 128 x 224 tiles, 5-stage pipeline */
    FASTID_VARIANT_TENSOR_FP4_PAIR = 5, /* FP4, 2-CTA clusters on tile pairs                    */
    FASTID_VARIANT_TENSOR_PAIR_2SM = 6, /* FP8 tile pairs as one 2-SM MMA (tcgen05 cta_group::2,
                                           M = 256): each CTA holds half of every reference
                                           stage, 7 stages                                    */
    FASTID_VARIANT_TENSOR_FP4_PAIR_2SM = 7 /* FP4 tile pairs as one 2-SM MMA                   */
};

fastid_status fastid_plan_create(fastid_ctx *ctx, const fastid_refdb *const *dbs, int32_t n_panels,
                                 const fastid_batch *batches, int32_t n_batches, int32_t k,
                                 uint32_t threshold, int32_t variant, fastid_plan **out);
fastid_status fastid_plan_run(fastid_plan *plan, fastid_stream stream);
fastid_status fastid_plan_capture(fastid_plan *plan, fastid_stream stream);
fastid_status fastid_plan_replay(fastid_plan *plan, fastid_stream stream);
fastid_status fastid_plan_info(const fastid_plan *plan, int64_t *n_queries, int64_t *n_units, int32_t *grid,
                               int32_t *variant, int64_t *workspace_bytes);
/* Synchronises the device and frees the plan.  NULL is accepted. */
fastid_status fastid_plan_destroy(fastid_plan *plan);

/*
 * fastid_topk_noalloc -- fastid_topk for callers that cannot allocate device
 * memory.  The paper has no counterpart; this entry point exists for
 * deployments, not for the method.
 *
 * Some callers may not call cudaMalloc (or any allocator) once they run: a
 * service that reserves its whole device-memory budget at start-up so that
 * nothing can fail later under memory pressure, a plug-in inside a host
 * runtime that owns every device allocation, or a latency-critical loop that
 * cannot afford an allocator call and its driver locks.  This call does the
 * same work as fastid_topk with the plain form (same arguments, results, order
 * and errors) but takes its scratch memory (padded queries, per-query
 * coefficients and per-segment top-k lists) from one array of
 * FASTID_NOALLOC_SCRATCH_BYTES that is part of the library's device code.  It
 * allocates nothing; the caller still provides inputs and outputs.
 *
 *  - A request whose scratch would exceed FASTID_NOALLOC_SCRATCH_BYTES
 *    (roughly: padded queries x loci / 8, plus ~20 MB of lists for k = 32 on
 *    a 152-SM GPU, two CTAs a SM) returns FASTID_EINVAL with the size it needed in
 *    fastid_last_error; nothing is enqueued.
 *  - The first call on a device looks up the array's device address there
 *    (and may make CUDA load that device code); make that first call before
 *    any stream capture.  The array stays resident on every device that used
 *    it until the process exits.  The address is kept per device, so after
 *    cudaDeviceReset (or anything else that destroys the device's primary
 *    context) later calls are invalid.
 *  - While profiling is on (fastid_profile), the call records events around
 *    its compare kernel like fastid_topk.
 *  - Every call uses the same array and it keeps the last call's contents
 *    (nothing in it needs to start at zero).  Calls whose kernels overlap on
 *    the GPU -- on different streams or host threads, or with different
 *    contexts -- race on it: serialise them.
 */
#define FASTID_NOALLOC_SCRATCH_BYTES (32u << 20)
fastid_status fastid_topk_noalloc(fastid_ctx *ctx, const fastid_refdb *db, const uint64_t *queries_dev,
                                  int64_t ld_q, int64_t n_q, const uint8_t *modes_dev, int32_t k,
                                  uint32_t threshold, uint32_t *out_scores_dev, int64_t *out_idx_dev,
                                  fastid_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTID_H */
