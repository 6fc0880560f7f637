// Reductions after a comparison launch: merge of per-segment top-k lists and
// the hit-list finish (count, overflow flag, sort by (q, r)).
#include "common.cuh"

namespace fastid {

namespace {

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_merge32(uint64_t a, uint64_t b, int lane) {
    uint64_t br = shfl64(b, 31 - lane);
    uint64_t v = a < br ? a : br;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        uint64_t p = shfl_xor64(v, j);
        bool lower = (lane & j) == 0;
        v = lower ? (v < p ? v : p) : (v < p ? p : v);
    }
    return v;
}

// CTA whose unit range contains unit u.
__device__ int64_t cta_of(const Partition &P, int64_t u) {
    int64_t c = (u * P.grid) / P.n_units;
    while (c + 1 < P.grid && part_begin(P, c + 1) <= u) ++c;
    while (c > 0 && part_begin(P, c) > u) --c;
    return c;
}

// One warp per query: merge the sorted k-lists of every segment that covered
// the query's tile.  The partition is over work groups (CTAs, or 2-CTA
// clusters when paired: a paired unit covers query tiles 2 qq and 2 qq + 1,
// taken by cluster ranks 0 and 1).  Segment lists are laid out
// [slot][tile_q][k] with slot = cta * max_seg + (segment index within the CTA).
__global__ void topk_merge_kernel(const uint64_t *__restrict__ partial, Partition P, int32_t tile_q, int32_t pair,
                                  int64_t n_q, int32_t k, uint32_t *__restrict__ out_scores,
                                  int64_t *__restrict__ out_idx) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= n_q) return;
    const int64_t qt = q / tile_q, ql = q - qt * tile_q;
    const int64_t qq = pair ? qt >> 1 : qt;
    const int64_t rank = pair ? qt & 1 : 0;
    const int64_t u_lo = qq * P.n_rt, u_hi = u_lo + P.n_rt - 1;
    const int64_t w_lo = cta_of(P, u_lo), w_hi = cta_of(P, u_hi);
    uint64_t acc = KEY_EMPTY;
    for (int64_t w = w_lo; w <= w_hi; ++w) {
        const int64_t first_qq = part_begin(P, w) / P.n_rt;
        const int64_t cta = pair ? 2 * w + rank : w;
        const int64_t slot = cta * P.max_seg + (qq - first_qq);
        uint64_t b = lane < k ? partial[(slot * tile_q + ql) * k + lane] : KEY_EMPTY;
        acc = warp_merge32(acc, b, lane);
    }
    if (lane < k) {
        out_scores[q * k + lane] = acc == KEY_EMPTY ? 0xFFFFFFFFu : (uint32_t)(acc >> 32);
        out_idx[q * k + lane] = acc == KEY_EMPTY ? -1ll : (int64_t)(uint32_t)acc;
    }
}

// Tensor launches: one warp per query; its tile's lists sit in one slot of
// every reference slice's group of its tile group (see TcSched).  Slot
// layout [slot][k][128].
struct MergeSched {
    int32_t n_panels;
    int32_t pair;
    int32_t k;
    TcSched sc[TC_MAXP];
    int64_t n_slots;   // slots in partial (checked by debug builds)
    uint32_t *status;  // the context's status word
    // accumulate: merge into the output lists instead of overwriting them,
    // this launch's reference indices taken + ref_offset
    int32_t accumulate;
    int64_t ref_offset;
    int64_t qspread;  // single-call jobs: output j is input query j (see spread_query_to_row)
};

// Debug builds (FASTID_DEBUG) check every slot a merge reads against the
// slot count; a slot out of range records ST_DEVICE with detail code 1 and is
// read as empty.  Release builds take the schedule's word for it.
__device__ __forceinline__ bool merge_slot_ok(const MergeSched &M, int64_t slot) {
#ifdef FASTID_DEBUG
    if (slot < 0 || slot >= M.n_slots) {
        if ((threadIdx.x & 31) == 0) {
            atomicOr(M.status, ST_DEVICE);
            atomicExch(M.status + 1, 1u);
        }
        return false;
    }
#else
    (void)M;
    (void)slot;
#endif
    return true;
}

__global__ void topk_merge_sched_kernel(const uint64_t *__restrict__ partial, const MergeSched M,
                                        const MergeJob *__restrict__ jobs, int64_t n_jobs,
                                        uint32_t *__restrict__ out_s, int64_t *__restrict__ out_i) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n_jobs) return;
    const int k = M.k;
    MergeJob jb;
    if (jobs) {
        jb = jobs[j];
    } else {
        jb.out_s = out_s + j * k;
        jb.out_i = out_i + j * k;
        jb.panel = 0;
        jb.q = (int32_t)spread_query_to_row(j, M.qspread);  // its operand row
    }
    const TcSched &sc = M.sc[jb.panel];
    const int64_t qt = jb.q / TC_TILE_Q, ql = jb.q - qt * TC_TILE_Q;
    const int64_t qq = M.pair ? qt >> 1 : qt;
    const int64_t rank = M.pair ? qt & 1 : 0;
    const int64_t x = qq / sc.tpx, li = qq - x * sc.tpx;
    uint64_t acc = KEY_EMPTY;
    for (int64_t y = 0; y < sc.b; ++y) {
        const int64_t wg = x * sc.b + y;
        const int64_t cta = M.pair ? 2 * wg + rank : wg;
        const int64_t slot = (int64_t)sc.slot0 + cta * sc.tpx + li;
        uint64_t v = lane < k && merge_slot_ok(M, slot) ? partial[(slot * k + lane) * TC_TILE_Q + ql] : KEY_EMPTY;
        acc = warp_merge32(acc, v, lane);
    }
    if (sc.t_groups > 0) {  // the tail group holding this query tile (see TcSched)
        const int64_t cpg = M.pair ? 2 : 1;
        const int64_t t = qq / sc.t_tpx, lt = qq - t * sc.t_tpx;
        const int64_t slot = (int64_t)sc.slot0 + (int64_t)sc.a * sc.b * cpg * sc.tpx + (t * cpg + rank) * sc.t_tpx + lt;
        uint64_t v = lane < k && merge_slot_ok(M, slot) ? partial[(slot * k + lane) * TC_TILE_Q + ql] : KEY_EMPTY;
        acc = warp_merge32(acc, v, lane);
    }
    if (M.accumulate) {
        // keys are (score << 32) | r: the offset moves r, never the score (r + offset < 2^32)
        if (acc != KEY_EMPTY) acc += (uint64_t)M.ref_offset;
        uint64_t run = KEY_EMPTY;
        if (lane < k) {
            const int64_t ri = jb.out_i[lane];
            if (ri >= 0) run = make_key(jb.out_s[lane], (uint32_t)ri);
        }
        acc = warp_merge32(acc, run, lane);
    }
    if (lane < k) {
        jb.out_s[lane] = acc == KEY_EMPTY ? 0xFFFFFFFFu : (uint32_t)(acc >> 32);
        jb.out_i[lane] = acc == KEY_EMPTY ? -1ll : (int64_t)(uint32_t)acc;
    }
}

// Streamed reference blocks: fold one block's lists (reference indices
// relative to the block, offset added here) into the running lists, one warp
// per query.  Both lists are ascending (score, reference) keys; a bitonic
// merge keeps the k smallest.
__global__ void topk_fold_kernel(uint32_t *__restrict__ run_s, int64_t *__restrict__ run_i,
                                 const uint32_t *__restrict__ blk_s, const int64_t *__restrict__ blk_i,
                                 int64_t offset, int64_t n_q, int32_t k) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= n_q) return;
    uint64_t a = KEY_EMPTY, b = KEY_EMPTY;
    if (lane < k) {
        const int64_t ia = run_i[q * k + lane];
        const int64_t ib = blk_i[q * k + lane];
        if (ia >= 0) a = make_key(run_s[q * k + lane], (uint32_t)ia);
        if (ib >= 0) b = make_key(blk_s[q * k + lane], (uint32_t)(ib + offset));
    }
    const uint64_t v = warp_merge32(a, b, lane);
    if (lane < k) {
        run_s[q * k + lane] = v == KEY_EMPTY ? 0xFFFFFFFFu : (uint32_t)(v >> 32);
        run_i[q * k + lane] = v == KEY_EMPTY ? -1ll : (int64_t)(uint32_t)v;
    }
}

// Streamed reference blocks, hit lists: after block b's hits are appended,
// snaps[b] = the count; the hits appended by block b, positions
// [snaps[b - 1], min(snaps[b], capacity)), get the block's first reference
// index added.
__global__ void hits_snap_kernel(const unsigned long long *__restrict__ count, unsigned long long *__restrict__ snap) {
    *snap = *count;
}

__global__ void hits_offset_kernel(const unsigned long long *__restrict__ snaps, int64_t b, int64_t capacity,
                                   int64_t *__restrict__ hit_r, int64_t r0) {
    const unsigned long long lo = b > 0 ? snaps[b - 1] : 0ull;
    const unsigned long long hi = min(snaps[b], (unsigned long long)capacity);
    for (unsigned long long i = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
         i += (unsigned long long)gridDim.x * blockDim.x)
        hit_r[i] += r0;
}

// ---- hit list finish ----------------------------------------------------
// sort_tmp layout: [0] = live count n (as u64), [1] = next power of two of n,
// then keys[P], then vals (u32)[P].

__global__ void hits_prep_kernel(const unsigned long long *__restrict__ count, int64_t capacity,
                                 int64_t *__restrict__ count_out, uint64_t *__restrict__ tmp,
                                 uint32_t *__restrict__ status) {
    unsigned long long c = *count;
    unsigned long long n = c < (unsigned long long)capacity ? c : (unsigned long long)capacity;
    unsigned long long p = 1;
    while (p < n) p <<= 1;
    tmp[0] = n;
    tmp[1] = p;
    *count_out = (int64_t)c;
    if (c > (unsigned long long)capacity) atomicOr(status, ST_OVERFLOW);
}

__global__ void hits_keys_kernel(const int64_t *__restrict__ hq, const int64_t *__restrict__ hr,
                                 const uint32_t *__restrict__ hs, uint64_t *__restrict__ tmp, int64_t P) {
    const uint64_t n = tmp[0], pn = tmp[1];
    uint64_t *keys = tmp + 2;
    uint32_t *vals = reinterpret_cast<uint32_t *>(tmp + 2 + P);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)pn;
         i += (int64_t)gridDim.x * blockDim.x) {
        if ((uint64_t)i < n) {
            keys[i] = ((uint64_t)hq[i] << 32) | (uint64_t)(uint32_t)hr[i];
            vals[i] = hs[i];
        } else {
            keys[i] = KEY_EMPTY;
            vals[i] = 0;
        }
    }
}

constexpr int SB = 2048;  // elements per shared-memory bitonic block

// All passes j < SB/2.. of stage `size` (or every stage up to SB when
// size == 0) inside blocks of SB contiguous elements.
__global__ void __launch_bounds__(SB / 2) bitonic_smem_kernel(uint64_t *__restrict__ tmp, int64_t P,
                                                              int64_t size) {
    const uint64_t pn = tmp[1];
    const int64_t base = (int64_t)blockIdx.x * SB;
    if ((uint64_t)base >= pn) return;
    if (size > 0 && (uint64_t)size > pn) return;
    __shared__ uint64_t sk[SB];
    __shared__ uint32_t sv[SB];
    uint64_t *keys = tmp + 2;
    uint32_t *vals = reinterpret_cast<uint32_t *>(tmp + 2 + P);
    const int64_t live = ((int64_t)pn - base) < SB ? ((int64_t)pn - base) : SB;
    for (int t = threadIdx.x; t < SB; t += blockDim.x) {
        sk[t] = t < live ? keys[base + t] : KEY_EMPTY;
        sv[t] = t < live ? vals[base + t] : 0u;
    }
    __syncthreads();
    auto pass = [&](int64_t sz, int j) {
        for (int t = threadIdx.x; t < SB / 2; t += blockDim.x) {
            int lo = 2 * t - (t & (j - 1));
            int hi = lo + j;
            int64_t gi = base + lo;
            bool up = (gi & sz) == 0;
            uint64_t a = sk[lo], b = sk[hi];
            if ((a > b) == up) {
                sk[lo] = b;
                sk[hi] = a;
                uint32_t tv = sv[lo];
                sv[lo] = sv[hi];
                sv[hi] = tv;
            }
        }
        __syncthreads();
    };
    if (size == 0) {
        for (int64_t sz = 2; sz <= SB && (uint64_t)sz <= (pn > 1 ? pn : 2); sz <<= 1)
            for (int j = (int)(sz >> 1); j > 0; j >>= 1) pass(sz, j);
    } else {
        for (int j = SB / 2; j > 0; j >>= 1) pass(size, j);
    }
    for (int t = threadIdx.x; t < live; t += blockDim.x) {
        keys[base + t] = sk[t];
        vals[base + t] = sv[t];
    }
}

__global__ void bitonic_global_kernel(uint64_t *__restrict__ tmp, int64_t P, int64_t size, int64_t j) {
    const uint64_t pn = tmp[1];
    if ((uint64_t)size > pn) return;
    uint64_t *keys = tmp + 2;
    uint32_t *vals = reinterpret_cast<uint32_t *>(tmp + 2 + P);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)pn / 2;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 2 * t - (t & (j - 1));
        int64_t hi = lo + j;
        bool up = (lo & size) == 0;
        uint64_t a = keys[lo], b = keys[hi];
        if ((a > b) == up) {
            keys[lo] = b;
            keys[hi] = a;
            uint32_t tv = vals[lo];
            vals[lo] = vals[hi];
            vals[hi] = tv;
        }
    }
}

__global__ void hits_unpack_kernel(const uint64_t *__restrict__ tmp, int64_t P, int64_t *__restrict__ hq,
                                   int64_t *__restrict__ hr, uint32_t *__restrict__ hs) {
    const uint64_t n = tmp[0];
    const uint64_t *keys = tmp + 2;
    const uint32_t *vals = reinterpret_cast<const uint32_t *>(tmp + 2 + P);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; (uint64_t)i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        hq[i] = (int64_t)(keys[i] >> 32);
        hr[i] = (int64_t)(uint32_t)keys[i];
        hs[i] = vals[i];
    }
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

int64_t hits_sort_elems(int64_t capacity) {
    int64_t p = 1;
    while (p < capacity) p <<= 1;
    return p < SB ? SB : p;
}

cudaError_t launch_topk_merge(const uint64_t *partial, const Partition &part, int64_t n_q, int32_t k,
                              uint32_t *out_scores, int64_t *out_idx, cudaStream_t s) {
    if (n_q == 0) return cudaSuccess;
    const int wpb = 8;
    int64_t blocks = (n_q + wpb - 1) / wpb;
    topk_merge_kernel<<<(unsigned)blocks, wpb * 32, 0, s>>>(partial, part, PL_TQ, 0, n_q, k, out_scores, out_idx);
    return cudaGetLastError();
}

cudaError_t launch_topk_merge_tile(const uint64_t *partial, const Partition &part, int32_t tile_q, int32_t pair,
                                   int64_t n_q, int32_t k, uint32_t *out_scores, int64_t *out_idx,
                                   cudaStream_t s) {
    if (n_q == 0) return cudaSuccess;
    const int wpb = 8;
    int64_t blocks = (n_q + wpb - 1) / wpb;
    topk_merge_kernel<<<(unsigned)blocks, wpb * 32, 0, s>>>(partial, part, tile_q, pair, n_q, k, out_scores,
                                                            out_idx);
    return cudaGetLastError();
}

cudaError_t launch_merge_sched(const uint64_t *partial, const TcLaunch &L, const MergeJob *jobs, int64_t n_jobs,
                               uint32_t *out_scores, int64_t *out_idx, cudaStream_t s, bool accumulate,
                               int64_t ref_offset) {
    if (n_jobs == 0) return cudaSuccess;
    MergeSched M;
    M.accumulate = accumulate ? 1 : 0;
    M.ref_offset = ref_offset;
    M.n_panels = L.n_panels;
    M.pair = L.pair;
    M.k = L.k;
    for (int p = 0; p < TC_MAXP; ++p) M.sc[p] = L.sched[p];
    M.n_slots = L.n_slots;
    M.status = L.status;
    M.qspread = L.qspread[0];
    const int wpb = 8;
    int64_t blocks = (n_jobs + wpb - 1) / wpb;
    topk_merge_sched_kernel<<<(unsigned)blocks, wpb * 32, 0, s>>>(partial, M, jobs, n_jobs, out_scores, out_idx);
    return cudaGetLastError();
}

cudaError_t launch_topk_fold(uint32_t *run_s, int64_t *run_i, const uint32_t *blk_s, const int64_t *blk_i,
                             int64_t offset, int64_t n_q, int32_t k, cudaStream_t s) {
    if (n_q == 0) return cudaSuccess;
    const int wpb = 8;
    topk_fold_kernel<<<(unsigned)((n_q + wpb - 1) / wpb), wpb * 32, 0, s>>>(run_s, run_i, blk_s, blk_i, offset,
                                                                             n_q, k);
    return cudaGetLastError();
}

cudaError_t launch_hits_block_offset(const unsigned long long *count, unsigned long long *snaps, int64_t b,
                                     int64_t capacity, int64_t *hit_r, int64_t r0, int grid, cudaStream_t s) {
    hits_snap_kernel<<<1, 1, 0, s>>>(count, snaps + b);
    if (r0 != 0 && capacity > 0) hits_offset_kernel<<<grid, 256, 0, s>>>(snaps, b, capacity, hit_r, r0);
    return cudaGetLastError();
}

// sort_tmp must hold 2 + hits_sort_elems(capacity) * 1.5 u64 words.
cudaError_t launch_hits_finish(unsigned long long *count, int64_t capacity, int64_t *hit_q,
                               int64_t *hit_r, uint32_t *hit_score, int64_t *count_out,
                               uint64_t *sort_tmp, uint32_t *status, cudaStream_t s) {
    const int64_t P = hits_sort_elems(capacity);
    hits_prep_kernel<<<1, 1, 0, s>>>(count, capacity, count_out, sort_tmp, status);
    if (capacity == 0) return cudaGetLastError();
    hits_keys_kernel<<<grid_for(P, 256), 256, 0, s>>>(hit_q, hit_r, hit_score, sort_tmp, P);
    const int nblk = (int)(P / SB);
    bitonic_smem_kernel<<<nblk, SB / 2, 0, s>>>(sort_tmp, P, 0);
    for (int64_t size = 2 * SB; size <= P; size <<= 1) {
        for (int64_t j = size >> 1; j >= SB; j >>= 1)
            bitonic_global_kernel<<<grid_for(P / 2, 256), 256, 0, s>>>(sort_tmp, P, size, j);
        bitonic_smem_kernel<<<nblk, SB / 2, 0, s>>>(sort_tmp, P, size);
    }
    hits_unpack_kernel<<<grid_for(capacity, 256), 256, 0, s>>>(sort_tmp, P, hit_q, hit_r, hit_score);
    return cudaGetLastError();
}

}  // namespace fastid
