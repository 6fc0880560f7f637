// Plain form of the overloaded matrix multiply (Sec. II-B, III-B): packed
// 32-bit words, AND + POPC on the integer pipes, register-blocked tiles
// staged through shared memory with cp.async.  Each group of eight ANDed
// word pairs goes through a carry-save adder tree first (and_popc8), so that
// four POPCs count eight words: POPC issues at 16 results a clock per SM,
// a quarter of the logic-op rate, and one POPC per word bound the loop.
//
// The paper's kernel (Algorithm 3 plus tiling, register blocking and
// coalescing, Sec. III-B) computes POPC(AND(XOR(A, B), A)) per word.  Here
// one contraction G = sum_w popc(R_w AND Q_w) serves both scores through the
// reference popcount |R| and per-query coefficients (a, b):
//     score = |R| + b - a G
//     mode 0: a = 2, b = |Q|  ->  |R| + |Q| - 2G = popc(R XOR Q)
//     mode 1: a = 1, b = 0    ->  |R| - G       = popc(R AND NOT Q)  (Eq. 1)
//
// CTA tile: 128 references x 128 queries, 256 threads, each thread owns 8
// references (rows tr + 16 i) and 8 queries (rows tq + 16 j) of the tile;
// two CTAs an SM.
// The grid is persistent: CTA c walks the units [c U / G, (c+1) U / G) of the
// query-tile-major list of (query tile, reference tile) units, so within one
// query tile a CTA sees references in increasing order.
//
// Epilogues (fused, the score matrix is never stored except by EPI_SCORES*):
//   EPI_SCORES16/32  write the full matrix (small problems only).
//   EPI_HITS         append every (q, r, score) with score <= threshold.
//   EPI_TOPK         keep per query the k smallest keys (score << 32 | r) of
//                    the CTA's segment in shared memory; the segment's list
//                    goes to scratch and a merge kernel combines segments.
#include "common.cuh"

namespace fastid {

namespace {

constexpr int KCP = PL_KC + 4;  // padded shared-memory row (u32): conflict-free LDS.128
constexpr int STG = 16;         // staged top-k candidates per query between merges
constexpr int NWARPS = PL_THREADS / 32;

struct PlainArgs {
    const uint32_t *refs32;
    const uint32_t *ref_norms;
    int64_t n_refs;
    int64_t ld32;
    int32_t n_kc;  // K stages of PL_KC words
    const uint32_t *q32;
    const QueryCoef *coef;
    int64_t n_q;
    uint32_t threshold;
    int32_t k;
    void *out;
    int64_t ld_out;
    int64_t capacity;
    int64_t *hit_q;
    int64_t *hit_r;
    uint32_t *hit_score;
    unsigned long long *hit_count;
    uint64_t *partial;
    Partition part;
    uint32_t *status;
    uint32_t two;  // 2 (see and_popc8)
};

struct TopkSmem {
    uint64_t list[PL_TQ][FASTID_MAX_K];  // sorted ascending; KEY_EMPTY pads
    uint64_t stage[PL_TQ][STG];
    uint64_t cut[PL_TQ];
    int32_t cnt[PL_TQ];
    int32_t ovf[2];
};

__device__ __forceinline__ void cp_async16(uint32_t *smem, const uint32_t *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

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

// Ascending bitonic sort of one key per lane across the warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            uint64_t p = shfl_xor64(v, j);
            bool up = (lane & size) == 0 || size == 32;
            bool lower = (lane & j) == 0;
            v = (lower == up) ? (v < p ? v : p) : (v < p ? p : v);
        }
    }
    return v;
}

// Given a sorted ascending (one key per lane) and b sorted ascending, return
// the 32 smallest of a U b, sorted ascending.
__device__ __forceinline__ uint64_t warp_merge32(uint64_t a, uint64_t b, int lane) {
    uint64_t br = shfl64(b, 31 - lane);
    uint64_t v = a < br ? a : br;  // bitonic: the 32 smallest
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        uint64_t p = shfl_xor64(v, j);
        bool lower = (lane & j) == 0;
        v = lower ? (v < p ? v : p) : (v < p ? p : v);
    }
    return v;
}

// Full adder of three bit vectors: sum (three-input XOR, LOP3 table 0x96)
// and carry (majority, table 0xE8), one LOP3 each -- written out, as the
// compiler's own code for the same expressions ran the step 1.35x slower.
__device__ __forceinline__ void full_add(uint32_t &sum, uint32_t &carry, uint32_t a, uint32_t b, uint32_t c) {
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(sum) : "r"(a), "r"(b), "r"(c));
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(carry) : "r"(a), "r"(b), "r"(c));
}

// acc + sum of popc(r_i AND q_i) over the 8 word pairs of (ra, rb) x (qa, qb):
// full adders reduce the eight ANDed words to bit vectors of weight 1, 1, 2
// and 4 -- x0+x1+x2 = s1 + 2 c1, x3+x4+x5 = s2 + 2 c2, s1+s2+x6 = s3 + 2 c3,
// c1+c2+c3 = t + 2 d -- so the eight words hold s3 + x7 + 2 t + 4 d ones per
// bit position.  `two` is 2, passed in so that the weighted adds stay
// multiply-adds (the FMA pipe, idle here) instead of shifts on the logic pipe.
__device__ __forceinline__ uint32_t and_popc8(const uint4 ra, const uint4 rb, const uint4 qa, const uint4 qb,
                                              uint32_t acc, uint32_t two) {
    const uint32_t x0 = ra.x & qa.x, x1 = ra.y & qa.y, x2 = ra.z & qa.z, x3 = ra.w & qa.w;
    const uint32_t x4 = rb.x & qb.x, x5 = rb.y & qb.y, x6 = rb.z & qb.z, x7 = rb.w & qb.w;
    uint32_t s1, c1, s2, c2, s3, c3, t, d;
    full_add(s1, c1, x0, x1, x2);
    full_add(s2, c2, x3, x4, x5);
    full_add(s3, c3, s1, s2, x6);
    full_add(t, d, c1, c2, c3);
    return (__popc(d) * two + __popc(t)) * two + (acc + __popc(s3) + __popc(x7));
}

// A reference operand's 16 bytes, read from shared memory for every four
// query columns.  The 8 x 8 register tile then holds its 64 counters, four
// query columns and one reference row, within 128 registers, so two CTAs
// share an SM: four warps per scheduler instead of two, to hide the POPC and
// LOP3 latencies.  Holding all eight reference rows instead takes 177
// registers and one CTA per SM (2048 x 20M: 480 ms against 435 ms, both
// without the cross-unit copy of the next unit's first stage); reading the
// row for every single query column keeps two CTAs but triples the
// shared-memory wavefronts (459 ms).  The volatile load keeps the compiler
// from merging the two reads of a row back into registers; within a warp it
// is a broadcast of two addresses, one shared-memory wavefront.
__device__ __forceinline__ uint4 lds128_once(const uint32_t *p) {
    uint4 v;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

template <int EPI>
__global__ void __launch_bounds__(PL_THREADS, 2) plain_kernel(const PlainArgs args) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t(*sR)[PL_TR][KCP] = reinterpret_cast<uint32_t(*)[PL_TR][KCP]>(smem_raw);
    uint32_t(*sQ)[PL_TQ][KCP] =
        reinterpret_cast<uint32_t(*)[PL_TQ][KCP]>(smem_raw + 2 * PL_TR * KCP * sizeof(uint32_t));
    TopkSmem *tk = reinterpret_cast<TopkSmem *>(smem_raw + 2 * (PL_TR + PL_TQ) * KCP * sizeof(uint32_t));

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tq = tid & 15;
    const int tr = tid >> 4;
    const Partition &P = args.part;
    const int64_t c = blockIdx.x;
    const int64_t u_begin = part_begin(P, c);
    const int64_t u_end = part_begin(P, c + 1);
    const uint64_t cut0 = initial_cut(args.threshold);

    if (EPI == EPI_TOPK) {
        for (int i = tid; i < PL_TQ * FASTID_MAX_K; i += PL_THREADS) (&tk->list[0][0])[i] = KEY_EMPTY;
        for (int i = tid; i < PL_TQ; i += PL_THREADS) {
            tk->cut[i] = cut0;
            tk->cnt[i] = 0;
        }
        if (tid < 2) tk->ovf[tid] = 0;
        __syncthreads();
    }

    // Loader mapping: each stage is 128 rows x 16 words per operand = 512
    // 16-byte chunks; 256 threads copy 2 chunks of R and 2 of Q.
    // Stage s of a unit goes to buffer (g + s) & 1, g counting the stages of
    // the CTA's earlier units, so that the next unit's first stage can be
    // copied into the free buffer during this unit's last stage and epilogue.
    auto issue_stage = [&](int st, const uint32_t *gR_, const uint32_t *gQ_, int kc) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            int chunk = tid + t * PL_THREADS;  // 0..511
            int row = chunk >> 2, part = chunk & 3;
            cp_async16(&sR[st][row][part * 4], gR_ + row * args.ld32 + kc * PL_KC + part * 4);
            cp_async16(&sQ[st][row][part * 4], gQ_ + row * args.ld32 + kc * PL_KC + part * 4);
        }
        cp_async_commit();
    };
    int g = 0;
    bool staged = false;  // this unit's first stage is already in flight
    int seg = 0;
    int64_t qt_prev = -1;
    for (int64_t u = u_begin; u < u_end; ++u) {
        const int64_t qt = u / P.n_rt;
        const int64_t rt = u - qt * P.n_rt;
        const int64_t r0 = rt * PL_TR;
        const int64_t q0 = qt * PL_TQ;

        if (EPI == EPI_TOPK && qt != qt_prev) {
            if (qt_prev >= 0) {
                // flush the finished segment's lists
                uint64_t *dst = args.partial + ((c * P.max_seg + seg) * PL_TQ) * (int64_t)args.k;
                for (int i = tid; i < PL_TQ * args.k; i += PL_THREADS) {
                    int qq = i / args.k, s = i - qq * args.k;
                    dst[i] = tk->list[qq][s];
                }
                __syncthreads();
                for (int i = tid; i < PL_TQ * FASTID_MAX_K; i += PL_THREADS) (&tk->list[0][0])[i] = KEY_EMPTY;
                for (int i = tid; i < PL_TQ; i += PL_THREADS) tk->cut[i] = cut0;
                __syncthreads();
                ++seg;
            }
            qt_prev = qt;
        }

        const uint32_t *gR = args.refs32 + r0 * args.ld32;
        const uint32_t *gQ = args.q32 + q0 * args.ld32;

        uint32_t acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0;

        if (!staged) issue_stage(g & 1, gR, gQ, 0);
        for (int kc = 0; kc < args.n_kc; ++kc) {
            const int st = (g + kc) & 1;
            if (kc + 1 < args.n_kc) {
                issue_stage(st ^ 1, gR, gQ, kc + 1);
                cp_async_wait<1>();
            } else if (u + 1 < u_end) {  // the next unit's first stage
                const int64_t qn = (u + 1) / P.n_rt;
                const int64_t rn = (u + 1) - qn * P.n_rt;
                issue_stage(st ^ 1, args.refs32 + rn * PL_TR * args.ld32, args.q32 + qn * PL_TQ * args.ld32, 0);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            static_assert(PL_KC % 8 == 0, "eight-word carry-save groups");
#pragma unroll
            for (int kk = 0; kk < PL_KC; kk += 8) {
#pragma unroll
                for (int jh = 0; jh < 8; jh += 4) {  // four query columns at a time
                    uint4 qa[4], qb[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        qa[j] = *reinterpret_cast<const uint4 *>(&sQ[st][tq + 16 * (jh + j)][kk]);
                        qb[j] = *reinterpret_cast<const uint4 *>(&sQ[st][tq + 16 * (jh + j)][kk + 4]);
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        // read once per four query columns (see lds128_once)
                        const uint4 ra = lds128_once(&sR[st][tr + 16 * i][kk]);
                        const uint4 rb = lds128_once(&sR[st][tr + 16 * i][kk + 4]);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            acc[i][jh + j] = and_popc8(ra, rb, qa[j], qb[j], acc[i][jh + j], args.two);
                    }
                }
            }
            __syncthreads();
        }
        g += args.n_kc;
        staged = u + 1 < u_end;

        // ---- epilogue: scores ----
        uint32_t nr[8];
        bool rvalid[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int64_t r = r0 + tr + 16 * i;
            rvalid[i] = r < args.n_refs;
            nr[i] = __ldg(args.ref_norms + r0 + tr + 16 * i);  // padded rows exist (norm 0)
        }
        uint32_t sc[8][8];
        bool qvalid[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int64_t q = q0 + tq + 16 * j;
            qvalid[j] = q < args.n_q;
            QueryCoef cf = args.coef[q];  // padded rows exist
#pragma unroll
            for (int i = 0; i < 8; ++i) sc[i][j] = nr[i] + cf.b - cf.a * acc[i][j];
        }

        if (EPI == EPI_SCORES16 || EPI == EPI_SCORES32) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!qvalid[j]) continue;
                int64_t q = q0 + tq + 16 * j;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (!rvalid[i]) continue;
                    int64_t r = r0 + tr + 16 * i;
                    if (EPI == EPI_SCORES16)
                        reinterpret_cast<uint16_t *>(args.out)[q * args.ld_out + r] = (uint16_t)sc[i][j];
                    else
                        reinterpret_cast<uint32_t *>(args.out)[q * args.ld_out + r] = sc[i][j];
                }
            }
        } else if (EPI == EPI_HITS) {
            bool any = false;
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int i = 0; i < 8; ++i) any |= qvalid[j] && rvalid[i] && sc[i][j] <= args.threshold;
            if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        bool pred = qvalid[j] && rvalid[i] && sc[i][j] <= args.threshold;
                        unsigned m = __ballot_sync(0xffffffffu, pred);
                        if (m == 0) continue;
                        int leader = __ffs(m) - 1;
                        unsigned long long base = 0;
                        if (lane == leader) base = atomicAdd(args.hit_count, (unsigned long long)__popc(m));
                        base = __shfl_sync(0xffffffffu, base, leader);
                        if (pred) {
                            unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
                            if (pos < (unsigned long long)args.capacity) {
                                args.hit_q[pos] = q0 + tq + 16 * j;
                                args.hit_r[pos] = r0 + tr + 16 * i;
                                args.hit_score[pos] = sc[i][j];
                            }
                        }
                    }
                }
            }
        } else {  // EPI_TOPK
            uint64_t done = 0;  // bit i*8+j: element already staged or rejected
            int pass = 0;
            while (true) {
                bool staged_any = false;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ql = tq + 16 * j;
                    const uint64_t cut = tk->cut[ql];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint64_t bit = 1ull << (i * 8 + j);
                        if (done & bit) continue;
                        const uint64_t key = make_key(sc[i][j], (uint32_t)(r0 + tr + 16 * i));
                        if (!(qvalid[j] && rvalid[i]) || key >= cut) {
                            done |= bit;  // the cut only decreases: rejected for good
                            continue;
                        }
                        int pos = atomicAdd(&tk->cnt[ql], 1);
                        if (pos < STG) {
                            tk->stage[ql][pos] = key;
                            done |= bit;
                            staged_any = true;
                        } else {
                            tk->ovf[pass & 1] = 1;
                            staged_any = true;
                        }
                    }
                }
                if (!__syncthreads_or(staged_any)) break;
                if (tid == 0) tk->ovf[(pass + 1) & 1] = 0;
                // merge staged candidates, one warp per query
                for (int ql = warp; ql < PL_TQ; ql += NWARPS) {
                    int cnt = tk->cnt[ql];
                    if (cnt == 0) continue;
                    if (cnt > STG) cnt = STG;
                    uint64_t a = tk->list[ql][lane];
                    uint64_t b = lane < cnt ? tk->stage[ql][lane] : KEY_EMPTY;
                    b = warp_sort32(b, lane);
                    uint64_t v = warp_merge32(a, b, lane);
                    tk->list[ql][lane] = lane < args.k ? v : KEY_EMPTY;
                    uint64_t kth = shfl64(v, args.k - 1);
                    if (lane == 0) {
                        tk->cut[ql] = kth < cut0 ? kth : cut0;
                        tk->cnt[ql] = 0;
                    }
                }
                __syncthreads();
                const int again = tk->ovf[pass & 1];
                ++pass;
                if (!again) break;
            }
            // leave both flags clear for the next tile (the K loop's barriers
            // order this before the next filter pass)
            if (tid == 0) tk->ovf[0] = tk->ovf[1] = 0;
        }
    }

    if (EPI == EPI_TOPK && qt_prev >= 0) {
        uint64_t *dst = args.partial + ((c * P.max_seg + seg) * PL_TQ) * (int64_t)args.k;
        for (int i = tid; i < PL_TQ * args.k; i += PL_THREADS) {
            int qq = i / args.k, s = i - qq * args.k;
            dst[i] = tk->list[qq][s];
        }
    }
}

size_t plain_smem(int epi) {
    size_t base = 2 * (size_t)(PL_TR + PL_TQ) * KCP * sizeof(uint32_t);
    if (epi == EPI_TOPK) base += sizeof(TopkSmem);
    return base;
}

template <int EPI>
const void *plain_fn() {
    return reinterpret_cast<const void *>(&plain_kernel<EPI>);
}

const void *plain_fn_by_epi(int epi) {
    switch (epi) {
        case EPI_SCORES16: return plain_fn<EPI_SCORES16>();
        case EPI_SCORES32: return plain_fn<EPI_SCORES32>();
        case EPI_HITS: return plain_fn<EPI_HITS>();
        default: return plain_fn<EPI_TOPK>();
    }
}

}  // namespace

int plain_grid_target(int epi, int device) {
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const void *fn = plain_fn_by_epi(epi);
    size_t smem = plain_smem(epi);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, PL_THREADS, smem);
    if (occ < 1) occ = 1;
    return sms * occ;
}

cudaError_t launch_plain(int epi, const uint32_t *refs32, const uint32_t *ref_norms, int64_t n_refs,
                         int64_t ld32, int32_t k_words32, const uint32_t *q32,
                         const QueryCoef *coef, int64_t n_q, uint32_t threshold, int32_t k,
                         void *out, int64_t ld_out, int64_t capacity, int64_t *hit_q,
                         int64_t *hit_r, uint32_t *hit_score, unsigned long long *hit_count,
                         uint64_t *partial, const Partition &part, uint32_t *status,
                         cudaStream_t s) {
    PlainArgs a;
    a.refs32 = refs32;
    a.ref_norms = ref_norms;
    a.n_refs = n_refs;
    a.ld32 = ld32;
    a.n_kc = (k_words32 + PL_KC - 1) / PL_KC;
    a.two = 2u;
    a.q32 = q32;
    a.coef = coef;
    a.n_q = n_q;
    a.threshold = threshold;
    a.k = k;
    a.out = out;
    a.ld_out = ld_out;
    a.capacity = capacity;
    a.hit_q = hit_q;
    a.hit_r = hit_r;
    a.hit_score = hit_score;
    a.hit_count = hit_count;
    a.partial = partial;
    a.part = part;
    a.status = status;
    size_t smem = plain_smem(epi);
    const void *fn = plain_fn_by_epi(epi);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    switch (epi) {
        case EPI_SCORES16: plain_kernel<EPI_SCORES16><<<part.grid, PL_THREADS, smem, s>>>(a); break;
        case EPI_SCORES32: plain_kernel<EPI_SCORES32><<<part.grid, PL_THREADS, smem, s>>>(a); break;
        case EPI_HITS: plain_kernel<EPI_HITS><<<part.grid, PL_THREADS, smem, s>>>(a); break;
        default: plain_kernel<EPI_TOPK><<<part.grid, PL_THREADS, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace fastid
