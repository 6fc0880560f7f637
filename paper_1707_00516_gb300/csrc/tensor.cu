// Tensor-core form of the overloaded matrix multiply on 5th-generation
// tensor cores (tcgen05), FP8 e4m3 operands, FP32 accumulation in TMEM.
//
// The paper computes POPC(AND(XOR(R, Q), R)) word by word (Eq. 1,
// Algorithm 3).  On 0/1 vectors the same counts are ordinary dot products,
// so the contraction can run as a real GEMM D = A B^T if the query side is
// encoded per mode (l < N; padding loci are 0 on both sides):
//     mode 1 (Eq. 1):  a_l = 1 - Q_l      D = sum_l R_l (1 - Q_l) = popc(R AND NOT Q)
//     mode 0 (XOR):    a_l = 1 - 2 Q_l    D = |R| - 2 G,   popc(R XOR Q) = D + |Q|
// with b_l = R_l.  So score = D + c_q (c_q = |Q| in mode 0, 0 in mode 1) and
// no reference popcount is needed.  Every partial sum is an integer of
// magnitude <= N <= 65536 < 2^24, exact in FP32 whatever the order of the
// additions; 0, +1 and -1 are exact in e4m3 (0x00, 0x38, 0xB8).
//
// Tile: M = 128 queries (TMEM lanes) x N = 256 references (TMEM columns),
// K staged 128 loci (one 128-byte swizzle atom) per pipeline stage by TMA.
// Warp roles in a 192-thread CTA, one CTA per SM (persistent):
//   warp 0       TMA producer (one lane)
//   warp 1       TMEM allocation + MMA issue (one lane)
//   warps 2..5   epilogue: TMEM -> registers -> score filter -> per-query
//                top-k (thread = query), hit list or full score matrix
// Two accumulators (2 x 256 TMEM columns) let the epilogue of one reference
// tile overlap the MMAs of the next.  Every mbarrier wait is bounded: on
// timeout the thread records FASTID_ETIMEOUT in the status word and the CTA
// drains and exits.
#include <cuda.h>

#include "common.cuh"

namespace fastid {

namespace {

constexpr int TC_BM = 128;            // queries per tile
constexpr int TC_BN = 256;            // references per tile
constexpr int TC_BK = 128;            // loci (bytes) per stage
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 192;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK;  // 16 KB
constexpr uint32_t TC_B_BYTES = TC_BN * TC_BK;  // 32 KB
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 2000000000ull;     // 2 s per wait

struct TensorArgs {
    int64_t n_refs;
    int64_t n_q;
    int32_t n_kb;  // K stages
    const float *qconst;  // c_q per padded query
    uint32_t threshold;   // already clamped to <= N
    int32_t k;
    int32_t epi;
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
};

// ---- PTX wrappers --------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and records a timeout) if the phase does not
// complete within WAIT_NS or if another thread of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t *status, uint32_t site) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > WAIT_NS) {
                *abort_flag = 1;
                atomicOr(status, ST_TIMEOUT);
                atomicExch(status + 1, site);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int32_t x,
                                            int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major,
// N = 256, M = 128.
__host__ __device__ constexpr uint32_t idesc_f8(int m, int n) {
    return (1u << 4)                      // D format: F32
           | (0u << 7) | (0u << 10)       // A, B format: E4M3
           | ((uint32_t)(n >> 3) << 17)   // N >> 3
           | ((uint32_t)(m >> 4) << 24);  // M >> 4
}

// Per-thread top-k list held in registers, ascending by score; entries of
// equal score keep arrival order (references arrive in increasing order, so
// the earlier entry has the lower index).  Inserting (xs, xr) is a fixed
// compare-select network, so all lanes of a warp insert in lock-step; a lane
// with nothing to insert passes xs = INT32_MAX, which changes nothing.
// For a runtime k <= 32 the first 32 - k slots hold INT32_MIN place-holders
// that nothing displaces, so the k kept entries sit in slots 32-k .. 31 and
// the k-th smallest is always slot 31 (static register indices only).
constexpr int TC_KMAX = 32;
constexpr int32_t NET_EMPTY = 0x7fffffff;
constexpr int32_t NET_HOLD = (int32_t)0x80000000;

__device__ __forceinline__ void net_insert(int32_t (&ls)[TC_KMAX], uint32_t (&lr)[TC_KMAX], int32_t xs,
                                           uint32_t xr) {
#pragma unroll
    for (int i = TC_KMAX - 1; i > 0; --i) {
        const bool shift = xs < ls[i - 1];
        const bool here = xs < ls[i];
        ls[i] = shift ? ls[i - 1] : (here ? xs : ls[i]);
        lr[i] = shift ? lr[i - 1] : (here ? xr : lr[i]);
    }
    const bool first = xs < ls[0];
    ls[0] = first ? xs : ls[0];
    lr[0] = first ? xr : lr[0];
}

struct TcSmem {
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __noinline__ void append_hit(unsigned long long *count, int64_t capacity, int64_t *hq, int64_t *hr,
                                       uint32_t *hs, int64_t q, int64_t r, uint32_t sc) {
    const unsigned long long pos = atomicAdd(count, 1ull);
    if (pos < (unsigned long long)capacity) {
        hq[pos] = q;
        hr[pos] = r;
        hs[pos] = sc;
    }
}

// Bounded wait that ignores the abort flag: used to drain this CTA's own
// asynchronous copies and MMAs before it exits.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, uint32_t *status, uint32_t site) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > WAIT_NS) {
            atomicOr(status, ST_TIMEOUT);
            atomicExch(status + 1, site);
            return;
        }
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tensor_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                  const TensorArgs args) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand stages, then control block, then top-k lists.
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t *base = smem_raw + pad;
    uint8_t *sA = base;
    uint8_t *sB = base + TC_STAGES * TC_A_BYTES;
    TcSmem *ctl = reinterpret_cast<TcSmem *>(base + TC_STAGES * (TC_A_BYTES + TC_B_BYTES));
    // per-thread staging of one 32-column chunk, [32][128] floats (rare path)
    float *stage_v = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(ctl) + 256);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const Partition &P = args.part;
    const int64_t c = blockIdx.x;
    const int64_t u_begin = part_begin(P, c), u_end = part_begin(P, c + 1);
    volatile int *abort_flag = &ctl->abort_flag;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), 1);
            mbar_init(smem_u32(&ctl->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->tfull[a]), 1);
            mbar_init(smem_u32(&ctl->tempty[a]), 128);
        }
        mbar_init(smem_u32(&ctl->done), 1);
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = ctl->tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok; ++u) {
                const int64_t qt = u / P.n_rt, rt = u - qt * P.n_rt;
                for (int kb = 0; kb < args.n_kb; ++kb) {
                    ok = mbar_wait(smem_u32(&ctl->empty[stage]), phase ^ 1u, abort_flag, args.status, 1);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&ctl->full[stage]);
                    mbar_expect_tx(fb, TC_A_BYTES + TC_B_BYTES);
                    tma_load_2d(smem_u32(sA + stage * TC_A_BYTES), &map_a, fb, kb * TC_BK, (int32_t)(qt * TC_BM));
                    tma_load_2d(smem_u32(sB + stage * TC_B_BYTES), &map_b, fb, kb * TC_BK, (int32_t)(rt * TC_BN));
                    ++issued;
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // Drain: the last fill of every stage has landed before the CTA
            // exits (fill n used stage n % S in phase (n / S) & 1).
            for (int64_t n = issued - 1; n >= 0 && n >= issued - TC_STAGES; --n)
                mbar_drain(smem_u32(&ctl->full[n % TC_STAGES]), (uint32_t)((n / TC_STAGES) & 1), args.status, 2);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f8(TC_BM, TC_BN);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok; ++u) {
                ok = mbar_wait(smem_u32(&ctl->tempty[acc]), acc_phase ^ 1u, abort_flag, args.status, 3);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_BN);
                for (int kb = 0; kb < args.n_kb; ++kb) {
                    ok = mbar_wait(smem_u32(&ctl->full[stage]), phase, abort_flag, args.status, 4);
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t ad = sw128_desc(smem_u32(sA + stage * TC_A_BYTES));
                    const uint64_t bd = sw128_desc(smem_u32(sB + stage * TC_B_BYTES));
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 32; ++kk)  // K = 32 FP8 per MMA: +32 bytes = +2 in the address field
                        tc_mma_f8(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb | kk) != 0);
                    tc_commit(smem_u32(&ctl->empty[stage]));
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(smem_u32(&ctl->tfull[acc]));
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
            // Drain: a commit completes after every MMA this thread issued.
            tc_commit(smem_u32(&ctl->done));
            mbar_drain(smem_u32(&ctl->done), 0, args.status, 5);
        }
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;            // TMEM lane quadrant this warp may access
        const int row = quad * 32 + lane;     // query row within the tile
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const float tplus1 = args.threshold == 0xFFFFFFFFu ? __int_as_float(0x7f800000) : (float)args.threshold + 1.0f;
        const int k = args.k;
        int acc = 0;
        uint32_t acc_phase = 0;
        int64_t qt_prev = -1;
        int seg = 0;
        int32_t ls[TC_KMAX];  // this thread's top-k scores (see net_insert)
        uint32_t lr[TC_KMAX]; // and their references
        float cq = 0.f;    // c_q
        float cut = 0.f;   // D must be < cut to be a candidate
        float cut0 = 0.f;  // cut while the list is not full
        bool qvalid = false;
        int64_t q = 0;
        for (int64_t u = u_begin; u < u_end; ++u) {
            const int64_t qt = u / P.n_rt, rt = u - qt * P.n_rt;
            if (qt != qt_prev) {
                if (args.epi == EPI_TOPK && qt_prev >= 0) {
                    uint64_t *dst = args.partial + ((c * P.max_seg + seg) * TC_BM + row) * (int64_t)k;
#pragma unroll
                    for (int i = 0; i < TC_KMAX; ++i)
                        if (i >= TC_KMAX - k)
                            dst[i - (TC_KMAX - k)] = ls[i] == NET_EMPTY ? KEY_EMPTY : make_key((uint32_t)ls[i], lr[i]);
                    ++seg;
                }
                qt_prev = qt;
                q = qt * TC_BM + row;
                qvalid = q < args.n_q;
                cq = args.qconst[q];
#pragma unroll
                for (int i = 0; i < TC_KMAX; ++i) {
                    ls[i] = i < TC_KMAX - k ? NET_HOLD : NET_EMPTY;
                    lr[i] = 0xFFFFFFFFu;
                }
                cut0 = qvalid ? tplus1 - cq : -__int_as_float(0x7f800000);
                cut = cut0;
            }
            const bool got = mbar_wait(smem_u32(&ctl->tfull[acc]), acc_phase, abort_flag, args.status, 6);
            __syncwarp();
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const int64_t r0 = rt * TC_BN;
            const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * TC_BN);
#pragma unroll 1
            for (int ch = 0; ch < TC_BN / 32; ++ch) {
                uint32_t v[32];
                __syncwarp();  // tcgen05.ld is warp-collective: reconverge first
                tmem_ld32(taddr + ch * 32, v);
                if (ch == TC_BN / 32 - 1) {
                    tc_fence_before();
                    mbar_arrive(smem_u32(&ctl->tempty[acc]));
                }
                const int64_t rc = r0 + ch * 32;
                if (args.epi == EPI_SCORES16 || args.epi == EPI_SCORES32) {
                    if (qvalid) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t r = rc + j;
                            if (r < args.n_refs) {
                                const uint32_t sc = (uint32_t)(int32_t)(__uint_as_float(v[j]) + cq);
                                if (args.epi == EPI_SCORES16)
                                    reinterpret_cast<uint16_t *>(args.out)[q * args.ld_out + r] = (uint16_t)sc;
                                else
                                    reinterpret_cast<uint32_t *>(args.out)[q * args.ld_out + r] = sc;
                            }
                        }
                    }
                    continue;
                }
                uint32_t m = 0;  // columns of this chunk that pass the filter
#pragma unroll
                for (int j = 0; j < 32; ++j) m |= (uint32_t)(__uint_as_float(v[j]) < cut) << j;
                if (rc + 32 > args.n_refs) m &= rc >= args.n_refs ? 0u : ((1u << (args.n_refs - rc)) - 1u);
                if (!__any_sync(0xffffffffu, m != 0u)) continue;
                if (args.epi == EPI_HITS) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (m & (1u << j))
                            append_hit(args.hit_count, args.capacity, args.hit_q, args.hit_r, args.hit_score, q,
                                       rc + j, (uint32_t)(int32_t)(__uint_as_float(v[j]) + cq));
                    continue;
                }
                // rare path: stage the chunk, then insert candidates in lock-step
#pragma unroll
                for (int j = 0; j < 32; ++j) stage_v[j * TC_BM + row] = __uint_as_float(v[j]);
                while (__any_sync(0xffffffffu, m != 0u)) {
                    int32_t xs = NET_EMPTY;
                    uint32_t xr = 0u;
                    if (m != 0u) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1u;
                        const float d = stage_v[j * TC_BM + row];
                        if (d < cut) {
                            xs = (int32_t)(d + cq);
                            xr = (uint32_t)(rc + j);
                        }
                    }
                    net_insert(ls, lr, xs, xr);
                    cut = ls[TC_KMAX - 1] == NET_EMPTY ? cut0 : (float)ls[TC_KMAX - 1] - cq;
                }
            }
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
        if (args.epi == EPI_TOPK && qt_prev >= 0 && !*abort_flag) {
            uint64_t *dst = args.partial + ((c * P.max_seg + seg) * TC_BM + row) * (int64_t)k;
#pragma unroll
            for (int i = 0; i < TC_KMAX; ++i)
                if (i >= TC_KMAX - k)
                    dst[i - (TC_KMAX - k)] = ls[i] == NET_EMPTY ? KEY_EMPTY : make_key((uint32_t)ls[i], lr[i]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ---- operand expansion ------------------------------------------------------

// Four bits (bit i of x) -> four bytes, byte i = 0x38 (e4m3 +1.0) or 0.
__device__ __forceinline__ uint32_t bits4_to_e4m3(uint32_t x) {
    uint32_t b = ((x & 0xFu) * 0x00204081u) & 0x01010101u;  // bit i -> byte i
    return b * 0x38u;
}

// Reference operand: byte l of row r = R_rl ? 0x38 : 0 for l < kpad (the
// packed rows are zero past N).  One thread per 16 output bytes.
__global__ void refs_e4m3_kernel(const uint64_t *__restrict__ packed, int64_t ld64, int64_t n_rows, int32_t kpad,
                                 uint8_t *__restrict__ out) {
    const int64_t per_row = kpad / 16;
    const int64_t total = n_rows * per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / per_row, c = t - r * per_row;
        const int64_t l0 = c * 16;
        const uint64_t w = packed[r * ld64 + (l0 >> 6)];
        const uint32_t bits = (uint32_t)(w >> (l0 & 63)) & 0xFFFFu;
        uint4 o;
        o.x = bits4_to_e4m3(bits);
        o.y = bits4_to_e4m3(bits >> 4);
        o.z = bits4_to_e4m3(bits >> 8);
        o.w = bits4_to_e4m3(bits >> 12);
        reinterpret_cast<uint4 *>(out + r * (int64_t)kpad)[c] = o;
    }
}

// Query operand per mode (see the header comment) and c_q.  One warp per row.
__global__ void queries_e4m3_kernel(const uint64_t *__restrict__ q, int64_t ld_q, int64_t n_q, int32_t n_words,
                                    int32_t n_loci, const uint8_t *__restrict__ modes, int64_t n_q_pad,
                                    int32_t kpad, uint8_t *__restrict__ out, float *__restrict__ qconst) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_q_pad; r += warps_total) {
        const bool valid = r < n_q;
        const bool mis = valid && modes[r] == FASTID_MODE_MISMATCH;
        uint32_t pc = 0;
        for (int32_t c = lane; c < kpad / 16; c += 32) {
            const int32_t l0 = c * 16;
            uint32_t bits = 0;
            if (valid && (l0 >> 6) < n_words) bits = (uint32_t)(q[r * ld_q + (l0 >> 6)] >> (l0 & 63)) & 0xFFFFu;
            // loci < N inside this 16-locus group
            const int32_t live = n_loci - l0;
            const uint32_t in_n = !valid ? 0u : live >= 16 ? 0xFFFFu : live <= 0 ? 0u : ((1u << live) - 1u);
            bits &= in_n;
            pc += __popc(bits);
            uint4 o;
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t qb = (bits >> (4 * i)) & 0xFu;   // Q_l
                const uint32_t nb = (in_n >> (4 * i)) & 0xFu;   // l < N
                // mode 1: 1 - Q_l  -> +1 where l < N and Q_l = 0
                // mode 0: 1 - 2Q_l -> +1 where Q_l = 0, -1 (0xB8 = 0x38 | 0x80) where Q_l = 1
                uint32_t plus = bits4_to_e4m3(nb & ~qb);
                uint32_t minus = mis ? (bits4_to_e4m3(qb) | (((qb * 0x00204081u) & 0x01010101u) * 0x80u)) : 0u;
                w[i] = plus | minus;
            }
            o.x = w[0];
            o.y = w[1];
            o.z = w[2];
            o.w = w[3];
            reinterpret_cast<uint4 *>(out + r * (int64_t)kpad)[c] = o;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
        if (lane == 0) qconst[r] = mis ? (float)pc : 0.f;
    }
}

size_t tensor_smem(int epi) {
    size_t s = 1024 + TC_STAGES * (size_t)(TC_A_BYTES + TC_B_BYTES) + 256;
    if (epi == EPI_TOPK) s += (size_t)32 * TC_BM * sizeof(float);
    return s;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

cudaError_t make_operand_map(CUtensorMap *map, const uint8_t *base, int64_t rows, int32_t kpad, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tensor_tile_q() { return TC_BM; }
int tensor_tile_r() { return TC_BN; }
int tensor_kpad(int32_t n_loci) { return (n_loci + TC_BK - 1) / TC_BK * TC_BK; }

cudaError_t launch_refs_e4m3(const uint64_t *packed, int64_t ld64, int64_t n_rows, int32_t kpad, uint8_t *out,
                             cudaStream_t s) {
    int64_t total = n_rows * (kpad / 16);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    refs_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, ld64, n_rows, kpad, out);
    return cudaGetLastError();
}

cudaError_t launch_queries_e4m3(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words, int32_t n_loci,
                                const uint8_t *modes, int64_t n_q_pad, int32_t kpad, uint8_t *out, float *qconst,
                                cudaStream_t s) {
    int64_t blocks = (n_q_pad + 7) / 8;
    if (blocks > 65535) blocks = 65535;
    queries_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(q, ld_q, n_q, n_words, n_loci, modes, n_q_pad, kpad, out,
                                                         qconst);
    return cudaGetLastError();
}

int tensor_grid_target(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

cudaError_t launch_tensor(int epi, const CUtensorMap &map_a, const CUtensorMap &map_b, int64_t n_refs, int64_t n_q,
                          int32_t kpad, const float *qconst, uint32_t threshold, int32_t k, void *out,
                          int64_t ld_out, int64_t capacity, int64_t *hit_q, int64_t *hit_r, uint32_t *hit_score,
                          unsigned long long *hit_count, uint64_t *partial, const Partition &part, uint32_t *status,
                          cudaStream_t s) {
    TensorArgs a;
    a.n_refs = n_refs;
    a.n_q = n_q;
    a.n_kb = kpad / TC_BK;
    a.qconst = qconst;
    a.threshold = threshold;
    a.k = k;
    a.epi = epi;
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
    size_t smem = tensor_smem(epi);
    cudaError_t e = cudaFuncSetAttribute(tensor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tensor_kernel<<<part.grid, TC_THREADS, smem, s>>>(map_a, map_b, a);
    return cudaGetLastError();
}

}  // namespace fastid
