// Tensor-core form of the overloaded matrix multiply on 5th-generation
// tensor cores (tcgen05), FP32 accumulation in TMEM, with the 0/+-1 operands
// in one of two encodings:
//   FP8   kind::f8f6f4, e4m3 bytes (0x00, 0x38 = +1, 0xB8 = -1), K = 32 a MMA
//   FP4   kind::mxf4 block-scaled, e2m1 nibbles (0x0, 0x2 = +1, 0xA = -1)
//         with every ue8m0 scale factor 2^0, K = 64 a MMA: twice the FP8
//         rate per SM clock on GB300, and a quarter of the FP8 copy's bytes.
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
// Tile: M = 128 queries (TMEM lanes) x N = 256 references (TMEM columns;
// 224 for FP4, whose two accumulators then leave TMEM columns 448-511 for the
// scale factors), K staged one 128-byte swizzle atom per pipeline stage by
// TMA (128 loci in FP8, 256 in FP4).
// Warp roles in a 192-thread CTA, one CTA per SM (persistent):
//   warp 0       TMA producer (one lane)
//   warp 1       TMEM allocation + MMA issue (one lane)
//   warps 2..5   epilogue: TMEM -> registers -> score filter -> per-query
//                top-k (thread = query), hit list or full score matrix
//   warps 6..    packed-reference launches only (PK): expansion of the packed
//                reference stage into the FP8 stage (see expand_stage)
// Two accumulators (2 x 256 TMEM columns) let the epilogue of one reference
// tile overlap the MMAs of the next.  Every mbarrier wait is bounded: on
// timeout the thread records FASTID_ETIMEOUT in the status word and the CTA
// drains and exits.
#include <cuda.h>

#include <cstring>

#include "common.cuh"

namespace fastid {

namespace {

constexpr int TC_BM = 128;          // queries per tile
constexpr int TC_BK = 128;          // loci (bytes) per stage
constexpr int TC_THREADS = 192;     // producer, MMA issuer, 4 epilogue warps
// PK: warps expanding packed references, after the 6 others.  Blocks of 257 to
// 384 threads get at most 168 registers a thread, which the 16-slot top-k
// fits (4 expanding warps) and the 32-slot one does not (2).
__host__ __device__ constexpr int pk_threads(int km) { return km == 16 ? 128 : 64; }
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK;  // 16 KB
// Packed reference stage of PK launches: BN rows of the stage's loci (128
// bits for FP8, 256 for FP4).
__host__ __device__ constexpr uint32_t pk_stage_bytes(int bn, bool f4) { return (uint32_t)bn * (f4 ? 32u : 16u); }
// FP4 launches: reference tiles of 224, unit scale factors in TMEM columns
// TC_SF_COL.. (A's from TC_SF_COL, B's from TC_SF_COL + 16), all lanes.
constexpr int TC_BN4 = 224;
constexpr uint32_t TC_SF_COL = 448;
constexpr uint32_t TC_SF_UNIT = 0x7F7F7F7Fu;  // four ue8m0 bytes of 2^0
constexpr uint64_t WAIT_NS = 2000000000ull;     // 2 s per wait
constexpr uint64_t RENDEZVOUS_NS = 50000000ull;  // 50 ms per panel entry, then go on alone

// Kernel variants: references per tile (the MMA's N) and pipeline depth (as
// many stages as shared memory holds: the pipeline is latency-bound, and on
// GB300 going from 3 to 4 stages took the FP4 2048 x 20M launch from 27.5 to
// 24.5 ms).
//   BN = 256: 32 KB reference stage, 4 stages, 2 x 256 TMEM columns
//   BN = 224: 28 KB reference stage, 5 stages (4 with a packed stage), 2 x 224
//             TMEM columns + scale factors (FP4)
//   BN = 128: 16 KB reference stage, 6 stages, 2 x 128 TMEM columns
//   CG2 (2-SM MMA, see tensor_kernel): each CTA holds half of every reference
//             stage, 7 stages (FP8 32 KB, FP4 30 KB a stage)
template <int BN, bool PK = false, bool CG2 = false>
struct TcShape {
    static constexpr int STAGES = CG2 ? 7 : BN == 128 ? 6 : (BN == 224 && !PK) ? 5 : 4;
    static constexpr uint32_t B_BYTES = (uint32_t)(CG2 ? BN / 2 : BN) * TC_BK;
    static constexpr uint32_t TMEM_COLS = BN == 128 ? 256 : 512;
};

// One database ("panel") of a launch, with its schedule (TcSched).
struct PanelDesc {
    int64_t n_refs;
    int64_t n_q;          // real query rows (the operand is padded to whole tiles)
    int64_t n_rt;         // reference tiles
    int32_t n_kb;         // K stages of 128 operand bytes
    TcSched sc;
    const float *qconst;  // c_q per padded query row
    int32_t qspread;      // see spread_row_to_query
};

struct TcMaps {
    CUtensorMap a[TC_MAXP];  // query operand of each panel (boxes 128 loci x 128 queries)
    // reference operand of each panel: boxes of 128 bytes x BN refs (BN/2 when
    // paired), or, for PK launches, packed boxes of 2 (FP8) or 4 (FP4) words
    // x BN refs
    CUtensorMap b[TC_MAXP];
};

struct TensorArgs {
    int32_t n_panels;
    PanelDesc panel[TC_MAXP];
    int32_t order[TC_MAXP];  // panels in the order every group walks them
    uint32_t threshold;    // already clamped to <= N
    int32_t k;
    int32_t epi;
    void *out;  // EPI_SCORES*: panel 0's [n_q][ld_out]
    int64_t ld_out;
    int64_t capacity;  // EPI_HITS: panel 0
    int64_t *hit_q;
    int64_t *hit_r;
    uint32_t *hit_score;
    unsigned long long *hit_count;
    uint64_t *partial;  // EPI_TOPK: [slots][k][128], see TcSched
    uint32_t *status;
    unsigned int *arrive;  // panel-entry counters (see the producer), or nullptr
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

// Multicast variant: the box lands at the same shared-memory offset in every
// CTA of ctamask and completes bytes on the mbarrier at the same offset there.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *map, uint32_t bar, int32_t x,
                                               int32_t y, uint16_t ctamask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%2, %3}], [%4], %5;"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "h"(ctamask)
        : "memory");
}

// L2 prefetch of one box (no shared-memory destination, no completion).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int32_t x, int32_t y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA in the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The MMA issuer is a whole converged warp: every lane runs its loop and its
// waits, and one lane, picked by elect.sync (the same lane every time in a
// converged warp), issues each tcgen05.mma and tcgen05.commit -- a commit
// tracks the operations of the thread that executes it.  A single lane
// running the loop alone, inside a branch the rest of its warp skips, left
// the tensor pipe idle for ~180 of every ~630 cycles of an FP4 stage.
#define FASTID_ELECT "elect.sync _|e, 0xffffffff;\n\t"

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("{\n\t.reg .pred e;\n\t" FASTID_ELECT
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

// Arrive (when the elected lane's prior tcgen05 operations complete) on the
// mbarrier at the same offset in every CTA of ctamask.
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t ctamask) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t" FASTID_ELECT
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}" ::"r"(
            bar),
        "h"(ctamask)
        : "memory");
}

// ---- 2-SM (cta_group::2) forms: the MMA of a CTA pair issued by its even
// CTA, M = 256 rows (128 in each CTA's shared memory and TMEM), the
// reference operand split along N (half in each CTA's shared memory) ----

// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Arrive on an mbarrier of (possibly) another CTA of the cluster, release
// ordering at cluster scope (bar: a shared::cluster address).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// TMA load into this CTA's shared memory whose completion counts on the
// mbarrier `bar` of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_cg2(uint32_t dst, const CUtensorMap *map, uint32_t bar, int32_t x,
                                                int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Arrive on the mbarrier at the same offset in every CTA of ctamask when the
// elected lane's prior cta_group::2 tcgen05 operations complete.
__device__ __forceinline__ void tc_commit_cg2_mc(uint32_t bar, uint16_t ctamask) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t" FASTID_ELECT
        "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}" ::"r"(
            bar),
        "h"(ctamask)
        : "memory");
}

__device__ __forceinline__ void tc_commit_cg2(uint32_t bar) {
    asm volatile("{\n\t.reg .pred e;\n\t" FASTID_ELECT
                 "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns, every column the value v.
__device__ __forceinline__ void tmem_fill16(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
}

// The 4 MMAs of one 128-byte K stage into accumulator d: operand descriptors
// +0, +2, +4, +6 (32 bytes of K each in the address field), the first MMA
// accumulating only when acc != 0, the others always; one asm block with its
// predicates set once, issued by the warp's elected lane.  At FP4 speed a
// stage is ~450 cycles of MMA work and the tensor pipe holds little more
// than one MMA in its queue, so the issuer's own path between stages (wait,
// descriptors, commit) must stay within about one MMA's time.
template <bool F4, bool CG2>
__device__ __forceinline__ void mma_stage4(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t sfa,
                                           uint32_t sfb, uint32_t acc) {
    const uint64_t a1 = ad + 2u, a2 = ad + 4u, a3 = ad + 6u, b1 = bd + 2u, b2 = bd + 4u, b3 = bd + 6u;
    if constexpr (F4) {
#define FASTID_MMA4_F4(CG)                                                                                         \
    asm volatile("{\n\t.reg .pred p, q, e;\n\t" FASTID_ELECT                                                                    \
                 "setp.ne.b32 p, %12, 0;\n\t"                                                                  \
                 "setp.ne.b32 q, %12, 0xFFFFFFFF;\n\t"                                                         \
                 "@e tcgen05.mma.cta_group::" CG ".kind::mxf4.block_scale.scale_vec::2X [%0], %1, %5, %9, [%10], [%11], p;\n\t" \
                 "@e tcgen05.mma.cta_group::" CG ".kind::mxf4.block_scale.scale_vec::2X [%0], %2, %6, %9, [%10], [%11], q;\n\t" \
                 "@e tcgen05.mma.cta_group::" CG ".kind::mxf4.block_scale.scale_vec::2X [%0], %3, %7, %9, [%10], [%11], q;\n\t" \
                 "@e tcgen05.mma.cta_group::" CG ".kind::mxf4.block_scale.scale_vec::2X [%0], %4, %8, %9, [%10], [%11], q;\n\t}" \
                 ::"r"(d), "l"(ad), "l"(a1), "l"(a2), "l"(a3), "l"(bd), "l"(b1), "l"(b2), "l"(b3), "r"(idesc),      \
                 "r"(sfa), "r"(sfb), "r"(acc)                                                                     \
                 : "memory")
        if constexpr (CG2)
            FASTID_MMA4_F4("2");
        else
            FASTID_MMA4_F4("1");
#undef FASTID_MMA4_F4
    } else {
        (void)sfa;
        (void)sfb;
#define FASTID_MMA4_F8(CG)                                                                                         \
    asm volatile("{\n\t.reg .pred p, q, e;\n\t" FASTID_ELECT                                                                    \
                 "setp.ne.b32 p, %10, 0;\n\t"                                                                  \
                 "setp.ne.b32 q, %10, 0xFFFFFFFF;\n\t"                                                         \
                 "@e tcgen05.mma.cta_group::" CG ".kind::f8f6f4 [%0], %1, %5, %9, p;\n\t"                          \
                 "@e tcgen05.mma.cta_group::" CG ".kind::f8f6f4 [%0], %2, %6, %9, q;\n\t"                          \
                 "@e tcgen05.mma.cta_group::" CG ".kind::f8f6f4 [%0], %3, %7, %9, q;\n\t"                          \
                 "@e tcgen05.mma.cta_group::" CG ".kind::f8f6f4 [%0], %4, %8, %9, q;\n\t}"                         \
                 ::"r"(d), "l"(ad), "l"(a1), "l"(a2), "l"(a3), "l"(bd), "l"(b1), "l"(b2), "l"(b3), "r"(idesc),      \
                 "r"(acc)                                                                                         \
                 : "memory")
        if constexpr (CG2)
            FASTID_MMA4_F8("2");
        else
            FASTID_MMA4_F8("1");
#undef FASTID_MMA4_F8
    }
}

// 32 lanes x one 32-bit column (every lane its own row).
__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return v;
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

// Instruction descriptor, kind::mxf4 (block-scaled): B scale-factor id 0
// (bits 4-5), A = B = E2M1 (1 at bits 7 and 10), both K-major, N >> 3 at bit
// 17, scale type UE8M0 (bit 23), M >> 4 at bit 24 (for M = 128 the same bit
// as M >> 7 at bit 27), A scale-factor id 0 (bits 29-30), K = 64 (bit 31 = 0).
__host__ __device__ constexpr uint32_t idesc_mxf4(int m, int n) {
    return (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (1u << 23) | ((uint32_t)(m >> 4) << 24);
}

// Per-thread top-k list held in registers, ascending by score; entries of
// equal score keep arrival order (references arrive in increasing order, so
// the earlier entry has the lower index).  Inserting (xs, xr) is a fixed
// compare-select network, so all lanes of a warp insert in lock-step; a lane
// with nothing to insert passes xs = INT32_MAX, which changes nothing.
// The network has KM slots (16 or 32, chosen per launch from k).  For a
// runtime k <= KM the first KM - k slots hold INT32_MIN place-holders that
// nothing displaces, so the k kept entries sit in slots KM-k .. KM-1 and the
// k-th smallest is always slot KM-1 (static register indices only).
constexpr int TC_KMAX = 32;
constexpr int32_t NET_EMPTY = 0x7fffffff;
constexpr int32_t NET_HOLD = (int32_t)0x80000000;

template <int KM>
__device__ __forceinline__ void net_insert(int32_t (&ls)[KM], uint32_t (&lr)[KM], int32_t xs, uint32_t xr) {
#pragma unroll
    for (int i = KM - 1; i > 0; --i) {
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
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t bfull[8];  // PK: reference stage expanded
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

// Panel-entry rendezvous.  Groups that share a reference slice read its
// tiles through L2 only while they walk it in step; entering a panel at
// different times (the previous panel's drift) breaks that.  So each CTA's
// producer counts itself in at every panel after the first and, if it has
// work there, waits for the whole grid before loading the panel's tiles.
// It is a hint, not a barrier the results depend on: the wait gives up
// after RENDEZVOUS_NS (a CTA that is not resident, or one that aborted) and
// the producer goes on alone.
__device__ __forceinline__ void panel_rendezvous(unsigned int *ctr, bool wait) {
    atomicAdd(ctr, 1u);
    if (!wait) return;
    const unsigned int n = gridDim.x;
    const uint64_t t0 = globaltimer();
    for (;;) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= n || globaltimer() - t0 > RENDEZVOUS_NS) return;
        __nanosleep(200);
    }
}

// The work of one group (see TcSched) in panel p: reference tiles
// [r_lo, r_hi) walked in chunks, query tiles (pairs) [q_lo, q_hi), top-k
// slots from slot (this CTA's first; one per query tile).  Empty
// (q_lo == q_hi) when the panel's grid and tail have no group wg.
struct GroupWork {
    int64_t r_lo, r_hi;
    int32_t q_lo, q_hi, chunk;
    int64_t slot;
};

// cpg: CTAs per group (2 when paired), rank: this CTA's rank in its group.
__device__ __forceinline__ GroupWork group_work(const TensorArgs &a, int64_t wg, int p, int cpg, int rank) {
    GroupWork w;
    w.r_lo = w.r_hi = 0;
    w.q_lo = w.q_hi = 0;
    w.chunk = 1;
    w.slot = 0;
    const TcSched &sc = a.panel[p].sc;
    const int64_t grid = (int64_t)sc.a * sc.b;
    if (sc.n_qq <= 0) return w;
    if (wg < grid) {
        const int64_t x = wg / sc.b, y = wg - x * sc.b;
        w.r_lo = y * (int64_t)sc.r_main / sc.b;
        w.r_hi = (y + 1) * (int64_t)sc.r_main / sc.b;
        w.q_lo = (int32_t)(x * sc.tpx);
        w.q_hi = (int32_t)min((int64_t)sc.n_qq, (x + 1) * sc.tpx);
        w.chunk = sc.chunk;
        w.slot = (int64_t)sc.slot0 + (wg * cpg + rank) * sc.tpx;
    } else if (wg < grid + sc.t_groups) {
        const int64_t t = wg - grid;
        w.r_lo = sc.r_main;
        w.r_hi = a.panel[p].n_rt;
        w.q_lo = (int32_t)min((int64_t)sc.n_qq, t * sc.t_tpx);
        w.q_hi = (int32_t)min((int64_t)sc.n_qq, (t + 1) * sc.t_tpx);
        w.chunk = sc.t_chunk;
        w.slot = (int64_t)sc.slot0 + grid * cpg * sc.tpx + (t * cpg + rank) * sc.t_tpx;
    }
    return w;
}

// Save / resume one thread's top-k list.  Slot layout [slot][k][128]: entry i
// of the 128 rows is contiguous, so a warp's accesses coalesce.  Keys
// ascending, empty entries KEY_EMPTY.
template <int KM>
__device__ __forceinline__ void list_save(uint64_t *slot_row, const int32_t (&ls)[KM], const uint32_t (&lr)[KM],
                                          int k) {
#pragma unroll
    for (int i = 0; i < KM; ++i)
        if (i >= KM - k)
            slot_row[(int64_t)(i - (KM - k)) * TC_BM] =
                ls[i] == NET_EMPTY ? KEY_EMPTY : make_key((uint32_t)ls[i], lr[i]);
}

template <int KM>
__device__ __forceinline__ void list_load(const uint64_t *slot_row, int32_t (&ls)[KM], uint32_t (&lr)[KM], int k) {
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        if (i >= KM - k) {
            const uint64_t key = slot_row[(int64_t)(i - (KM - k)) * TC_BM];
            ls[i] = key == KEY_EMPTY ? NET_EMPTY : (int32_t)(key >> 32);
            lr[i] = (uint32_t)key;
        } else {
            ls[i] = NET_HOLD;
            lr[i] = 0xFFFFFFFFu;
        }
    }
}

// PK launches: the reference operand arrives packed (TC_P_BYTES per stage,
// row r at r * 16 bytes: loci 0-63 then 64-127 of the stage) and warps 6.. (pk_threads)
// expand it into the FP8 stage the MMA reads.  A reference "1" is e4m3 2.0
// (byte 0x40) and the query operand is encoded at half scale (+-0.5), so D is
// unchanged.
//
// Locus order.  D sums over loci, so both operands may list the loci of a
// 32-locus group in any common order.  PK uses the order that makes expansion
// cheapest: byte 4j + k of the group holds locus 8k + j (j = 0..7, k = 0..3).
// Then the four bytes 4j .. 4j+3 are bit j of each byte of the group's packed
// word w, moved to bit 6 by one shift and kept by one mask:
// (w << (6 - j)) & 0x40404040 (no other bit reaches a bit 6).  The query
// operand of PK launches is written in the same order (encode_query_row).
// The stage layout is the TMA's 128-byte swizzle: 16-byte chunk c of row r
// sits at r * 128 + ((c ^ (r & 7)) << 4) from a 1024-byte aligned base.
constexpr uint32_t PK_BIT6 = 0x40404040u;

template <int NT>
__device__ __forceinline__ void expand_stage(const uint8_t *sp, uint8_t *sb, int t) {
#pragma unroll
    for (int rr = 0; rr < 256 / NT; ++rr) {
        const int r = t + NT * rr;
        const uint2 lo = *reinterpret_cast<const uint2 *>(sp + r * 16);
        const uint2 hi = *reinterpret_cast<const uint2 *>(sp + r * 16 + 8);
        const uint32_t w[4] = {lo.x, lo.y, hi.x, hi.y};  // 32 loci each
#pragma unroll
        for (int m = 0; m < 4; ++m) {  // chunks 2m (j = 0..3) and 2m + 1 (j = 4..7) of group m
            const uint32_t x = w[m];
            const uint4 o0 = make_uint4((x << 6) & PK_BIT6, (x << 5) & PK_BIT6, (x << 4) & PK_BIT6,
                                        (x << 3) & PK_BIT6);
            const uint4 o1 = make_uint4((x << 2) & PK_BIT6, (x << 1) & PK_BIT6, x & PK_BIT6, (x >> 1) & PK_BIT6);
            *reinterpret_cast<uint4 *>(sb + r * 128 + (((2 * m) ^ (r & 7)) << 4)) = o0;
            *reinterpret_cast<uint4 *>(sb + r * 128 + (((2 * m + 1) ^ (r & 7)) << 4)) = o1;
        }
    }
}

// FP4 (PK launches): the stage holds 256 loci of each reference row (4
// packed words, row r at r * 32 bytes) and each 32-locus word becomes one
// 16-byte chunk of e2m1 nibbles, in the same 128-byte swizzle.  Locus order
// inside a chunk: nibble n of its 32-bit word j holds locus 4n + j, so word j
// is bit j of every nibble of the packed word w moved to bit 1 (e2m1 +1.0 =
// 0x2) by one shift and kept by one mask.  The query operand of every FP4
// launch is written in the same order (encode_query_row_f4), and so is the
// database's FP4 copy (refs_e2m1_kernel).
constexpr uint32_t PK4_BIT1 = 0x22222222u;

// Work unit u = one half row (row u / 2, words 4 (u % 2) .. 4 (u % 2) + 3),
// so that a warp reads 512 consecutive bytes of the packed stage -- a thread
// per row read at a 32-byte stride and took twice the shared-memory
// wavefronts -- and each 16-byte chunk store of a warp still meets every bank
// group four times; a thread's loads all go first.  (64 queries x 20M:
// 2.21 -> 2.07 ms at k = 16, 2.83 -> 2.40 ms at k = 32.)
template <int NT, int BN>
__device__ __forceinline__ void expand_stage_f4(const uint8_t *sp, uint8_t *sb, int t) {
    constexpr int ITER = (2 * BN + NT - 1) / NT;
    uint4 xs[ITER];  // every load first, so that their latencies overlap
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int u = t + it * NT;
        if (u < 2 * BN) xs[it] = *reinterpret_cast<const uint4 *>(sp + u * 16);
    }
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int u = t + it * NT;
        if (u >= 2 * BN) break;
        const int r = u >> 1, h = u & 1;
        const uint4 x4 = xs[it];
        const uint32_t w[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = 4 * h + i;
            const uint32_t x = w[i];
            const uint4 o = make_uint4((x << 1) & PK4_BIT1, x & PK4_BIT1, (x >> 1) & PK4_BIT1, (x >> 2) & PK4_BIT1);
            *reinterpret_cast<uint4 *>(sb + r * 128 + ((c ^ (r & 7)) << 4)) = o;
        }
    }
}

// PAIR: 2-CTA clusters; both CTAs walk the same reference tiles for the two
// query tiles of a pair (rank r takes tile 2 qq + r), and each multicasts half
// of every reference stage into both CTAs' shared memory.
// PK: packed reference operand expanded on chip (see expand_stage).
// F4: block-scaled FP4 operands (kind::mxf4, BN = 224); else FP8 (BN = 256 or 128).
// CG2 (with PAIR): the pair's MMA is one 2-SM tcgen05.mma (cta_group::2, M =
// 256) issued by the even CTA: each CTA loads its own query tile and HALF of
// every reference stage into its own shared memory (no multicast), the
// tensor cores of both SMs read both halves, and each CTA's TMEM receives
// its own 128 query rows x BN references.  A stage then costs each SM 16 KB
// of queries + BN/2 references' bytes instead of the whole reference stage,
// which leaves room for 7 stages.  Both CTAs' loads complete on the even
// CTA's full barrier; its commits release both CTAs' stages and accumulators;
// both epilogues release an accumulator on the even CTA's barrier.
template <int BN, bool PAIR, int KM, bool PK, bool F4, bool CG2 = false>
__global__ void __launch_bounds__(PK ? TC_THREADS + pk_threads(KM) : TC_THREADS, 1)
    tensor_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ TensorArgs args) {
    using S = TcShape<BN, PK, CG2>;
    static_assert(!CG2 || (PAIR && !PK), "2-SM MMA launches are paired, over an operand copy");
    static_assert(F4 ? BN == TC_BN4 : BN != TC_BN4, "FP4 launches use 224-reference tiles, FP8 ones 256 or 128");
    static_assert(!PAIR || BN != 128, "paired launches use 256- or 224-reference tiles");
    static_assert(!PK || (BN != 128 && !PAIR), "packed-reference launches use unpaired 256- or 224-reference tiles");
    constexpr uint32_t P_BYTES = pk_stage_bytes(BN, F4);
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand stages (queries, references, and for PK the
    // packed reference stages), then the control block, then staging.
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t *base = smem_raw + pad;
    uint8_t *sA = base;
    uint8_t *sB = base + S::STAGES * TC_A_BYTES;
    uint8_t *sP = base + S::STAGES * (TC_A_BYTES + S::B_BYTES);  // PK only
    TcSmem *ctl = reinterpret_cast<TcSmem *>(sP + (PK ? S::STAGES * P_BYTES : 0));

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t c = blockIdx.x;                     // this CTA: owner of top-k slots
    const int rank = PAIR ? (int)cluster_rank() : 0;
    const int64_t wg = PAIR ? (c >> 1) : c;            // work group: cluster or CTA
    volatile int *abort_flag = &ctl->abort_flag;

    if (tid == 0) {
        for (int s = 0; s < S::STAGES; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), 1);
            // multicast pairs: both CTAs' MMAs release a stage; 2-SM pairs: the even CTA's MMA
            mbar_init(smem_u32(&ctl->empty[s]), (PAIR && !CG2) ? 2 : 1);
            if (PK) mbar_init(smem_u32(&ctl->bfull[s]), pk_threads(KM));  // every expanding thread
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->tfull[a]), 1);
            mbar_init(smem_u32(&ctl->tempty[a]), CG2 ? 256 : 128);  // 2-SM: both CTAs' epilogues
        }
        mbar_init(smem_u32(&ctl->done), 1);
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if (CG2) {  // one warp of each CTA of the pair, together: the same columns in both
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&ctl->tmem_base)),
                         "r"(S::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&ctl->tmem_base)),
                         "r"(S::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();  // the peer's barriers exist before any multicast targets them
    tc_fence_after();
    const uint32_t tmem_base = ctl->tmem_base;
    if (F4) {
        // unit scale factors: TMEM columns TC_SF_COL .. TC_SF_COL + 63 of every
        // lane (each epilogue warp fills its lane quadrant) before any MMA
        if (warp >= 2 && warp < 6) {
            const uint32_t t = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + TC_SF_COL;
#pragma unroll
            for (int c = 0; c < 64; c += 16) tmem_fill16(t + c, TC_SF_UNIT);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        // Per stage: one wait for the slot (inline when it is already free),
        // the expected bytes, the loads at stage offsets from the first slot and
        // coordinates fixed per reference tile (a short path, like the MMA
        // issuer's, so that the producer keeps up at FP4 speed).
        if (lane == 0) {
            const uint32_t full0 = smem_u32(&ctl->full[0]), empty0 = smem_u32(&ctl->empty[0]);
            const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB), sP0 = smem_u32(sP);
            // this CTA's reference rows of a (paired) tile start at rt * BN + boff
            const int32_t boff = PAIR ? rank * (BN / 2) : 0;
            // bytes landing on a full barrier: 2-SM pairs count both CTAs' loads
            // on the even CTA's; multicast pairs both halves on each CTA's
            constexpr uint32_t TX = CG2 ? 2 * (TC_A_BYTES + S::B_BYTES) : TC_A_BYTES + (PK ? P_BYTES : S::B_BYTES);
            uint32_t stage = 0;
            uint32_t phase = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int pi = 0; pi < args.n_panels && ok; ++pi) {
                const int p = args.order[pi];
                const GroupWork W = group_work(args, wg, p, PAIR ? 2 : 1, rank);
                if (pi > 0 && args.arrive) panel_rendezvous(args.arrive + pi, W.q_lo < W.q_hi);
                if (W.q_lo >= W.q_hi) continue;
                const CUtensorMap *ma = &maps.a[p];
                const CUtensorMap *mb = &maps.b[p];
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(ma)) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mb)) : "memory");
                const int n_kb = args.panel[p].n_kb;
                const bool pf = args.panel[p].sc.pf != 0 && W.q_hi - W.q_lo == 1;
                for (int64_t rc = W.r_lo; rc < W.r_hi && ok; rc += W.chunk) {
                    const int64_t re = min(rc + W.chunk, W.r_hi);
                    for (int32_t qq = W.q_lo; qq < W.q_hi && ok; ++qq) {
                        const int32_t ya = (int32_t)((PAIR ? 2 * (int64_t)qq + rank : (int64_t)qq) * TC_BM);
                        for (int64_t rt = rc; rt < re && ok; ++rt) {
                            const int32_t yb = (int32_t)(rt * BN) + boff;
                            // A group with one query tile streams its slice once: fetch the
                            // next reference tile into L2 while this one is consumed, so the
                            // group that reaches a tile first does not wait on DRAM (where
                            // the schedule enables it, see TcSched::pf).
                            const bool pft = !PK && pf && rt + 1 < W.r_hi;
                            for (int kb = 0; kb < n_kb; ++kb) {
                                const uint32_t eb = empty0 + 8u * stage;
                                if (!mbar_try_wait(eb, phase ^ 1u)) {
                                    ok = mbar_wait(eb, phase ^ 1u, abort_flag, args.status, 1);
                                    if (!ok) break;
                                }
                                const uint32_t fb = full0 + 8u * stage;
                                const int32_t x = kb * TC_BK;
                                if (CG2) {
                                    // both CTAs' bytes complete on the even CTA's full barrier
                                    const uint32_t fb0 = mapa_rank(fb, 0);
                                    if (rank == 0) mbar_expect_tx(fb, TX);
                                    tma_load_2d_cg2(sA0 + stage * TC_A_BYTES, ma, fb0, x, ya);
                                    tma_load_2d_cg2(sB0 + stage * S::B_BYTES, mb, fb0, x, yb);
                                } else {
                                    mbar_expect_tx(fb, TX);
                                    tma_load_2d(sA0 + stage * TC_A_BYTES, ma, fb, x, ya);
                                    if (PK)  // the stage's loci as packed words (2 FP8, 4 FP4) x BN references
                                        tma_load_2d(sP0 + stage * P_BYTES, mb, fb, kb * (F4 ? 4 : 2), yb);
                                    else if (PAIR)  // this CTA's half, into both CTAs
                                        tma_load_2d_mc(sB0 + stage * S::B_BYTES + rank * (S::B_BYTES / 2), mb, fb, x, yb,
                                                       (uint16_t)0x3);
                                    else
                                        tma_load_2d(sB0 + stage * S::B_BYTES, mb, fb, x, yb);
                                }
                                if (pft) tma_prefetch_2d(mb, x, yb + BN);
                                ++issued;
                                if (++stage == S::STAGES) {
                                    stage = 0;
                                    phase ^= 1u;
                                }
                            }
                        }
                    }
                }
            }
            // Drain: the last fill of every stage has landed before the CTA
            // exits (fill n used stage n % S in phase (n / S) & 1).
            for (int64_t n = issued - 1; n >= 0 && n >= issued - S::STAGES; --n) {
                // (2-SM pairs: the even CTA's full barriers count both CTAs' fills)
                if (!CG2 || rank == 0)
                    mbar_drain(smem_u32(&ctl->full[n % S::STAGES]), (uint32_t)((n / S::STAGES) & 1), args.status, 2);
                // paired: both MMAs' releases of this stage (the peer's arrive
                // remotely) have landed before the CTA exits
                if (PAIR)
                    mbar_drain(smem_u32(&ctl->empty[n % S::STAGES]), (uint32_t)((n / S::STAGES) & 1), args.status, 7);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (2-SM pairs: the even CTA's) ----------------
        // The whole warp, converged; one elected lane issues (see tc_commit).
        // Per stage: one barrier wait (inline when the stage is already full),
        // the stage's descriptors as constant offsets from the first stage's,
        // four MMAs in one asm block, one commit (see mma_stage4).
        if (!CG2 || rank == 0) {
            constexpr int MM = CG2 ? 2 * TC_BM : TC_BM;
            constexpr uint32_t idesc = F4 ? idesc_mxf4(MM, BN) : idesc_f8(MM, BN);
            constexpr uint32_t A_STEP = TC_A_BYTES >> 4, B_STEP = S::B_BYTES >> 4;  // descriptor units a stage
            const uint64_t ad0 = sw128_desc(smem_u32(sA)), bd0 = sw128_desc(smem_u32(sB));
            const uint32_t full0 = smem_u32(&ctl->full[0]), empty0 = smem_u32(&ctl->empty[0]);
            const uint32_t bfull0 = smem_u32(&ctl->bfull[0]);
            const uint32_t sfa = tmem_base + TC_SF_COL, sfb = tmem_base + TC_SF_COL + 16;
            uint32_t stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int pi = 0; pi < args.n_panels && ok; ++pi) {
                const int p = args.order[pi];
                const GroupWork W = group_work(args, wg, p, PAIR ? 2 : 1, rank);
                if (W.q_lo >= W.q_hi) continue;
                const int n_kb = args.panel[p].n_kb;
                for (int64_t rc = W.r_lo; rc < W.r_hi && ok; rc += W.chunk) {
                    const int64_t re = min(rc + W.chunk, W.r_hi);
                    for (int32_t qq = W.q_lo; qq < W.q_hi && ok; ++qq) {
                        for (int64_t rt = rc; rt < re && ok; ++rt) {
                            const uint32_t tempty = smem_u32(&ctl->tempty[acc]);
                            if (!mbar_try_wait(tempty, acc_phase ^ 1u)) {
                                ok = mbar_wait(tempty, acc_phase ^ 1u, abort_flag, args.status, 3);
                                if (!ok) break;
                            }
                            tc_fence_after();  // the epilogue's reads of this accumulator come first
                            const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                            for (int kb = 0; kb < n_kb; ++kb) {
                                const uint32_t fb = full0 + 8u * stage;
                                if (!mbar_try_wait(fb, phase)) {
                                    ok = mbar_wait(fb, phase, abort_flag, args.status, 4);
                                    if (!ok) break;
                                }
                                if (PK && !mbar_try_wait(bfull0 + 8u * stage, phase)) {
                                    ok = mbar_wait(bfull0 + 8u * stage, phase, abort_flag, args.status, 8);
                                    if (!ok) break;
                                }
                                // (the stage's operands were written by TMA, or by the expanding
                                // warps behind an async-proxy fence, and are ordered by the barrier)
                                mma_stage4<F4, CG2>(d_tmem, ad0 + stage * A_STEP, bd0 + stage * B_STEP, idesc, sfa,
                                                    sfb, kb != 0);
                                const uint32_t eb = empty0 + 8u * stage;
                                if (CG2)
                                    tc_commit_cg2_mc(eb, (uint16_t)0x3);
                                else if (PAIR)
                                    tc_commit_mc(eb, (uint16_t)0x3);
                                else
                                    tc_commit(eb);
                                if (++stage == S::STAGES) {
                                    stage = 0;
                                    phase ^= 1u;
                                }
                            }
                            if (!ok) break;
                            if (CG2)  // both CTAs' accumulators are full
                                tc_commit_cg2_mc(smem_u32(&ctl->tfull[acc]), (uint16_t)0x3);
                            else
                                tc_commit(smem_u32(&ctl->tfull[acc]));
                            if (++acc == 2) {
                                acc = 0;
                                acc_phase ^= 1u;
                            }
                        }
                    }
                }
            }
            // Drain: a commit completes after every MMA this thread issued.
            if (CG2)
                tc_commit_cg2(smem_u32(&ctl->done));
            else
                tc_commit(smem_u32(&ctl->done));
            mbar_drain(smem_u32(&ctl->done), 0, args.status, 5);
        }
    } else if (PK && warp >= 6) {
        // ---------------- PK: reference expansion, warps 6.. ----------------
        const int t = tid - 192;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int pi = 0; pi < args.n_panels && ok; ++pi) {
            const int p = args.order[pi];
            const GroupWork W = group_work(args, wg, p, PAIR ? 2 : 1, rank);
            if (W.q_lo >= W.q_hi) continue;
            const int n_kb = args.panel[p].n_kb;
            for (int64_t rc = W.r_lo; rc < W.r_hi && ok; rc += W.chunk) {
                const int64_t re = min(rc + W.chunk, W.r_hi);
                for (int32_t qq = W.q_lo; qq < W.q_hi && ok; ++qq) {
                    for (int64_t rt = rc; rt < re && ok; ++rt) {
                        for (int kb = 0; kb < n_kb; ++kb) {
                            ok = mbar_wait(smem_u32(&ctl->full[stage]), phase, abort_flag, args.status, 9);
                            if (!ok) break;
                            if (F4)
                                expand_stage_f4<pk_threads(KM), BN>(sP + stage * P_BYTES, sB + stage * S::B_BYTES, t);
                            else
                                expand_stage<pk_threads(KM)>(sP + stage * P_BYTES, sB + stage * S::B_BYTES, t);
                            // generic-proxy writes, read next by the tensor core (async proxy)
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            mbar_arrive(smem_u32(&ctl->bfull[stage]));
                            if (++stage == S::STAGES) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;            // TMEM lane quadrant this warp may access
        const int row = quad * 32 + lane;     // query row within the tile
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const float tplus1 = args.threshold == 0xFFFFFFFFu ? __int_as_float(0x7f800000) : (float)args.threshold + 1.0f;
        const int k = args.k;
        const bool topk = args.epi == EPI_TOPK;
        int acc = 0;
        uint32_t acc_phase = 0;
        int32_t ls[KM];   // this thread's top-k scores (see net_insert)
        uint32_t lr[KM];  // and their references
        bool ok = true;
        for (int pi = 0; pi < args.n_panels && ok; ++pi) {
            const int p = args.order[pi];
            const GroupWork W = group_work(args, wg, p, PAIR ? 2 : 1, rank);
            if (W.q_lo >= W.q_hi) continue;
            const PanelDesc &P = args.panel[p];
            const int64_t n_refs = P.n_refs;
            for (int64_t rc = W.r_lo; rc < W.r_hi && ok; rc += W.chunk) {
                const int64_t re = min(rc + W.chunk, W.r_hi);
                for (int32_t qq = W.q_lo; qq < W.q_hi && ok; ++qq) {
                    const int64_t qt = PAIR ? 2 * (int64_t)qq + rank : qq;
                    const int64_t qr = qt * TC_BM + row;                     // operand row
                    const int64_t q = spread_row_to_query(qr, P.qspread);  // input query
                    const bool qvalid = q < P.n_q;
                    const float cq = P.qconst[qr];
                    const float cut0 = qvalid ? tplus1 - cq : -__int_as_float(0x7f800000);
                    uint64_t *slot = args.partial + (W.slot + (qq - W.q_lo)) * (int64_t)k * TC_BM + row;
                    if (topk && rc > W.r_lo) {
                        list_load(slot, ls, lr, k);
                    } else {
#pragma unroll
                        for (int i = 0; i < KM; ++i) {
                            ls[i] = i < KM - k ? NET_HOLD : NET_EMPTY;
                            lr[i] = 0xFFFFFFFFu;
                        }
                    }
                    float cut = ls[KM - 1] == NET_EMPTY ? cut0 : (float)ls[KM - 1] - cq;
                    for (int64_t rt = rc; rt < re; ++rt) {
                        const bool got = mbar_wait(smem_u32(&ctl->tfull[acc]), acc_phase, abort_flag, args.status, 6);
                        __syncwarp();
                        if (!__all_sync(0xffffffffu, got)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int64_t r0 = rt * BN;
                        const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * BN);
#pragma unroll 1
                        for (int ch = 0; ch < BN / 32; ++ch) {
                            uint32_t v[32];
                            __syncwarp();  // tcgen05.ld is warp-collective: reconverge first
                            tmem_ld32(taddr + ch * 32, v);
                            const int64_t rch = r0 + ch * 32;
                            if (args.epi == EPI_SCORES16 || args.epi == EPI_SCORES32) {
                                if (qvalid) {
#pragma unroll
                                    for (int j = 0; j < 32; ++j) {
                                        const int64_t r = rch + j;
                                        if (r < n_refs) {
                                            const uint32_t sc = (uint32_t)(int32_t)(__uint_as_float(v[j]) + cq);
                                            if (args.epi == EPI_SCORES16)
                                                reinterpret_cast<uint16_t *>(args.out)[q * args.ld_out + r] =
                                                    (uint16_t)sc;
                                            else
                                                reinterpret_cast<uint32_t *>(args.out)[q * args.ld_out + r] = sc;
                                        }
                                    }
                                }
                                continue;
                            }
                            // Common case first: nothing in the chunk beats the cut
                            // (the chunk's minimum, by a tree of fminf).
                            float mn[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) mn[j] = fminf(__uint_as_float(v[j]), __uint_as_float(v[j + 16]));
#pragma unroll
                            for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                                for (int j = 0; j < w; ++j) mn[j] = fminf(mn[j], mn[j + w]);
                            if (!__any_sync(0xffffffffu, mn[0] < cut)) continue;
                            uint32_t m = 0;  // columns of this chunk that pass the filter
#pragma unroll
                            for (int j = 0; j < 32; ++j) m |= (uint32_t)(__uint_as_float(v[j]) < cut) << j;
                            if (rch + 32 > n_refs) m &= rch >= n_refs ? 0u : ((1u << (n_refs - rch)) - 1u);
                            if (!__any_sync(0xffffffffu, m != 0u)) continue;
                            if (args.epi == EPI_HITS) {
#pragma unroll
                                for (int j = 0; j < 32; ++j)
                                    if (m & (1u << j))
                                        append_hit(args.hit_count, args.capacity, args.hit_q, args.hit_r,
                                                   args.hit_score, q, rch + j,
                                                   (uint32_t)(int32_t)(__uint_as_float(v[j]) + cq));
                                continue;
                            }
                            // rare path: insert the candidates in lock-step, column by
                            // column in increasing order (so each lane inserts its own
                            // in increasing reference order); a column some lane needs
                            // is re-read from TMEM by the whole warp (the accumulator
                            // is released only after the tile, below)
                            uint32_t mm = __reduce_or_sync(0xffffffffu, m);
                            while (mm != 0u) {
                                const int j = __ffs(mm) - 1;
                                mm &= mm - 1u;
                                const float d = __uint_as_float(tmem_ld1(taddr + ch * 32 + j));
                                int32_t xs = NET_EMPTY;
                                uint32_t xr = 0u;
                                if (((m >> j) & 1u) && d < cut) {
                                    xs = (int32_t)(d + cq);
                                    xr = (uint32_t)(rch + j);
                                }
                                net_insert(ls, lr, xs, xr);
                                cut = ls[KM - 1] == NET_EMPTY ? cut0 : (float)ls[KM - 1] - cq;
                            }
                        }
                        // every column of the tile is processed: the MMA may reuse the accumulator
                        tc_fence_before();
                        if (CG2)  // on the even CTA's barrier
                            mbar_arrive_cluster(mapa_rank(smem_u32(&ctl->tempty[acc]), 0));
                        else
                            mbar_arrive(smem_u32(&ctl->tempty[acc]));
                        if (++acc == 2) {
                            acc = 0;
                            acc_phase ^= 1u;
                        }
                    }
                    if (topk && ok) list_save(slot, ls, lr, k);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();  // neither CTA leaves while the other may still address it
    tc_fence_after();
    if (warp == 1) {
        if (CG2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(S::TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(S::TMEM_COLS)
                         : "memory");
    }
}

// ---- operand expansion ------------------------------------------------------

// Four bits (bit i of x) -> four bytes, byte i = 0x38 (e4m3 +1.0) or 0.
__device__ __forceinline__ uint32_t bits4_to_e4m3(uint32_t x) {
    uint32_t b = ((x & 0xFu) * 0x00204081u) & 0x01010101u;  // bit i -> byte i
    return b * 0x38u;
}

// Reference operand: byte l of row r = R_rl ? 0x38 : 0 for l < kpad, from
// packed rows at stride ld64 of which the first n_src rows and n_words words
// exist (zero elsewhere: padding rows and loci).  One thread per 16 output
// bytes; streaming loads and stores (each byte is touched once, and the
// operand is larger than L2), so that a concurrent comparison keeps its L2.
__global__ void refs_e4m3_kernel(const uint64_t *__restrict__ packed, int64_t ld64, int64_t n_src, int32_t n_words,
                                 int64_t n_rows, int32_t kpad, uint8_t *__restrict__ out) {
    const int64_t per_row = kpad / 16;
    const int64_t total = n_rows * per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / per_row, c = t - r * per_row;
        const int64_t l0 = c * 16;
        const int32_t wi = (int32_t)(l0 >> 6);
        const uint64_t w = (r < n_src && wi < n_words) ? __ldcs(packed + r * ld64 + wi) : 0ull;
        const uint32_t bits = (uint32_t)(w >> (l0 & 63)) & 0xFFFFu;
        uint4 o;
        o.x = bits4_to_e4m3(bits);
        o.y = bits4_to_e4m3(bits >> 4);
        o.z = bits4_to_e4m3(bits >> 8);
        o.w = bits4_to_e4m3(bits >> 12);
        __stcs(reinterpret_cast<uint4 *>(out + r * (int64_t)kpad) + c, o);
    }
}

// Query operand per mode (see the header comment) and c_q for one row, by one
// warp.  src == nullptr (a padding row) writes zeros.
// `one` is the e4m3 byte of +1 on this operand's scale: 0x38 (1.0) against the
// FP8 reference operand, 0x30 (0.5) against PK's expanded references (2.0).
// pk: PK's locus order (see expand_stage), else loci in order.
__device__ __forceinline__ void encode_query_row(const uint64_t *__restrict__ src, bool mis, int32_t n_words,
                                                 int32_t n_loci, int32_t kpad, uint8_t *__restrict__ dst,
                                                 float *__restrict__ qc, int lane, uint32_t one = 0x38u,
                                                 bool pk = false) {
    const bool valid = src != nullptr;
    uint32_t pc = 0;
    if (pk) {
        // chunk c: words i = 0..3 hold j = 4 (c & 1) + i; byte k of word i is
        // locus 32 (c >> 1) + 8k + j
        for (int32_t c = lane; c < kpad / 16; c += 32) {
            const int32_t l0 = (c >> 1) * 32;
            uint32_t bits = 0;
            if (valid && (l0 >> 6) < n_words) bits = (uint32_t)(src[l0 >> 6] >> (l0 & 63));
            const int32_t live = n_loci - l0;
            const uint32_t in_n = !valid ? 0u : live >= 32 ? 0xFFFFFFFFu : live <= 0 ? 0u : ((1u << live) - 1u);
            bits &= in_n;
            const int32_t j0 = 4 * (c & 1);
            pc += __popc(bits & (0x0F0F0F0Fu << j0));
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t qb = (bits >> (j0 + i)) & 0x01010101u;  // Q_l, one per byte
                const uint32_t nb = (in_n >> (j0 + i)) & 0x01010101u;  // l < N
                w[i] = (nb & ~qb) * one | (mis ? qb * (one | 0x80u) : 0u);
            }
            reinterpret_cast<uint4 *>(dst)[c] = make_uint4(w[0], w[1], w[2], w[3]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
        if (lane == 0) *qc = mis ? (float)pc : 0.f;
        return;
    }
    for (int32_t c = lane; c < kpad / 16; c += 32) {
        const int32_t l0 = c * 16;
        uint32_t bits = 0;
        if (valid && (l0 >> 6) < n_words) bits = (uint32_t)(src[l0 >> 6] >> (l0 & 63)) & 0xFFFFu;
        // loci < N inside this 16-locus group
        const int32_t live = n_loci - l0;
        const uint32_t in_n = !valid ? 0u : live >= 16 ? 0xFFFFu : live <= 0 ? 0u : ((1u << live) - 1u);
        bits &= in_n;
        pc += __popc(bits);
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t qb = (bits >> (4 * i)) & 0xFu;   // Q_l
            const uint32_t nb = (in_n >> (4 * i)) & 0xFu;   // l < N
            // mode 1: 1 - Q_l  -> +1 where l < N and Q_l = 0
            // mode 0: 1 - 2Q_l -> +1 where Q_l = 0, -1 (sign bit 0x80 set) where Q_l = 1
            const uint32_t plus = (((nb & ~qb) * 0x00204081u) & 0x01010101u) * one;
            const uint32_t minus = mis ? ((qb * 0x00204081u) & 0x01010101u) * (one | 0x80u) : 0u;
            w[i] = plus | minus;
        }
        reinterpret_cast<uint4 *>(dst)[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
    if (lane == 0) *qc = mis ? (float)pc : 0.f;
}

// Reference operand, FP4: row r holds kbytes = (loci padded to 256) / 2
// bytes; its 16-byte chunk c covers loci 32c .. 32c + 31, in the nibble order
// of expand_stage_f4 (nibble n of 32-bit word j = locus 32c + 4n + j).  From
// packed rows at stride ld64 of which the first n_src rows and n_words words
// exist (zero elsewhere).  One thread per 16 output bytes, streaming loads and
// stores as in refs_e4m3_kernel.
__global__ void refs_e2m1_kernel(const uint64_t *__restrict__ packed, int64_t ld64, int64_t n_src, int32_t n_words,
                                 int64_t n_rows, int32_t kbytes, uint8_t *__restrict__ out) {
    const int64_t per_row = kbytes / 16;
    const int64_t total = n_rows * per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / per_row, c = t - r * per_row;
        const int32_t wi = (int32_t)(c >> 1);
        const uint64_t w = (r < n_src && wi < n_words) ? __ldcs(packed + r * ld64 + wi) : 0ull;
        const uint32_t x = (uint32_t)(w >> (32 * (c & 1)));
        const uint4 o = make_uint4((x << 1) & PK4_BIT1, x & PK4_BIT1, (x >> 1) & PK4_BIT1, (x >> 2) & PK4_BIT1);
        __stcs(reinterpret_cast<uint4 *>(out + r * (int64_t)kbytes) + c, o);
    }
}

// Query operand, FP4, per mode and c_q for one row, by one warp: e2m1 +1
// (0x2) where l < N and Q_l = 0; in mode 0 also -1 (0xA) where Q_l = 1; 0
// elsewhere.  Same nibble order as the reference operand.  src == nullptr (a
// padding row) writes zeros.
__device__ __forceinline__ void encode_query_row_f4(const uint64_t *__restrict__ src, bool mis, int32_t n_words,
                                                    int32_t n_loci, int32_t kbytes, uint8_t *__restrict__ dst,
                                                    float *__restrict__ qc, int lane) {
    const bool valid = src != nullptr;
    uint32_t pc = 0;
    for (int32_t c = lane; c < kbytes / 16; c += 32) {
        const int32_t l0 = c * 32;
        uint32_t bits = 0;
        if (valid && (l0 >> 6) < n_words) bits = (uint32_t)(src[l0 >> 6] >> (l0 & 63));
        const int32_t live = n_loci - l0;
        const uint32_t in_n = !valid ? 0u : live >= 32 ? 0xFFFFFFFFu : live <= 0 ? 0u : ((1u << live) - 1u);
        bits &= in_n;
        pc += __popc(bits);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t qb = (bits >> j) & 0x11111111u;  // Q at nibble n = locus 4n + j
            const uint32_t nb = (in_n >> j) & 0x11111111u;  // l < N
            w[j] = ((nb & ~qb) << 1) | (mis ? qb * 0xAu : 0u);
        }
        reinterpret_cast<uint4 *>(dst)[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
    if (lane == 0) *qc = mis ? (float)pc : 0.f;
}

// Operand row r encodes input query spread_row_to_query(r, spread).
__global__ void queries_e2m1_kernel(const uint64_t *__restrict__ q, int64_t ld_q, int64_t n_q, int32_t n_words,
                                    int32_t n_loci, const uint8_t *__restrict__ modes, int64_t n_q_pad,
                                    int32_t kbytes, uint8_t *__restrict__ out, float *__restrict__ qconst,
                                    int64_t spread) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_q_pad; r += warps_total) {
        const int64_t src = spread_row_to_query(r, spread);
        const bool valid = src < n_q;
        encode_query_row_f4(valid ? q + src * ld_q : nullptr, valid && modes[src] == FASTID_MODE_MISMATCH, n_words,
                            n_loci, kbytes, out + r * (int64_t)kbytes, qconst + r, lane);
    }
}

__global__ void queries_e4m3_kernel(const uint64_t *__restrict__ q, int64_t ld_q, int64_t n_q, int32_t n_words,
                                    int32_t n_loci, const uint8_t *__restrict__ modes, int64_t n_q_pad,
                                    int32_t kpad, uint8_t *__restrict__ out, float *__restrict__ qconst,
                                    uint32_t one, bool pk, int64_t spread) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_q_pad; r += warps_total) {
        const int64_t src = spread_row_to_query(r, spread);
        const bool valid = src < n_q;
        encode_query_row(valid ? q + src * ld_q : nullptr, valid && modes[src] == FASTID_MODE_MISMATCH, n_words,
                         n_loci, kpad, out + r * (int64_t)kpad, qconst + r, lane, one, pk);
    }
}

// Batched form: one job per operand row of every panel.
__global__ void prep_jobs_kernel(const PrepJob *__restrict__ jobs, int64_t n_jobs) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_jobs; j += warps_total) {
        const PrepJob jb = jobs[j];
        const bool mis = jb.src != nullptr && *jb.mode == FASTID_MODE_MISMATCH;
        if (jb.f4)
            encode_query_row_f4(jb.src, mis, jb.n_words, jb.n_loci, jb.kpad, jb.dst, jb.qc, lane);
        else
            encode_query_row(jb.src, mis, jb.n_words, jb.n_loci, jb.kpad, jb.dst, jb.qc, lane);
    }
}

template <int BN, bool PK = false, bool CG2 = false>
size_t tensor_smem(bool f4 = false) {
    using S = TcShape<BN, PK, CG2>;
    return 1024 + S::STAGES * (size_t)(TC_A_BYTES + S::B_BYTES + (PK ? pk_stage_bytes(BN, f4) : 0)) + 256;
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
int tensor_tile_r() { return 256; }
int tensor_tile_r4() { return TC_BN4; }
int tensor_kpad(int32_t n_loci) { return (n_loci + TC_BK - 1) / TC_BK * TC_BK; }
int tensor_kbytes4(int32_t n_loci) { return (n_loci + 2 * TC_BK - 1) / (2 * TC_BK) * TC_BK; }

cudaError_t launch_refs_e2m1(const uint64_t *packed, int64_t ld64, int64_t n_src, int32_t n_words, int64_t n_rows,
                             int32_t kbytes, uint8_t *out, int max_blocks, cudaStream_t s) {
    int64_t total = n_rows * (kbytes / 16);
    int64_t blocks = (total + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) return cudaSuccess;
    refs_e2m1_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, ld64, n_src, n_words, n_rows, kbytes, out);
    return cudaGetLastError();
}

cudaError_t launch_queries_e2m1(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words, int32_t n_loci,
                                const uint8_t *modes, int64_t n_q_pad, int32_t kbytes, uint8_t *out, float *qconst,
                                int64_t spread, cudaStream_t s) {
    int64_t blocks = (n_q_pad + 7) / 8;
    if (blocks > 65535) blocks = 65535;
    queries_e2m1_kernel<<<(unsigned)blocks, 256, 0, s>>>(q, ld_q, n_q, n_words, n_loci, modes, n_q_pad, kbytes, out,
                                                         qconst, spread);
    return cudaGetLastError();
}

cudaError_t launch_refs_e4m3(const uint64_t *packed, int64_t ld64, int64_t n_src, int32_t n_words, int64_t n_rows,
                             int32_t kpad, uint8_t *out, int max_blocks, cudaStream_t s) {
    int64_t total = n_rows * (kpad / 16);
    int64_t blocks = (total + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) return cudaSuccess;
    refs_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, ld64, n_src, n_words, n_rows, kpad, out);
    return cudaGetLastError();
}

cudaError_t launch_queries_e4m3(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words, int32_t n_loci,
                                const uint8_t *modes, int64_t n_q_pad, int32_t kpad, uint8_t *out, float *qconst,
                                bool half, int64_t spread, cudaStream_t s) {
    int64_t blocks = (n_q_pad + 7) / 8;
    if (blocks > 65535) blocks = 65535;
    queries_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(q, ld_q, n_q, n_words, n_loci, modes, n_q_pad, kpad, out,
                                                         qconst, half ? 0x30u : 0x38u, half, spread);
    return cudaGetLastError();
}

// PK reference operand: the packed rows [rows][ld64] uint64 themselves, in
// boxes of box_words words (2 = 128 loci for FP8 stages, 4 = 256 for FP4) x
// box_rows references, unswizzled.
cudaError_t make_packed_map(CUtensorMap *map, const uint64_t *packed, int64_t rows, int64_t ld64, int box_words,
                            int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)ld64, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld64 * 8};
    cuuint32_t box[2] = {(cuuint32_t)box_words, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(packed), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_prep_jobs(const PrepJob *jobs, int64_t n_jobs, cudaStream_t s) {
    if (n_jobs == 0) return cudaSuccess;
    int64_t blocks = (n_jobs + 7) / 8;
    if (blocks > 65535) blocks = 65535;
    prep_jobs_kernel<<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    return cudaGetLastError();
}

// Largest number of 2-CTA clusters of the paired kernel that can be resident
// at once (0 if clusters are unavailable).
int tensor_pair_clusters(int device) {
    size_t smem = tensor_smem<256>();
    if (cudaFuncSetAttribute(tensor_kernel<256, true, TC_KMAX, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(sms & ~1);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tensor_kernel<256, true, TC_KMAX, false, false>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int tensor_grid_target(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

namespace {

// One launch of tensor_kernel<BN, PAIR, KM, PK, F4, CG2> over n_groups work
// groups (2-CTA clusters when paired).
template <int BN, bool PAIR, int KM, bool PK = false, bool F4 = false, bool CG2 = false>
cudaError_t launch_variant(const TcMaps &maps, const TensorArgs &a, int32_t n_groups, int epi, cudaStream_t s) {
    const size_t smem = tensor_smem<BN, PK, CG2>(F4);
    cudaError_t e = cudaFuncSetAttribute(tensor_kernel<BN, PAIR, KM, PK, F4, CG2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((PAIR ? 2 : 1) * n_groups);
    cfg.blockDim = dim3(PK ? TC_THREADS + pk_threads(KM) : TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = PAIR ? 2 : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, tensor_kernel<BN, PAIR, KM, PK, F4, CG2>, maps, a);
}

}  // namespace

cudaError_t launch_tensor_multi(int bn, const TcLaunch &L, cudaStream_t s) {
    TcMaps maps;
    TensorArgs a;
    memset(&maps, 0, sizeof maps);
    memset(&a, 0, sizeof a);
    if (L.n_panels < 1 || L.n_panels > TC_MAXP) return cudaErrorInvalidValue;
    if (L.n_groups < 1) return cudaSuccess;
    a.n_panels = L.n_panels;
    for (int p = 0; p < L.n_panels; ++p) {
        maps.a[p] = L.map_a[p];
        maps.b[p] = L.map_b[p];
        a.panel[p].n_refs = L.n_refs[p];
        a.panel[p].n_q = L.n_q[p];
        a.panel[p].n_rt = L.n_rt[p];
        a.panel[p].n_kb = L.kpad[p] / TC_BK;
        a.panel[p].sc = L.sched[p];
        a.panel[p].qconst = L.qconst[p];
        a.panel[p].qspread = L.qspread[p];
        a.order[p] = L.order[p];
    }
    a.threshold = L.threshold;
    a.k = L.k;
    a.epi = L.epi;
    a.out = L.out;
    a.ld_out = L.ld_out;
    a.capacity = L.capacity;
    a.hit_q = L.hit_q;
    a.hit_r = L.hit_r;
    a.hit_score = L.hit_score;
    a.hit_count = L.hit_count;
    a.partial = L.partial;
    a.status = L.status;
    a.arrive = L.arrive;
    // 16-slot lists when k allows (half the insert network, 32 fewer registers)
    const bool k16 = L.epi != EPI_TOPK || L.k <= 16;
    if (L.f4) {  // 224-reference tiles whatever bn says
        if (L.pk) {
            if (L.pair) return cudaErrorInvalidValue;
            return k16 ? launch_variant<TC_BN4, false, 16, true, true>(maps, a, L.n_groups, L.epi, s)
                       : launch_variant<TC_BN4, false, 32, true, true>(maps, a, L.n_groups, L.epi, s);
        }
        if (L.pair && L.cg2)
            return k16 ? launch_variant<TC_BN4, true, 16, false, true, true>(maps, a, L.n_groups, L.epi, s)
                       : launch_variant<TC_BN4, true, 32, false, true, true>(maps, a, L.n_groups, L.epi, s);
        if (L.pair) return k16 ? launch_variant<TC_BN4, true, 16, false, true>(maps, a, L.n_groups, L.epi, s)
                               : launch_variant<TC_BN4, true, 32, false, true>(maps, a, L.n_groups, L.epi, s);
        return k16 ? launch_variant<TC_BN4, false, 16, false, true>(maps, a, L.n_groups, L.epi, s)
                   : launch_variant<TC_BN4, false, 32, false, true>(maps, a, L.n_groups, L.epi, s);
    }
    if (L.pair && bn != 256) return cudaErrorInvalidValue;
    if (L.pk) {
        if (L.pair || bn != 256) return cudaErrorInvalidValue;
        return k16 ? launch_variant<256, false, 16, true>(maps, a, L.n_groups, L.epi, s)
                   : launch_variant<256, false, 32, true>(maps, a, L.n_groups, L.epi, s);
    }
    if (L.pair && L.cg2)
        return k16 ? launch_variant<256, true, 16, false, false, true>(maps, a, L.n_groups, L.epi, s)
                   : launch_variant<256, true, 32, false, false, true>(maps, a, L.n_groups, L.epi, s);
    if (L.pair) return k16 ? launch_variant<256, true, 16>(maps, a, L.n_groups, L.epi, s)
                           : launch_variant<256, true, 32>(maps, a, L.n_groups, L.epi, s);
    if (bn == 128) return k16 ? launch_variant<128, false, 16>(maps, a, L.n_groups, L.epi, s)
                              : launch_variant<128, false, 32>(maps, a, L.n_groups, L.epi, s);
    return k16 ? launch_variant<256, false, 16>(maps, a, L.n_groups, L.epi, s)
               : launch_variant<256, false, 32>(maps, a, L.n_groups, L.epi, s);
}

}  // namespace fastid
