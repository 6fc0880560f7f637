// Microbenchmarks of the roofline denominators that the comparison kernels
// are measured against, run on the GPU they are measured on.
//
//   tensor  tcgen05.mma from shared-memory operands, one CTA per SM:
//             kind::f8f6f4  e4m3 x e4m3 -> f32, M = 128, N = 256, K = 32
//             kind::mxf4    e2m1 x e2m1 with unit ue8m0 block scale factors
//                           -> f32, M = 128, N = 224 or 256, K = 64
//           The same kernel, given operands and one stage of MMAs, returns
//           D = A B^T: an exactness check of both operand encodings and of
//           the block-scaled instruction descriptor on a single tile.
//   alu     POPC alone, LOP3 alone, and the plain form's inner sequence
//           (AND, POPC, and a 3-input add per two words)
//   b1 mma  mma.sync m16n8k256 b1 AND + POPC, the binary tensor-core path
//
// Each probe reports its device time (CUDA events) and the SM clock seen by
// its CTAs (clock64 against %globaltimer), so rates can be stated per clock
// per SM as well as per second.  This is measurement code: the comparison
// library does not link it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

constexpr int PM = 128;            // MMA M (TMEM lanes)
constexpr int ROWB = 128;          // bytes of K per operand row (one 128-byte swizzle atom)
constexpr uint32_t SF_COL = 448;   // first TMEM column of the unit scale factors
constexpr uint32_t SF_UNIT = 0x7F7F7F7Fu;  // four ue8m0 bytes of 2^0
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptors (PTX ISA, tcgen05 instruction descriptor tables).
// kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3 (0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f8(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// kind::mxf4: B scale-factor id 0 (bits 4-5), A = B = E2M1 (1 at bits 7 and
// 10), N >> 3 at bit 17, scale type UE8M0 (bit 23), M >> 4 at bit 24 (for
// M = 128 the same bit as M >> 7 at bit 27), A scale-factor id 0 (29-30).
__host__ __device__ constexpr uint32_t idesc_mxf4(int m, int n) {
    return (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (1u << 23) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_mxf4(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sfa,
                                         uint32_t sfb, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
}

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

struct ProbeCtl {
    uint64_t done;
    uint64_t stage_bar;  // sync probes: committed to every round
    uint64_t ready_bar;  // sync probes: completed once, then waited on every round
    uint32_t tmem_base;
};

// One CTA: operands A [128][128 B] and B [N][128 B] (K-major rows, bytes as
// the MMA kind reads them) copied into shared memory in the 128-byte swizzle,
// nst times at distinct addresses (stages, as the comparison kernel's ring
// holds them), then `iters` rounds of 4 MMAs over the 128 bytes of K of
// stage it % nst into one TMEM accumulator.  sync (bits): after each round's
// 4 MMAs the issuing thread also waits on an mbarrier phase that has already
// completed (1), fences (2) and commits to an mbarrier (4) -- 7 is the
// per-stage work of the comparison kernel's MMA thread without its data.  d_out (optional, [128][N] f32) receives the accumulator.
// cyc[2 * blockIdx.x] = SM clocks of the MMA loop, cyc[2 * blockIdx.x + 1] =
// its nanoseconds.  A wait that runs out sets *status = 1.
// NST and SYNC are compile-time so that the issuing loop is as short as the
// hardware allows: with a runtime stage modulo and three runtime branches in
// it, the single issuing thread alone held FP4 N = 224 to 79 % and FP8 to 91 %
// of these rates.
template <bool F4, int N, int NST, int SYNC>
__global__ void __launch_bounds__(192, 1)
    mma_probe_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b, int iters,
                     float *__restrict__ d_out, unsigned long long *__restrict__ cyc, uint32_t *status) {
    constexpr int nst = NST;
    constexpr int sync = SYNC;
    extern __shared__ uint8_t smem_raw[];
    constexpr int STAGE = (PM + N) * ROWB;  // a multiple of 1024
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    ProbeCtl *ctl = reinterpret_cast<ProbeCtl *>(base + nst * STAGE);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < nst * (PM + N) * 8; i += blockDim.x) {
        const int st = i / ((PM + N) * 8), j = i - st * (PM + N) * 8;
        const int row = j >> 3, c = j & 7;
        const bool isa = row < PM;
        const int r = isa ? row : row - PM;
        const uint4 v = *reinterpret_cast<const uint4 *>((isa ? a : b) + (size_t)r * ROWB + c * 16);
        *reinterpret_cast<uint4 *>(base + st * STAGE + (isa ? 0 : PM * ROWB) + r * ROWB + ((c ^ (r & 7)) << 4)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl->done)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl->stage_bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl->ready_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->ready_bar)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&ctl->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    if (F4 && warp >= 2) {  // unit scale factors in columns SF_COL.. of every lane
        const uint32_t t = tmem + ((uint32_t)((warp & 3) * 32) << 16) + SF_COL;
#pragma unroll
        for (int c = 0; c < 64; c += 16) tmem_st16(t + c, SF_UNIT);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1 && lane == 0) {
        const uint64_t ad0 = sw128_desc(smem_u32(base)), bd0 = sw128_desc(smem_u32(base + PM * ROWB));
        const long long c0 = clock64();
        const uint64_t n0 = globaltimer();
        for (int it = 0; it < iters; ++it) {
            // stage it % NST (NST a power of two): constant offsets in the descriptors' address field
            const uint32_t st = NST == 1 ? 0u : (uint32_t)it & (NST - 1);
            const uint64_t ad = ad0 + st * (STAGE >> 4), bd = bd0 + st * (STAGE >> 4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per MMA: +2 in the address field
                if (F4)
                    mma_mxf4(tmem, ad + 2u * kk, bd + 2u * kk, idesc_mxf4(PM, N), tmem + SF_COL, tmem + SF_COL + 16,
                             (it | kk) != 0);
                else
                    mma_f8(tmem, ad + 2u * kk, bd + 2u * kk, idesc_f8(PM, N), (it | kk) != 0);
            }
            if constexpr ((sync & 1) != 0) {  // phase 0 of ready_bar completed at set-up: the wait succeeds at once
                while (!mbar_try_wait(smem_u32(&ctl->ready_bar), 0)) {
                }
            }
            if constexpr ((sync & 2) != 0) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if constexpr ((sync & 4) != 0)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&ctl->stage_bar))
                             : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&ctl->done))
                     : "memory");
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(smem_u32(&ctl->done), 0)) {
            if (globaltimer() - t0 > WAIT_NS) {
                atomicExch(status, 1u);
                break;
            }
        }
        const long long c1 = clock64();
        const uint64_t n1 = globaltimer();
        if (cyc) {
            cyc[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
            cyc[2 * blockIdx.x + 1] = n1 - n0;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (d_out && warp >= 2) {
        const int quad = warp & 3, row = quad * 32 + lane;
        const uint32_t t = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < N; c += 32) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(t + c, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) d_out[(size_t)row * N + c + j] = __uint_as_float(v[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// Operand bytes for the rate runs: e4m3 0, +1, -1 (0x00, 0x38, 0xB8) for
// kind::f8f6f4, any nibble (every e2m1 code is a finite value) for mxf4.
__global__ void fill_kernel(uint8_t *p, size_t n, bool f4) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const uint8_t f8[4] = {0x00, 0x38, 0xB8, 0x38};
        p[i] = f4 ? (uint8_t)h : f8[h & 3];
    }
}

// ALU probes: 1024 threads a CTA, 8 independent chains per thread.
//   op 0: x = popc(x)                      (1 POPC per element)
//   op 1: x = lop3(x, y, z, 0x96)          (1 LOP3 per element)
//   op 2: acc += popc(r & acc) + popc(q & acc) over 4 x 4 accumulators (the
//         AND + POPC sequence: 2 AND, 2 POPC, 1 IADD3 per two words; the
//         accumulator stands in for the operand loads so that nothing is
//         loop-invariant)
//   op 3: the same count by a carry-save (Harley-Seal) tree over 8 ANDed
//         words at a time, for 4 (reference, query) pairs: per 8 words 8
//         AND, 7 carry-save adders (2 LOP3 each: sum 0x96, majority 0xE8),
//         one POPC of the eights and one add; the pair's `fours` word stands
//         in for the operand loads
//   op 4: the plain kernel's step (and_popc8): per 8 words 8 AND, 4 full
//         adders (LOP3 sum and majority), 4 POPC and the weighted
//         multiply-adds, on 4 accumulators a thread that are the next step's
//         query words
// Counted elements: op 0 POPC, op 1 LOP3, op 2 POPC, op 3 and 4 word pairs.
// Op 3 holds 49 registers a thread, so its two CTAs a SM run one after the
// other: per-SM rates are taken over the whole launch.
__device__ __forceinline__ uint32_t lop3_sum(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lop3_maj(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// carry-save adder: (hi, lo) = a + b + c bitwise
__device__ __forceinline__ void csa(uint32_t &hi, uint32_t &lo, uint32_t a, uint32_t b, uint32_t c) {
    hi = lop3_maj(a, b, c);
    lo = lop3_sum(a, b, c);
}

// Full adder as the plain kernel writes it (non-volatile LOP3, so that the
// compiler schedules it freely): sum 0x96, carry (majority) 0xE8.
__device__ __forceinline__ void fa_probe(uint32_t &sum, uint32_t &carry, uint32_t a, uint32_t b, uint32_t c) {
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(sum) : "r"(a), "r"(b), "r"(c));
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(carry) : "r"(a), "r"(b), "r"(c));
}

// The plain comparison kernel's word-pair step, restated: popc of the AND of
// 8 word pairs added to acc through four full adders (one LOP3 for the sum,
// one for the carry) and weighted multiply-adds by an opaque 2.
__device__ __forceinline__ uint32_t and_popc8_probe(const uint32_t (&r)[8], uint32_t q0, uint32_t q1, uint32_t q2,
                                                    uint32_t q3, uint32_t acc, uint32_t two) {
    // the query words of each full adder's three inputs differ, so that no
    // adder factors into (adder of reference words) AND q
    const uint32_t x0 = r[0] & q0, x1 = r[1] & q1, x2 = r[2] & q2, x3 = r[3] & q3, x4 = r[4] & q1, x5 = r[5] & q2,
                   x6 = r[6] & q3, x7 = r[7] & q0;
    uint32_t s1, c1, s2, c2, s3, c3, t, d;
    fa_probe(s1, c1, x0, x1, x2);
    fa_probe(s2, c2, x3, x4, x5);
    fa_probe(s3, c3, s1, s2, x6);
    fa_probe(t, d, c1, c2, c3);
    return (__popc(d) * two + __popc(t)) * two + (acc + __popc(s3) + __popc(x7));
}

template <int OP>
__global__ void __launch_bounds__(1024) alu_probe_kernel(uint32_t seed, int iters, uint32_t *out,
                                                         unsigned long long *cyc) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (seed + t * 8 + j) * 0x9E3779B9u;
    __syncthreads();
    const long long c0 = clock64();
    const uint64_t n0 = globaltimer();
    uint32_t res = 0;
    if (OP == 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j) asm volatile("popc.b32 %0, %0;" : "+r"(x[j]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) res += x[j];
    } else if (OP == 1) {
        const uint32_t y = seed ^ 0x5bd1e995u, z = seed * 3u + 1u;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[j]) : "r"(y), "r"(z));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) res += x[j];
    } else if (OP == 3) {
        uint32_t ones[4], twos[4], fours[4], tot[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            ones[p] = x[p];
            twos[p] = x[p + 4];
            fours[p] = x[p] ^ x[7 - p];
            tot[p] = 0;
        }
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) asm volatile("and.b32 %0, %1, %2;" : "=r"(w[i]) : "r"(x[i]), "r"(fours[p]));
                uint32_t tA, tB, fA, fB, e;
                csa(tA, ones[p], ones[p], w[0], w[1]);
                csa(tB, ones[p], ones[p], w[2], w[3]);
                csa(fA, twos[p], twos[p], tA, tB);
                csa(tA, ones[p], ones[p], w[4], w[5]);
                csa(tB, ones[p], ones[p], w[6], w[7]);
                csa(fB, twos[p], twos[p], tA, tB);
                csa(e, fours[p], fours[p], fA, fB);
                uint32_t pe;
                asm volatile("popc.b32 %0, %1;" : "=r"(pe) : "r"(e));
                tot[p] += pe;
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) res += 8 * tot[p] + 4 * __popc(fours[p]) + 2 * __popc(twos[p]) + __popc(ones[p]);
    } else if (OP == 4) {
        const uint32_t two = seed == 0xFFFFFFFFu ? 3u : 2u;  // 2, opaque to the compiler
        // four accumulators; they are the query words of the next step's
        // ANDs (each (reference word, query word) pair once a step), so nothing
        // is loop-invariant
        uint32_t a0 = x[0] ^ x[7], a1 = x[1] ^ x[6], a2 = x[2] ^ x[5], a3 = x[3] ^ x[4];
        for (int it = 0; it < iters; ++it) {
            const uint32_t b0 = and_popc8_probe(x, a0, a1, a2, a3, a0, two);
            const uint32_t b1 = and_popc8_probe(x, a1, a2, a3, a0, a1, two);
            const uint32_t b2 = and_popc8_probe(x, a2, a3, a0, a1, a2, two);
            const uint32_t b3 = and_popc8_probe(x, a3, a0, a1, a2, a3, two);
            a0 = b0;
            a1 = b1;
            a2 = b2;
            a3 = b3;
        }
        uint32_t acc[4] = {a0, a1, a2, a3};
#pragma unroll
        for (int j = 0; j < 4; ++j) res += acc[j];
    } else {
        uint32_t acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = x[i] ^ x[4 + j];
        // each accumulator feeds its own next AND, so no operand is loop-invariant
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t p0, p1;
                    asm volatile("{\n\t.reg .b32 w;\n\tand.b32 w, %1, %2;\n\tpopc.b32 %0, w;\n\t}"
                                 : "=r"(p0) : "r"(x[i]), "r"(acc[i][j]));
                    asm volatile("{\n\t.reg .b32 w;\n\tand.b32 w, %1, %2;\n\tpopc.b32 %0, w;\n\t}"
                                 : "=r"(p1) : "r"(x[4 + j]), "r"(acc[i][j]));
                    acc[i][j] += p0 + p1;
                }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) res += acc[i][j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cyc[2 * blockIdx.x] = (unsigned long long)(clock64() - c0);
        cyc[2 * blockIdx.x + 1] = globaltimer() - n0;
    }
    out[t] = res;
}

// b1 tensor-core probe: 8 independent m16n8k256 AND + POPC accumulators a warp.
__global__ void __launch_bounds__(256) b1_probe_kernel(uint32_t seed, int iters, uint32_t *out,
                                                       unsigned long long *cyc) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[4], bb[2];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = (seed + t * 4 + j) * 0x9E3779B9u;
    bb[0] = a[0] ^ 0xA5A5A5A5u;
    bb[1] = a[1] * 7u;
    int c[8][4];
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[m][j] = 0;
    __syncthreads();
    const long long c0 = clock64();
    const uint64_t n0 = globaltimer();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int m = 0; m < 8; ++m)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                : "+r"(c[m][0]), "+r"(c[m][1]), "+r"(c[m][2]), "+r"(c[m][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(bb[0]), "r"(bb[1]));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cyc[2 * blockIdx.x] = (unsigned long long)(clock64() - c0);
        cyc[2 * blockIdx.x + 1] = globaltimer() - n0;
    }
    int r = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) r += c[m][j];
    out[t] = (uint32_t)r;
}

struct Timed {
    double ms = 0.0;         // CUDA-event time of the launch
    double clocks_med = 0.0; // median SM clocks of the timed loop over CTAs
    double mhz_med = 0.0;    // median clocks / ns over CTAs
};

int finish_timing(cudaEvent_t e0, cudaEvent_t e1, const unsigned long long *d_cyc, int n, Timed *t) {
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    std::vector<unsigned long long> h(2 * (size_t)n);
    if (cudaMemcpy(h.data(), d_cyc, h.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    std::vector<double> c(n), f(n);
    for (int i = 0; i < n; ++i) {
        c[i] = (double)h[2 * i];
        f[i] = h[2 * i + 1] ? (double)h[2 * i] / (double)h[2 * i + 1] * 1e3 : 0.0;
    }
    std::nth_element(c.begin(), c.begin() + n / 2, c.end());
    std::nth_element(f.begin(), f.begin() + n / 2, f.end());
    t->ms = ms;
    t->clocks_med = c[n / 2];
    t->mhz_med = f[n / 2];
    return 0;
}

template <bool F4, int N, int NST, int SYNC>
int run_mma(int iters, int grid, const uint8_t *a_host, const uint8_t *b_host, float *d_host, Timed *t) {
    auto kern = mma_probe_kernel<F4, N, NST, SYNC>;
    constexpr int nst = NST;
    // > half of the SM's shared memory: one CTA per SM (each holds all 512 TMEM columns)
    const size_t need = 1024 + (size_t)nst * (PM + N) * ROWB + 64;
    const size_t smem = need < 120 * 1024 ? 120 * 1024 : need;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    uint8_t *a = nullptr, *b = nullptr;
    float *d = nullptr;
    unsigned long long *cyc = nullptr;
    uint32_t *status = nullptr;
    int rc = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t st = 0;
    if (cudaMalloc(&a, PM * ROWB) || cudaMalloc(&b, (size_t)N * ROWB) || cudaMalloc(&cyc, 16 * (size_t)grid) ||
        cudaMalloc(&status, 4) || (d_host && cudaMalloc(&d, sizeof(float) * PM * N)))
        goto out;
    if (a_host) {
        if (cudaMemcpy(a, a_host, PM * ROWB, cudaMemcpyHostToDevice) ||
            cudaMemcpy(b, b_host, (size_t)N * ROWB, cudaMemcpyHostToDevice))
            goto out;
    } else {
        fill_kernel<<<16, 256>>>(a, PM * ROWB, F4);
        fill_kernel<<<16, 256>>>(b, (size_t)N * ROWB, F4);
    }
    if (cudaMemset(status, 0, 4) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) goto out;
    cudaEventRecord(e0);
    kern<<<grid, 192, smem>>>(a, b, iters, d, cyc, status);
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || finish_timing(e0, e1, cyc, grid, t)) goto out;
    if (cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost)) goto out;
    if (st) {
        rc = 2;
        goto out;
    }
    if (d_host && cudaMemcpy(d_host, d, sizeof(float) * PM * N, cudaMemcpyDeviceToHost)) goto out;
    rc = 0;
out:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    cudaFree(d);
    cudaFree(cyc);
    cudaFree(status);
    return rc;
}

int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

}  // namespace

extern "C" {

// One tcgen05 MMA probe launch.  f4: 0 kind::f8f6f4 (n = 256), 1 kind::mxf4
// (n = 224 or 256).  nst: operand stages cycled through (1 .. 4; 1 re-reads
// the same shared memory every round; 1 or 4).  sync: 0, or 7 for a wait on a
// completed mbarrier phase, a tcgen05 fence and a commit every round of 4
// MMAs.  grid <= 0: one CTA per SM.  a_host [128][128] and b_host
// [n][128] operand bytes (both NULL: filled on the device); d_host [128][n]
// (optional, grid must be 1) receives D.  Outputs: event ms, median clocks
// and MHz of the MMA loop over CTAs.  Returns 0, 1 (CUDA error or bad
// arguments) or 2 (the completion wait ran out).
int fastid_peaks_mma(int f4, int n, int iters, int grid, int nst, int sync, const uint8_t *a_host,
                     const uint8_t *b_host, float *d_host, double *ms, double *clocks, double *mhz) {
    if (grid <= 0) grid = sms();
    if (iters < 1 || (nst != 1 && nst != 4) || (sync != 0 && sync != 7) || (d_host && grid != 1) ||
        (!a_host) != (!b_host))
        return 1;
    Timed t;
    int rc;
#define FASTID_PROBE_RUN(F4, N)                                                                                   \
    (nst == 1 ? (sync ? run_mma<F4, N, 1, 7>(iters, grid, a_host, b_host, d_host, &t)                             \
                      : run_mma<F4, N, 1, 0>(iters, grid, a_host, b_host, d_host, &t))                            \
              : (sync ? run_mma<F4, N, 4, 7>(iters, grid, a_host, b_host, d_host, &t)                             \
                      : run_mma<F4, N, 4, 0>(iters, grid, a_host, b_host, d_host, &t)))
    if (!f4 && n == 256)
        rc = FASTID_PROBE_RUN(false, 256);
    else if (f4 && n == 224)
        rc = FASTID_PROBE_RUN(true, 224);
    else if (f4 && n == 256)
        rc = FASTID_PROBE_RUN(true, 256);
    else
        return 1;
#undef FASTID_PROBE_RUN
    if (ms) *ms = t.ms;
    if (clocks) *clocks = t.clocks_med;
    if (mhz) *mhz = t.mhz_med;
    return rc;
}

// ALU probe (op 0 POPC, 1 LOP3, 2 AND + POPC + IADD3, 3 Harley-Seal, 4 the
// plain kernel's carry-save step) on blocks_per_sm
// CTAs of 1024 threads per SM.  *elements: counted operations of the launch.
int fastid_peaks_alu(int op, int iters, int blocks_per_sm, double *ms, double *clocks, double *mhz,
                     double *elements) {
    if (op < 0 || op > 4 || iters < 1 || blocks_per_sm < 1) return 1;
    const int grid = sms() * blocks_per_sm, threads = 1024;
    uint32_t *out = nullptr;
    unsigned long long *cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Timed t;
    int rc = 1;
    if (cudaMalloc(&out, 4 * (size_t)grid * threads) || cudaMalloc(&cyc, 16 * (size_t)grid) ||
        cudaEventCreate(&e0) || cudaEventCreate(&e1))
        goto out;
    cudaEventRecord(e0);
    if (op == 0) alu_probe_kernel<0><<<grid, threads>>>(12345u, iters, out, cyc);
    if (op == 1) alu_probe_kernel<1><<<grid, threads>>>(12345u, iters, out, cyc);
    if (op == 2) alu_probe_kernel<2><<<grid, threads>>>(12345u, iters, out, cyc);
    if (op == 3) alu_probe_kernel<3><<<grid, threads>>>(12345u, iters, out, cyc);
    if (op == 4) alu_probe_kernel<4><<<grid, threads>>>(12345u, iters, out, cyc);
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || finish_timing(e0, e1, cyc, grid, &t)) goto out;
    if (elements) *elements = (double)grid * threads * (double)iters * 32.0;
    rc = 0;
out:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (ms) *ms = t.ms;
    if (clocks) *clocks = t.clocks_med;
    if (mhz) *mhz = t.mhz_med;
    return rc;
}

// b1 AND + POPC mma.sync probe on blocks_per_sm CTAs of 256 threads per SM.
// *bit_macs: 16 x 8 x 256 bit products per instruction, summed over the launch.
int fastid_peaks_b1(int iters, int blocks_per_sm, double *ms, double *clocks, double *mhz, double *bit_macs) {
    if (iters < 1 || blocks_per_sm < 1) return 1;
    const int grid = sms() * blocks_per_sm, threads = 256;
    uint32_t *out = nullptr;
    unsigned long long *cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Timed t;
    int rc = 1;
    if (cudaMalloc(&out, 4 * (size_t)grid * threads) || cudaMalloc(&cyc, 16 * (size_t)grid) ||
        cudaEventCreate(&e0) || cudaEventCreate(&e1))
        goto out;
    cudaEventRecord(e0);
    b1_probe_kernel<<<grid, threads>>>(777u, iters, out, cyc);
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || finish_timing(e0, e1, cyc, grid, &t)) goto out;
    if (bit_macs) *bit_macs = (double)grid * (threads / 32) * (double)iters * 8.0 * 16.0 * 8.0 * 256.0;
    rc = 0;
out:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (ms) *ms = t.ms;
    if (clocks) *clocks = t.clocks_med;
    if (mhz) *mhz = t.mhz_med;
    return rc;
}

}  // extern "C"
