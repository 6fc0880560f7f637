// Profile preparation kernels: packing (Sec. II-A), mixtures (per-word OR),
// database rows with popcounts, and the per-query operands of the plain form.
#include "common.cuh"

namespace fastid {

namespace {

// Four allele bytes -> four bits (byte i -> bit i).  Each byte is first
// normalised to 0/1; the multiply then moves byte i (at bit 8i) to bit 24+i:
// the multiplier 2^24 + 2^17 + 2^10 + 2^3 places byte i's term at 8i + 24 - 7j
// for multiplier term j, so only i == j lands in bits 24..27, the i < j terms
// land at distinct positions below bit 20 (no carries) and i > j overflow.
__device__ __forceinline__ uint32_t bytes4_to_bits(uint32_t x) {
    uint32_t nz = __vcmpne4(x, 0u) & 0x01010101u;
    return (nz * 0x01020408u) >> 24;
}

// One warp per row; lane handles 64-bit words lane, lane+32, ...
__global__ void pack_kernel(const uint8_t *__restrict__ alleles, int64_t n, int32_t n_loci,
                            int64_t ld_alleles, uint64_t *__restrict__ packed, int64_t ld_words,
                            uint32_t *__restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const bool vec = ((ld_alleles & 15) == 0) && ((reinterpret_cast<uintptr_t>(alleles) & 15) == 0);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
         row += warps_total) {
        const uint8_t *a = alleles + row * ld_alleles;
        uint64_t *o = packed + row * ld_words;
        uint32_t pc = 0;
        for (int64_t w = lane; w < ld_words; w += 32) {
            uint64_t word = 0;
            const int64_t l0 = w * 64;
            if (l0 + 64 <= n_loci && vec) {
                const uint4 *p = reinterpret_cast<const uint4 *>(a + l0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint4 v = __ldg(p + c);
                    uint64_t b = (uint64_t)bytes4_to_bits(v.x) | ((uint64_t)bytes4_to_bits(v.y) << 4) |
                                 ((uint64_t)bytes4_to_bits(v.z) << 8) |
                                 ((uint64_t)bytes4_to_bits(v.w) << 12);
                    word |= b << (16 * c);
                }
            } else if (l0 < n_loci) {
                const int64_t lim = (n_loci - l0) < 64 ? (n_loci - l0) : 64;
                for (int64_t t = 0; t < lim; ++t)
                    word |= (uint64_t)(a[l0 + t] != 0) << t;
            }
            o[w] = word;
            pc += __popcll(word);
        }
        if (norms) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
            if (lane == 0) norms[row] = pc;
        }
    }
}

__global__ void mix_kernel(const uint64_t *__restrict__ src, int64_t ld_src, int32_t n_words,
                           const int32_t *__restrict__ offsets, int64_t n_mix,
                           uint64_t *__restrict__ out, int64_t ld_out, uint32_t *__restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t m = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); m < n_mix;
         m += warps_total) {
        const int32_t s0 = offsets[m], s1 = offsets[m + 1];
        uint32_t pc = 0;
        for (int64_t w = lane; w < ld_out; w += 32) {
            uint64_t v = 0;
            if (w < n_words)
                for (int32_t s = s0; s < s1; ++s) v |= __ldg(src + (int64_t)s * ld_src + w);
            out[m * ld_out + w] = v;
            pc += __popcll(v);
        }
        if (norms) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
            if (lane == 0) norms[m] = pc;
        }
    }
}

// dst[r][w] = src[r][w] for r < n, w < n_words; zero elsewhere up to n_pad
// rows and ld_dst words.  norms[r] = popcount of the row (0 for padding rows).
__global__ void copy_rows_kernel(const uint64_t *__restrict__ src, int64_t n, int64_t ld_src,
                                 int32_t n_words, uint64_t *__restrict__ dst, int64_t n_pad,
                                 int64_t ld_dst, uint32_t *__restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_pad;
         r += warps_total) {
        uint32_t pc = 0;
        for (int64_t w = lane; w < ld_dst; w += 32) {
            uint64_t v = (r < n && w < n_words) ? __ldg(src + r * ld_src + w) : 0ull;
            dst[r * ld_dst + w] = v;
            pc += __popcll(v);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
        if (lane == 0 && norms) norms[r] = pc;
    }
}

// Plain-form query operands: rows of 32-bit words at stride ld32 (padded to
// n_q_pad rows, zero beyond n_q / n_words) and per-query coefficients.
__global__ void query_prep_kernel(const uint64_t *__restrict__ q, int64_t ld_q, int64_t n_q,
                                  int32_t n_words, const uint8_t *__restrict__ modes,
                                  uint32_t *__restrict__ q32, int64_t n_q_pad, int64_t ld32,
                                  QueryCoef *__restrict__ coef) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ld64 = ld32 / 2;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_q_pad;
         r += warps_total) {
        uint32_t pc = 0;
        for (int64_t w = lane; w < ld64; w += 32) {
            uint64_t v = (r < n_q && w < n_words) ? __ldg(q + r * ld_q + w) : 0ull;
            reinterpret_cast<uint2 *>(q32 + r * ld32)[w] = make_uint2((uint32_t)v, (uint32_t)(v >> 32));
            pc += __popcll(v);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
        if (lane == 0) {
            QueryCoef c;
            if (r < n_q && modes[r] == FASTID_MODE_MISMATCH) {
                c.a = 2u;  // popc(R ^ Q) = |R| + |Q| - 2 popc(R & Q)
                c.b = pc;
            } else {
                c.a = 1u;  // Eq. 1: popc(R & ~Q) = |R| - popc(R & Q)
                c.b = 0u;
            }
            coef[r] = c;
        }
    }
}

int warp_grid(int64_t rows, int warps_per_block) {
    int64_t blocks = (rows + warps_per_block - 1) / warps_per_block;
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

cudaError_t launch_pack(const uint8_t *alleles, int64_t n, int32_t n_loci, int64_t ld_alleles,
                        uint64_t *packed, int64_t ld_words, uint32_t *norms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    pack_kernel<<<warp_grid(n, 8), 256, 0, s>>>(alleles, n, n_loci, ld_alleles, packed, ld_words, norms);
    return cudaGetLastError();
}

cudaError_t launch_mix(const uint64_t *src, int64_t ld_src, int32_t n_words, const int32_t *offsets,
                       int64_t n_mix, uint64_t *out, int64_t ld_out, uint32_t *norms, cudaStream_t s) {
    if (n_mix == 0) return cudaSuccess;
    mix_kernel<<<warp_grid(n_mix, 8), 256, 0, s>>>(src, ld_src, n_words, offsets, n_mix, out, ld_out, norms);
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(const uint64_t *src, int64_t n, int64_t ld_src, int32_t n_words,
                             uint64_t *dst, int64_t n_pad, int64_t ld_dst, uint32_t *norms,
                             cudaStream_t s) {
    if (n_pad == 0) return cudaSuccess;
    copy_rows_kernel<<<warp_grid(n_pad, 8), 256, 0, s>>>(src, n, ld_src, n_words, dst, n_pad, ld_dst, norms);
    return cudaGetLastError();
}

cudaError_t launch_query_prep(const uint64_t *q, int64_t ld_q, int64_t n_q, int32_t n_words,
                              const uint8_t *modes, uint32_t *q32, int64_t n_q_pad, int64_t ld32,
                              QueryCoef *coef, cudaStream_t s) {
    if (n_q_pad == 0) return cudaSuccess;
    query_prep_kernel<<<warp_grid(n_q_pad, 8), 256, 0, s>>>(q, ld_q, n_q, n_words, modes, q32, n_q_pad,
                                                            ld32, coef);
    return cudaGetLastError();
}

}  // namespace fastid
