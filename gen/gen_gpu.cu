// Device version of the seeded allele generator in gen/__init__.py, for
// databases too large to draw on the host.  It implements the same published
// counter-based function independently (SplitMix64 output function of
// Steele, Lea and Flood, OOPSLA 2014):
//   draw32(seed, stream, row, locus) =
//       splitmix64(key(seed, stream) ^ (row << 24 | locus)) >> 32
//   key(seed, stream) = splitmix64(splitmix64(seed) ^ stream)
//   allele = draw32(...) < thr[locus]
// The per-locus thresholds are computed on the host and passed in.  This file
// holds no comparison arithmetic and is not part of the comparison library.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One thread per 4 consecutive loci of a row; writes 4 allele bytes.
__global__ void gen_alleles_kernel(uint64_t key, const int64_t *__restrict__ rows, int64_t row0,
                                   int64_t n_rows, const uint32_t *__restrict__ thr, int32_t n_loci,
                                   uint8_t *__restrict__ out, int64_t ld_out) {
    const int64_t per_row = (n_loci + 3) / 4;
    const int64_t total = n_rows * per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / per_row;
        const int32_t l0 = (int32_t)(t - i * per_row) * 4;
        const uint64_t row = rows ? (uint64_t)rows[i] : (uint64_t)(row0 + i);
        uint32_t packed4 = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int32_t l = l0 + b;
            if (l < n_loci) {
                const uint32_t d = (uint32_t)(splitmix64(key ^ ((row << 24) | (uint64_t)l)) >> 32);
                packed4 |= (uint32_t)(d < thr[l]) << (8 * b);
            }
        }
        uint8_t *o = out + i * ld_out + l0;
        if (l0 + 4 <= n_loci && ((reinterpret_cast<uintptr_t>(o) & 3) == 0)) {
            *reinterpret_cast<uint32_t *>(o) = packed4;
        } else {
            for (int b = 0; b < 4 && l0 + b < n_loci; ++b) o[b] = (uint8_t)(packed4 >> (8 * b));
        }
    }
}

}  // namespace

extern "C" {

// Allele rows on the device: out[i][l] for i < n_rows, l < n_loci, with row
// index rows[i] (device int64 array) or row0 + i when rows is NULL.
// Returns a cudaError_t value.
int gen_alleles(uint64_t seed, uint64_t stream_id, const int64_t *rows_dev, int64_t row0, int64_t n_rows,
                const uint32_t *thr_dev, int32_t n_loci, uint8_t *out_dev, int64_t ld_out, void *stream) {
    if (n_rows <= 0) return 0;
    const uint64_t key = splitmix64(splitmix64(seed) ^ stream_id);
    int64_t total = n_rows * ((n_loci + 3) / 4);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    gen_alleles_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key, rows_dev, row0, n_rows, thr_dev,
                                                                           n_loci, out_dev, ld_out);
    return (int)cudaGetLastError();
}

}  // extern "C"
