/*
 * CPU oracle for the FastID all-pairs comparison.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * path: it works on unpacked 0/1 alleles, one locus at a time, exactly as the
 * paper states the method.
 *
 * Paper: Samsi et al., "A Linear Algebra Approach to Fast DNA Mixture
 * Analysis Using GPUs" (arXiv:1707.00516).
 *   Sec. II-A, Eq. 1:  P_ij = POPCOUNT(AND(XOR(R_i, Q_j), R_i))
 *   Sec. II-A:         the XOR alone counts every minor-allele difference
 *                      between two individuals.
 *   Algorithm 1/2:     the same operations, word by word, summed over the
 *                      profile, for every (unknown, known) pair.
 * Here a "word" is a single locus, so POPCOUNT of a one-bit value is the
 * value itself and the sum over loci is the population count.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC fastid_oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * Sec. II-A (conversion of alleles to unsigned integers; worked example
 * 0x06001440 = 100668480).  Reading used throughout this project: locus l is
 * bit (l mod 64) of 64-bit word l / 64, least significant bit first, so the
 * little-endian bytes equal those of the 32-bit packing (bit l mod 32 of word
 * l / 32).  Words past the last locus are zero.
 */
void oracle_pack(const uint8_t *alleles, int64_t n, int32_t n_loci, int64_t ld_alleles,
                 uint64_t *out, int64_t ld_words)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t *row = out + i * ld_words;
        for (int64_t w = 0; w < ld_words; ++w)
            row[w] = 0;
        for (int32_t l = 0; l < n_loci; ++l)
            if (alleles[i * ld_alleles + l] != 0)
                row[l / 64] |= (uint64_t)1 << (l % 64);
    }
}

/*
 * A mixture is the union of the minor alleles of its contributors
 * (Sec. I and II-A: a mixture shows every minor allele present in any
 * contributor).  out[m][l] = OR over the source rows offsets[m] ..
 * offsets[m+1]-1 of src[s][l].
 */
void oracle_mix(const uint8_t *src, int32_t n_loci, const int32_t *offsets, int64_t n_mix,
                uint8_t *out)
{
    for (int64_t m = 0; m < n_mix; ++m) {
        uint8_t *o = out + m * (int64_t)n_loci;
        for (int32_t l = 0; l < n_loci; ++l) {
            uint8_t v = 0;
            for (int32_t s = offsets[m]; s < offsets[m + 1]; ++s)
                v = (uint8_t)(v | (src[(int64_t)s * n_loci + l] != 0));
            o[l] = v;
        }
    }
}

/* One (reference, query) pair, locus by locus: XOR, then AND with the
 * reference (Eq. 1), then count.  *mis gets the XOR count, *une the Eq. 1
 * count. */
static void pair_counts(const uint8_t *r, const uint8_t *q, int32_t n_loci,
                        uint32_t *mis, uint32_t *une)
{
    uint32_t m = 0, u = 0;
    for (int32_t l = 0; l < n_loci; ++l) {
        uint8_t a = (uint8_t)(r[l] != 0);   /* R_i at this locus */
        uint8_t b = (uint8_t)(q[l] != 0);   /* Q_j at this locus */
        uint8_t x = (uint8_t)(a ^ b);       /* XOR(R_i, Q_j)            */
        uint8_t y = (uint8_t)(x & a);       /* AND(XOR(R_i, Q_j), R_i)  */
        m += x;                             /* POPCOUNT summed over loci */
        u += y;
    }
    *mis = m;
    *une = u;
}

/*
 * Algorithm 2: every unknown q against every known r.
 * Output layout: mis[q * n_r + r], une[q * n_r + r]; either may be NULL.
 * n_threads <= 0 uses the OpenMP default.
 */
void oracle_scores(const uint8_t *R, int64_t n_r, const uint8_t *Q, int64_t n_q, int32_t n_loci,
                   uint32_t *mis, uint32_t *une, int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads <= 0)
        n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t q = 0; q < n_q; ++q) {
        for (int64_t r = 0; r < n_r; ++r) {
            uint32_t m, u;
            pair_counts(R + r * n_loci, Q + q * n_loci, n_loci, &m, &u);
            if (mis) mis[q * n_r + r] = m;
            if (une) une[q * n_r + r] = u;
        }
    }
}

/* The same counts for an explicit list of (q, r) pairs. */
void oracle_score_pairs(const uint8_t *R, const uint8_t *Q, int32_t n_loci,
                        const int64_t *qi, const int64_t *ri, int64_t n_pairs,
                        uint32_t *mis, uint32_t *une, int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads <= 0)
        n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
    for (int64_t p = 0; p < n_pairs; ++p) {
        uint32_t m, u;
        pair_counts(R + ri[p] * n_loci, Q + qi[p] * n_loci, n_loci, &m, &u);
        if (mis) mis[p] = m;
        if (une) une[p] = u;
    }
}

int32_t oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
