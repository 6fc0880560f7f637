// Host check of the query spreading of tensor calls (common.cuh): for every
// tile count s and query count n_q of an operand padded to whole tiles (or
// tile pairs), spread_row_to_query and spread_query_to_row are inverse
// bijections on [0, 128 s), exactly n_q rows hold a real query, and
// consecutive input queries sit in different tiles.  Prints "bad <count>".
#include <cstdio>
#include <vector>

#include "common.cuh"

using namespace fastid;

int main() {
    long bad = 0;
    for (int64_t s = 1; s <= 64; ++s) {
        const int64_t rows = s * TC_TILE_Q;
        std::vector<char> seen(rows, 0);
        for (int64_t r = 0; r < rows; ++r) {
            const int64_t q = spread_row_to_query(r, s);
            if (q < 0 || q >= rows || seen[q]) {
                ++bad;
                continue;
            }
            seen[q] = 1;
            if (spread_query_to_row(q, s) != r) ++bad;
            // tile r / 128 holds queries congruent to it modulo s
            if (q % s != r / TC_TILE_Q) ++bad;
        }
        for (int64_t q = 0; q + 1 < rows && s > 1; ++q)
            if (spread_query_to_row(q, s) / TC_TILE_Q == spread_query_to_row(q + 1, s) / TC_TILE_Q) ++bad;
    }
    // the padding of real calls: n_q queries in round_up(n_q, 128 p) rows, p = 1 or 2
    for (int p = 1; p <= 2; ++p)
        for (int64_t n_q = 1; n_q <= 4000; n_q += (n_q < 300 ? 1 : 37)) {
            const int64_t tile = (int64_t)TC_TILE_Q * p;
            const int64_t pad = (n_q + tile - 1) / tile * tile, s = pad / TC_TILE_Q;
            int64_t real = 0;
            for (int64_t r = 0; r < pad; ++r) real += spread_row_to_query(r, s) < n_q;
            if (real != n_q) ++bad;
            for (int64_t q = 0; q < n_q; ++q) {
                const int64_t r = spread_query_to_row(q, s);
                if (r < 0 || r >= pad) ++bad;
            }
        }
    std::printf("bad %ld\n", bad);
    return bad != 0;
}
