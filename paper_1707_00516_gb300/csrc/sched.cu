// Host-side work schedule of a tensor-form launch (see TcSched in common.cuh).
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"

namespace fastid {

namespace {

// Bytes of reference tiles all groups of a launch may keep in flight at once
// (about a third of the 129 MB L2).
constexpr int64_t L2_CHUNK_BUDGET = 48ll << 20;

// L2 prefetch of the next reference tile (single-tile groups): only where a
// slice is shared by several groups -- the first to reach a tile would
// otherwise wait on DRAM -- and all slices' prefetched tiles fit in a quarter
// of L2.  A lone group per slice gains nothing, and one tile ahead for each of
// 76-152 slices overflows L2: measured on 20M references at N = 2048, 64-256
// queries took 10-18 ms with the prefetch against 5.8-8.7 ms without.
constexpr int64_t PREFETCH_BUDGET = 32ll << 20;

// Relative cost of a reference tile for a group with several query tiles
// (chunks re-read from L2, top-k lists saved and resumed, no prefetch) over
// one with a single query tile, which streams its slice once with the next
// tile prefetched: 1 + TPX_PENALTY + SLICE_PENALTY * b.  Fit to sweeps of
// a x b grids on GB300 at N = 512 .. 16384 (4M references, 15 .. 21 query
// tile pairs, and 2048 queries x 20M references).
constexpr double TPX_PENALTY = 0.08;
constexpr double SLICE_PENALTY = 0.005;

// A tail (see TcSched) is added where it shortens the busiest group by at
// least this fraction.
constexpr double TAIL_MIN_GAIN = 0.02;

// Relative cost of a reference tile in a tail group (several query tiles over
// chunks re-read from L2, lists saved and resumed) against one in the grid
// (one query tile, prefetched stream).  Measured on 2048 queries x 20M
// references at N = 2048 (a tail of 4 groups x 2 tile pairs): 1.2, 1.3 and 1.4
// all gave 40.7 ms against 41.8 ms without a tail, while the grid model's own
// penalty (1.1) left the tail finishing last (43.3 ms).
constexpr double TAIL_COST = 1.3;

#ifdef FASTID_DEBUG
// Debug builds: every (query tile, reference tile) unit of the panel is
// covered exactly once by the grid and the tail, and every CTA's top-k slots
// are distinct and inside [slot0, slot_end).  The unit and slot mapping
// restates the kernel's group_work (csrc/tensor.cu).
bool schedule_consistent(const TcSched &sc, int64_t n_qq, int64_t n_rt, int cpg, int64_t slot_end) {
    if (n_qq <= 0 || n_rt <= 0) return true;
    std::vector<uint8_t> cov((size_t)(n_qq * n_rt), 0);
    std::vector<uint8_t> used((size_t)std::max<int64_t>(slot_end - sc.slot0, 0), 0);
    const int64_t grid = (int64_t)sc.a * sc.b;
    for (int64_t wg = 0; wg < grid + sc.t_groups; ++wg) {
        int64_t r_lo, r_hi, q_lo, q_hi, base, tpx;
        if (wg < grid) {
            const int64_t x = wg / sc.b, y = wg - x * sc.b;
            r_lo = y * (int64_t)sc.r_main / sc.b;
            r_hi = (y + 1) * (int64_t)sc.r_main / sc.b;
            tpx = sc.tpx;
            q_lo = x * tpx;
            q_hi = std::min<int64_t>(n_qq, (x + 1) * tpx);
            base = sc.slot0 + wg * cpg * tpx;
        } else {
            const int64_t t = wg - grid;
            r_lo = sc.r_main;
            r_hi = n_rt;
            tpx = sc.t_tpx;
            q_lo = std::min<int64_t>(n_qq, t * tpx);
            q_hi = std::min<int64_t>(n_qq, (t + 1) * tpx);
            base = sc.slot0 + grid * cpg * sc.tpx + t * cpg * tpx;
        }
        for (int64_t qq = q_lo; qq < q_hi; ++qq) {
            for (int rank = 0; rank < cpg; ++rank) {
                const int64_t s = base + rank * tpx + (qq - q_lo) - sc.slot0;
                if (s < 0 || s >= (int64_t)used.size() || used[(size_t)s]++) return false;
            }
            for (int64_t rt = r_lo; rt < r_hi; ++rt)
                if (++cov[(size_t)(qq * n_rt + rt)] != 1) return false;
        }
    }
    for (uint8_t c : cov)
        if (c != 1) return false;
    return true;
}
#endif

}  // namespace

int32_t make_tensor_schedule(int n, const int64_t *n_qq, const int64_t *n_rt, const int64_t *tile_bytes,
                             int32_t G, int32_t ctas_per_group, TcSched *sched, int32_t *order,
                             int32_t *n_slots) {
    int64_t slots = 0;
    int32_t groups = 0;
    for (int p = 0; p < n; ++p) {
        TcSched &sc = sched[p];
        sc.n_qq = (int32_t)n_qq[p];
        sc.slot0 = (int32_t)slots;
        sc.a = sc.b = 0;
        sc.tpx = 1;
        sc.chunk = 1;
        sc.pf = 0;
        sc.r_main = (int32_t)std::max<int64_t>(n_rt[p], 0);
        sc.t_groups = 0;
        sc.t_tpx = 1;
        sc.t_chunk = 1;
        if (n_qq[p] <= 0 || n_rt[p] <= 0) continue;
        // a x b grid minimising the busiest group's cost: its reference
        // tiles, weighted as above when it holds several query tiles.
        double best = -1.0;
        int64_t best_a = 1, best_b = 1, best_t = 1;
        for (int64_t a = 1; a <= std::min<int64_t>(n_qq[p], G); ++a) {
            const int64_t tpx = (n_qq[p] + a - 1) / a;
            const int64_t a_eff = (n_qq[p] + tpx - 1) / tpx;
            const int64_t b = std::min<int64_t>(G / a_eff, n_rt[p]);
            if (b < 1) continue;
            const double tiles = (double)(tpx * ((n_rt[p] + b - 1) / b));
            const double cost = tpx == 1 ? tiles : tiles * (1.0 + TPX_PENALTY + SLICE_PENALTY * (double)b);
            if (best < 0.0 || cost < best) {
                best = cost;
                best_a = a_eff;
                best_b = b;
                best_t = tpx;
            }
        }
        sc.a = (int32_t)best_a;
        sc.b = (int32_t)best_b;
        sc.tpx = (int32_t)best_t;
        const int64_t slice = (n_rt[p] + best_b - 1) / best_b;
        if (best_t == 1) {
            sc.chunk = (int32_t)std::max<int64_t>(1, slice);  // one segment per slice: nothing to resume
            sc.pf = best_a >= 2 && best_b * tile_bytes[p] <= PREFETCH_BUDGET;
        } else {
            const int64_t c = L2_CHUNK_BUDGET / std::max<int64_t>(1, best_b * tile_bytes[p]);
            sc.chunk = (int32_t)std::min<int64_t>(std::max<int64_t>(2, c), std::max<int64_t>(1, slice));
        }
        // Tail: groups the a x b grid leaves idle take the last reference
        // tiles for several query tiles each, and the grid's slices shrink so
        // that both finish together: r_main / b = t_tpx * (n_rt - r_main) * cost,
        // with the several-query-tile cost of the model above.
        const int64_t spare = (int64_t)G - best_a * best_b;
        if (best_t == 1 && best_a >= 2 && spare >= 1) {
            const int64_t tg = std::min<int64_t>(spare, best_a);
            const int64_t tt = (best_a + tg - 1) / tg;
            const int64_t tg_eff = (best_a + tt - 1) / tt;
            const double f = (double)tt * TAIL_COST;
            const int64_t r_main = (int64_t)((double)n_rt[p] * f / (1.0 / (double)best_b + f));
            const double old_busy = (double)((n_rt[p] + best_b - 1) / best_b);
            const double new_busy = (double)((r_main + best_b - 1) / best_b);
            if (r_main >= best_b && r_main < n_rt[p] && new_busy <= old_busy * (1.0 - TAIL_MIN_GAIN)) {
                sc.r_main = (int32_t)r_main;
                sc.t_groups = (int32_t)tg_eff;
                sc.t_tpx = (int32_t)tt;
                const int64_t c = L2_CHUNK_BUDGET / std::max<int64_t>(1, tg_eff * tile_bytes[p]);
                sc.t_chunk = (int32_t)std::min<int64_t>(std::max<int64_t>(2, c), n_rt[p] - r_main);
                if (best_t == 1) sc.chunk = (int32_t)std::max<int64_t>(1, (r_main + best_b - 1) / best_b);
            }
        }
        groups = std::max<int32_t>(groups, sc.a * sc.b + sc.t_groups);
        slots += (int64_t)sc.a * sc.b * ctas_per_group * sc.tpx + (int64_t)sc.t_groups * ctas_per_group * sc.t_tpx;
        if (slots > INT32_MAX) return -1;
#ifdef FASTID_DEBUG
        if (!schedule_consistent(sc, n_qq[p], n_rt[p], ctas_per_group, slots)) return -2;
#endif
    }
    // Largest panel first: every group enters it together, so the groups of
    // a slice stay in step and share its tiles through L2; the small panels
    // at the end absorb the drift.
    std::vector<double> work(n);
    for (int p = 0; p < n; ++p) {
        work[p] = (double)std::max<int64_t>(n_qq[p], 0) * (double)std::max<int64_t>(n_rt[p], 0) * (double)tile_bytes[p];
        order[p] = p;
    }
    std::stable_sort(order, order + n, [&](int32_t x, int32_t y) { return work[x] > work[y]; });
    *n_slots = (int32_t)slots;
    return groups;
}

}  // namespace fastid
