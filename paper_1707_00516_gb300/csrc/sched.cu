// Host-side work schedule of a tensor-form launch (see TcSched in common.cuh).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fastid {

namespace {

// Bytes of reference tiles all groups of a launch may keep in flight at once
// (about a third of the 129 MB L2).
constexpr int64_t L2_CHUNK_BUDGET = 48ll << 20;

// Balance a schedule with one query tile per group may lose before a
// multi-tile one (with list save / resume) is preferred.
constexpr double TPX1_SLACK = 1.08;

}  // namespace

int32_t make_tensor_schedule(int n, const int64_t *n_qq, const int64_t *n_rt, const int64_t *unit_cost,
                             const int64_t *tile_bytes, int32_t G, TcSched *sched, int32_t *max_tpx) {
    std::vector<double> cost(n, 0.0);
    double total = 0.0;
    for (int p = 0; p < n; ++p) {
        cost[p] = (double)n_qq[p] * (double)n_rt[p] * (double)unit_cost[p];
        total += cost[p];
    }
    // Groups per panel, proportional to cost (at least one per busy panel).
    std::vector<int64_t> gp(n, 0);
    int64_t used = 0;
    for (int p = 0; p < n; ++p) {
        if (cost[p] <= 0.0) continue;
        gp[p] = std::max<int64_t>(1, (int64_t)((double)G * cost[p] / total));
        used += gp[p];
    }
    while (used > G) {  // shrink the largest share
        int q = -1;
        for (int p = 0; p < n; ++p)
            if (gp[p] > 1 && (q < 0 || gp[p] > gp[q])) q = p;
        if (q < 0) break;
        --gp[q];
        --used;
    }
    while (used < G && total > 0.0) {  // grow the most loaded panel
        int q = -1;
        double worst = -1.0;
        for (int p = 0; p < n; ++p)
            if (cost[p] > 0.0 && cost[p] / (double)gp[p] > worst) {
                worst = cost[p] / (double)gp[p];
                q = p;
            }
        ++gp[q];
        ++used;
    }

    int32_t g0 = 0, mt = 1;
    for (int p = 0; p < n; ++p) {
        TcSched &sc = sched[p];
        sc.n_qq = (int32_t)n_qq[p];
        sc.g0 = g0;
        sc.a = sc.b = 0;
        sc.tpx = 1;
        sc.chunk = 1;
        if (cost[p] <= 0.0) continue;
        // a x b grid minimising the busiest group's reference tiles; one query
        // tile per group (nothing to save and resume) wins unless it costs
        // more than TPX1_SLACK in balance.
        int64_t best_ms = -1, best_a = 1, best_b = 1, best_t = 1;
        int64_t one_ms = -1, one_a = 1, one_b = 1;
        for (int64_t a = 1; a <= std::min<int64_t>(n_qq[p], gp[p]); ++a) {
            const int64_t tpx = (n_qq[p] + a - 1) / a;
            const int64_t a_eff = (n_qq[p] + tpx - 1) / tpx;
            const int64_t b = std::min<int64_t>(gp[p] / a_eff, n_rt[p]);
            if (b < 1) continue;
            const int64_t ms = tpx * ((n_rt[p] + b - 1) / b);
            if (best_ms < 0 || ms < best_ms || (ms == best_ms && tpx < best_t)) {
                best_ms = ms;
                best_a = a_eff;
                best_b = b;
                best_t = tpx;
            }
            if (tpx == 1 && (one_ms < 0 || ms < one_ms)) {
                one_ms = ms;
                one_a = a_eff;
                one_b = b;
            }
        }
        if (one_ms > 0 && (double)one_ms <= (double)best_ms * TPX1_SLACK) {
            best_ms = one_ms;
            best_a = one_a;
            best_b = one_b;
            best_t = 1;
        }
        sc.a = (int32_t)best_a;
        sc.b = (int32_t)best_b;
        sc.tpx = (int32_t)best_t;
        const int64_t slice = (n_rt[p] + best_b - 1) / best_b;
        if (best_t == 1) {
            sc.chunk = (int32_t)std::max<int64_t>(1, slice);  // one segment per slice: nothing to resume
        } else {
            const int64_t budget = L2_CHUNK_BUDGET * gp[p] / std::max<int64_t>(1, G);
            const int64_t c = budget / std::max<int64_t>(1, best_b * tile_bytes[p]);
            sc.chunk = (int32_t)std::min<int64_t>(std::max<int64_t>(2, c), std::max<int64_t>(1, slice));
        }
        g0 += sc.a * sc.b;
        mt = std::max(mt, sc.tpx);
    }
    *max_tpx = mt;
    return g0;
}

}  // namespace fastid
