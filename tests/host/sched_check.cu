// Host check of the tensor form's work schedule (make_tensor_schedule in
// csrc/sched.cu) over many shapes: the a x b grid and the tail (TcSched) cover
// every (query tile, reference tile) unit exactly once, every CTA's top-k slots
// are distinct and below n_slots, and the merge's slot formula finds each
// query tile's slots.  The unit mapping restates group_work (csrc/tensor.cu)
// and the merge's slot arithmetic (topk_merge_sched_kernel, csrc/reduce.cu) on
// the host; a change there must be made here too.  Exit status 0 = all pass.
#include <cstdio>
#include <vector>
#include <set>
#include <cstdlib>
#include "common.cuh"
using namespace fastid;
struct GW { int64_t r_lo, r_hi, q_lo, q_hi, slot; };
static GW gw(const TcSched &sc, int64_t n_rt, int64_t wg, int cpg, int rank) {
    GW w{0, 0, 0, 0, 0};
    const int64_t grid = (int64_t)sc.a * sc.b;
    if (sc.n_qq <= 0) return w;
    if (wg < grid) {
        int64_t x = wg / sc.b, y = wg - x * sc.b;
        w.r_lo = y * (int64_t)sc.r_main / sc.b; w.r_hi = (y + 1) * (int64_t)sc.r_main / sc.b;
        w.q_lo = x * sc.tpx; w.q_hi = std::min<int64_t>(sc.n_qq, (x + 1) * sc.tpx);
        w.slot = sc.slot0 + (wg * cpg + rank) * sc.tpx;
    } else if (wg < grid + sc.t_groups) {
        int64_t t = wg - grid;
        w.r_lo = sc.r_main; w.r_hi = n_rt;
        w.q_lo = std::min<int64_t>(sc.n_qq, t * sc.t_tpx); w.q_hi = std::min<int64_t>(sc.n_qq, (t + 1) * sc.t_tpx);
        w.slot = sc.slot0 + grid * cpg * sc.tpx + (t * cpg + rank) * sc.t_tpx;
    }
    return w;
}
int main() {
    int bad = 0, n_tail = 0, cases = 0;
    for (int G : {76, 152, 75, 10}) for (int cpg : {1, 2}) for (int64_t nqq = 1; nqq <= 40; ++nqq)
    for (int64_t nrt : {1ll, 2ll, 3ll, 7ll, 100ll, 3907ll, 15625ll, 78125ll}) {
        int64_t tb = 512 * 1024;
        TcSched sc[1]; int32_t order[1]; int32_t ns = 0;
        int32_t groups = make_tensor_schedule(1, &nqq, &nrt, &tb, G, cpg, sc, order, &ns);
        ++cases;
        if (groups < 1 || groups > G) { printf("groups %d G %d\n", groups, G); ++bad; continue; }
        if (sc[0].t_groups) ++n_tail;
        // coverage: each (qq, rt) once; slots: unique per (group cta, qq), < ns
        std::vector<int> cov(nqq * nrt, 0);
        std::set<int64_t> slots;
        for (int64_t wg = 0; wg < groups; ++wg) for (int rank = 0; rank < cpg; ++rank) {
            GW w = gw(sc[0], nrt, wg, cpg, rank);
            if (w.q_lo >= w.q_hi) continue;
            for (int64_t qq = w.q_lo; qq < w.q_hi; ++qq) {
                int64_t s = w.slot + (qq - w.q_lo);
                if (s < 0 || s >= ns || !slots.insert(s).second) { printf("slot %lld ns %d\n", (long long)s, ns); ++bad; }
                if (rank == 0) for (int64_t rt = w.r_lo; rt < w.r_hi; ++rt) cov[qq * nrt + rt]++;
            }
        }
        for (size_t i = 0; i < cov.size(); ++i) if (cov[i] != 1) { printf("cov G%d nqq%lld nrt%lld i%zu=%d\n", G, (long long)nqq, (long long)nrt, i, cov[i]); ++bad; break; }
        // merge's slot formula equals the owning group's slot
        for (int64_t qq = 0; qq < nqq; ++qq) for (int rank = 0; rank < cpg; ++rank) {
            const TcSched &s = sc[0];
            int64_t x = qq / s.tpx, li = qq - x * s.tpx;
            for (int64_t y = 0; y < s.b; ++y) {
                int64_t wg = x * s.b + y; int64_t cta = cpg == 2 ? 2 * wg + rank : wg;
                int64_t slot = s.slot0 + cta * s.tpx + li;
                GW w = gw(s, nrt, wg, cpg, rank);
                if (w.r_lo < w.r_hi && slot != w.slot + (qq - w.q_lo)) { printf("merge slot mismatch\n"); ++bad; }
            }
            if (s.t_groups > 0) {
                int64_t t = qq / s.t_tpx, lt = qq - t * s.t_tpx;
                int64_t slot = s.slot0 + (int64_t)s.a * s.b * cpg * s.tpx + (t * cpg + rank) * s.t_tpx + lt;
                GW w = gw(s, nrt, (int64_t)s.a * s.b + t, cpg, rank);
                if (slot != w.slot + (qq - w.q_lo)) { printf("tail merge slot mismatch\n"); ++bad; }
            }
        }
        if (G == 76 && cpg == 2 && (nqq == 8 || nqq == 3) && (nrt == 78125 || nrt == 3907))
            printf("G%d nqq%lld nrt%lld: a%d b%d tpx%d chunk%d pf%d r_main%d t_groups%d t_tpx%d t_chunk%d groups%d slots%d\n",
                   G, (long long)nqq, (long long)nrt, sc[0].a, sc[0].b, sc[0].tpx, sc[0].chunk, sc[0].pf, sc[0].r_main,
                   sc[0].t_groups, sc[0].t_tpx, sc[0].t_chunk, groups, ns);
    }
    printf("cases %d with tail %d bad %d\n", cases, n_tail, bad);
    return bad != 0;
}
