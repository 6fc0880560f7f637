"""Parity at the full workload sizes, in the launch configuration bench.py
times: 2048 unknowns x 20,000,000 references (N = 2048, top-32, T = 512) and
2048 mixtures x 1,000,000 references (N = 4096, top-16 within score <= 0, and
the hit list at score <= 0).

The oracle cannot produce the whole score matrix here, so the checks are
  * every returned (query, reference) score equals the oracle's, computed one
    pair at a time;
  * each list is sorted by (score, reference) and within the threshold;
  * no reference of a seeded random sample of 4096 beats a list's k-th entry
    (and every sampled reference that should be in a list is);
  * every planted contributor (score 0) is found;
  * the plain and tensor forms return identical lists.
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher  # noqa: E402

CASES = {
    "c3": dict(n_refs=20_000_000, n_loci=2048, k=32, T=512, forms=("tensor", "plain")),
    "c2": dict(n_refs=1_000_000, n_loci=4096, k=16, T=0, forms=("tensor", "plain")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fullsize_sampled_parity(name):
    import __graft_entry__
    import bench
    __graft_entry__.build()
    cfg = CASES[name]
    n_refs, n_loci, k, T = cfg["n_refs"], cfg["n_loci"], cfg["k"], cfg["T"]
    seed = gen.config_seed(int(name[1]))
    s = Searcher(0, B.FORM_AUTO)
    db, thr = bench.build_db(s, seed, n_refs, n_loci, B.REFS_TENSOR)
    recipe = bench.recipe_for(name, n_refs=n_refs)
    thr_dev = torch.from_numpy(thr.view(np.int32)).cuda()
    q, modes = bench.device_queries(s, seed, recipe, thr_dev, n_loci)
    results, hits = {}, {}
    for form in cfg["forms"]:
        B.fastid_set_form(s.ctx, B.FORM_PLAIN if form == "plain" else B.FORM_TENSOR)
        sc, ix = s.topk(db, q, modes, k, T)
        torch.cuda.synchronize()
        assert B.fastid_sync_status(s.ctx) == B.OK
        results[form] = (sc.cpu().numpy().view(np.uint32).copy(), ix.cpu().numpy().copy())
        if T == 0:
            hq, hr, hs, hc = s.hits(db, q, modes, 0, 1 << 22)
            torch.cuda.synchronize()
            assert B.fastid_sync_status(s.ctx) == B.OK
            n = int(hc.item())
            hits[form] = (hq[:n].cpu().numpy(), hr[:n].cpu().numpy(), hs[:n].cpu().numpy().view(np.uint32))
    db.close()
    s.ctx.close()
    sc, ix = results[cfg["forms"][0]]
    for form in cfg["forms"][1:]:
        assert np.array_equal(results[form][0], sc) and np.array_equal(results[form][1], ix), form
        if hits:
            assert all(np.array_equal(a, b) for a, b in zip(hits[form], hits[cfg["forms"][0]])), form

    # host side: the queries' alleles (oracle mix of regenerated contributors)
    Q = oracle.mix(gen.source_alleles(recipe, thr), recipe.offsets)
    n_q = Q.shape[0]
    valid = ix >= 0
    # 1. every returned pair, one at a time
    qi = np.nonzero(valid)[0]
    ri = ix[valid]
    uniq, inv = np.unique(ri, return_inverse=True)
    R_ret = gen.allele_rows(seed, gen.STREAM_DB, uniq, thr)
    mis, une = oracle.score_pairs(R_ret, Q, qi, inv)
    exp = np.where(recipe.modes[qi] == gen.MODE_MISMATCH, mis, une)
    assert np.array_equal(sc[valid], exp)
    # 2. sorted by (score, ref), within the threshold, empty slots at the end
    key = np.where(valid, sc.astype(np.uint64) << np.uint64(32) | ix.astype(np.uint64) & np.uint64(0xFFFFFFFF),
                   np.uint64(0xFFFFFFFFFFFFFFFF))
    assert np.all(key[:, 1:] >= key[:, :-1])
    assert np.all(np.diff(key, axis=1)[valid[:, 1:]] > 0)
    if T != 0xFFFFFFFF:
        assert np.all(sc[valid] <= T)
    # 3. sampled references never beat the k-th entry, and belong when they should
    rng = np.random.default_rng(seed + 99)
    sample = np.sort(rng.choice(n_refs, 4096, replace=False))
    R_s = gen.allele_rows(seed, gen.STREAM_DB, sample, thr)
    smis, sune = oracle.scores(R_s, Q)
    ss = oracle.select(smis, sune, recipe.modes)
    kth = key[:, -1]
    skey = ss.astype(np.uint64) << np.uint64(32) | sample.astype(np.uint64)[None, :]
    ok_t = ss <= T if T != 0xFFFFFFFF else np.ones_like(ss, dtype=bool)
    should = ok_t & (skey <= kth[:, None])
    for j in range(n_q):
        got = set(ix[j][valid[j]].tolist())
        need = set(sample[should[j]].tolist())
        assert need <= got, (j, sorted(need - got)[:5])
    # 4. planted contributors
    for j in range(n_q):
        for r in recipe.planted(j):
            assert r in ix[j], (j, r)
    # 5. the hit list at score <= 0: every hit scores 0, sorted by (q, r); it
    #    holds every planted contributor and every sampled zero
    if hits:
        hq, hr, hs = hits[cfg["forms"][0]]
        assert np.all(hs == 0)
        assert np.all(np.diff(hq * n_refs + hr) > 0)
        uh, ih = np.unique(hr, return_inverse=True)
        Rh = gen.allele_rows(seed, gen.STREAM_DB, uh, thr)
        hmis, hune = oracle.score_pairs(Rh, Q, hq, ih)
        assert np.all(np.where(recipe.modes[hq] == gen.MODE_MISMATCH, hmis, hune) == 0)
        hit_set = set(zip(hq.tolist(), hr.tolist()))
        for j in range(n_q):
            for r in recipe.planted(j):
                assert (j, r) in hit_set, (j, r)
        zq, zr = np.nonzero(ss == 0)
        assert set(zip(zq.tolist(), sample[zr].tolist())) <= hit_set
