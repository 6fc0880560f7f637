"""fastid_topk_noalloc, the top-k entry point for callers that cannot allocate
device memory (services with a fixed memory budget, plug-ins whose host owns
every device allocation, latency-critical loops that avoid allocator calls).

It must give exactly what fastid_topk gives, call after call, although its
scratch is one fixed array in the library that keeps the previous call's
contents.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.search import Searcher
    s = Searcher(0, B.FORM_PLAIN)
    n_refs, n_loci, seed = 30000, 1000, 4242
    thr = gen.maf_thresholds(seed, n_loci)
    R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
    yield B, s, db, thr, n_refs, n_loci, seed, R
    db.close()
    s.ctx.close()


def _queries(s, rec, thr, n_loci):
    src = torch.from_numpy(gen.source_alleles(rec, thr)).cuda()
    q = s.build_queries(src, torch.from_numpy(rec.offsets).cuda(), n_loci).clone()
    return q, torch.from_numpy(rec.modes).cuda()


def _run(B, fn, s, db, q, modes, k, T):
    sc = torch.full((q.shape[0], k), 7, dtype=torch.int32, device="cuda")
    ix = torch.full((q.shape[0], k), 7, dtype=torch.int64, device="cuda")
    fn(s.ctx, db, q, modes, k, T, sc, ix)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    return sc.cpu().numpy(), ix.cpu().numpy()


def test_noalloc_matches_topk_on_consecutive_calls(env):
    B, s, db, thr, n_refs, n_loci, seed, R = env
    # two different query sets, so the second call runs over the first call's
    # leftovers in the shared array
    rec_a = gen.concat_recipes(gen.recipe_individuals(150, n_refs, n_loci, seed, n_planted=40),
                               gen.recipe_mixtures(170, n_refs, n_loci, seed, 2, 5))
    rec_b = gen.recipe_mixtures(77, n_refs, n_loci, seed, 2, 4, fresh_base=1 << 31, salt=0xD7)
    for rec, k, T in ((rec_a, 32, B.NO_THRESHOLD), (rec_b, 16, 60)):
        q, modes = _queries(s, rec, thr, n_loci)
        ref_sc, ref_ix = _run(B, B.fastid_topk, s, db, q, modes, k, T)
        got_sc, got_ix = _run(B, B.fastid_topk_noalloc, s, db, q, modes, k, T)
        # integer results: exact equality (zero tolerance, as every parity test here)
        assert np.array_equal(got_sc, ref_sc)
        assert np.array_equal(got_ix, ref_ix)
        for j in range(rec.n_queries):
            for r in rec.planted(j):
                assert r in got_ix[j]
    # the second call ran over the first call's leftovers: check it against
    # the oracle directly as well
    Q = oracle.mix(gen.source_alleles(rec_b, thr), rec_b.offsets)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, rec_b.modes), 16, 60)
    assert np.array_equal(got_sc.view(np.uint32), es)
    assert np.array_equal(got_ix, ei)


def test_noalloc_allocates_nothing(env):
    """After the first call on the device (which looks up the array's
    address), calls take nothing from the context's memory pool and leave
    the device's free memory unchanged, while fastid_topk does take pool
    scratch."""
    B, s, db, thr, n_refs, n_loci, seed, R = env
    rec = gen.recipe_mixtures(200, n_refs, n_loci, seed, 2, 5, salt=0xA1)
    q, modes = _queries(s, rec, thr, n_loci)
    sc = torch.empty((q.shape[0], 32), dtype=torch.int32, device="cuda")
    ix = torch.empty((q.shape[0], 32), dtype=torch.int64, device="cuda")
    B.fastid_topk_noalloc(s.ctx, db, q, modes, 32, B.NO_THRESHOLD, sc, ix)
    torch.cuda.synchronize()
    before = B.fastid_memory_info(s.ctx)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.fastid_topk_noalloc(s.ctx, db, q, modes, 32, B.NO_THRESHOLD, sc, ix)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    after = B.fastid_memory_info(s.ctx)
    assert after["pool_allocs"] == before["pool_allocs"]
    assert after["pool_used_bytes"] == before["pool_used_bytes"]
    assert free1 == free0
    B.fastid_topk(s.ctx, db, q, modes, 32, B.NO_THRESHOLD, sc, ix)
    torch.cuda.synchronize()
    assert B.fastid_memory_info(s.ctx)["pool_allocs"] > after["pool_allocs"]


def test_noalloc_rejects_oversized_request(env):
    B, s, db, thr, n_refs, n_loci, seed, R = env
    # 150,000 padded queries x 1024 bits of loci = 19.2 MB of padded queries
    # alone, plus ~50 MB of lists: over the fixed 32 MiB
    n_q = 150000
    q = torch.zeros((n_q, (n_loci + 63) // 64), dtype=torch.int64, device="cuda")
    modes = torch.ones(n_q, dtype=torch.uint8, device="cuda")
    sc = torch.empty((n_q, 32), dtype=torch.int32, device="cuda")
    ix = torch.empty((n_q, 32), dtype=torch.int64, device="cuda")
    with pytest.raises(B.FastIDError) as e:
        B.fastid_topk_noalloc(s.ctx, db, q, modes, 32, B.NO_THRESHOLD, sc, ix)
    assert e.value.status == B.EINVAL
    assert "FASTID_NOALLOC_SCRATCH_BYTES" in str(e.value)
