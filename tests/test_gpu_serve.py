"""Continuous-batching server: requests that arrive while others run are
coalesced into waves on several slots, and every request's result equals its
result when run alone (and the oracle's)."""
import threading

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher  # noqa: E402
from paper_1707_00516_gb300.serve import Server  # noqa: E402


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, B.FORM_TENSOR)
    n_refs, n_loci, seed = 12000, 700, 333
    thr = gen.maf_thresholds(seed, n_loci)
    R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
    yield s, db, R, thr, seed
    db.close()
    s.ctx.close()


def _requests(R, thr, seed, n_req, rng):
    reqs = []
    for i in range(n_req):
        n = int(rng.integers(1, 65))
        rec = gen.recipe_mixtures(n, R.shape[0], R.shape[1], seed, 1, 5, fresh_base=(i + 1) << 22, salt=7000 + i)
        rec.modes[:] = rng.integers(0, 2, n).astype(np.uint8)
        Q = oracle.mix(gen.source_alleles(rec, thr), rec.offsets)
        reqs.append((oracle.pack(Q), rec.modes.copy(), Q))
    return reqs


def test_results_alone_equal_results_in_the_mix(env):
    s, db, R, thr, seed = env
    k, T = 16, 200
    rng = np.random.default_rng(1)
    reqs = _requests(R, thr, seed, 48, rng)
    # alone: one fastid_topk per request
    alone = []
    for packed, modes, _ in reqs:
        q = torch.from_numpy(packed.view(np.int64)).cuda()
        sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), k, T)
        alone.append((sc.cpu().numpy().view(np.uint32), ix.cpu().numpy()))
    # in the mix: four client threads submit concurrently
    srv = Server(s.ctx, db, k, T, hbm_budget_bytes=256 << 20, max_wave=512, max_slots=3)
    futs = [None] * len(reqs)

    def client(ids):
        for i in ids:
            futs[i] = srv.submit(reqs[i][0], reqs[i][1])

    threads = [threading.Thread(target=client, args=(list(range(t, len(reqs), 4)),)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = [f.result(timeout=120) for f in futs]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs)
    assert st["waves"] < len(reqs)  # requests were coalesced
    for (a_sc, a_ix), (g_sc, g_ix) in zip(alone, got):
        assert np.array_equal(a_sc, g_sc) and np.array_equal(a_ix, g_ix)
    # and alone equals the oracle (spot-check a few requests)
    for i in (0, 17, 47):
        _, modes, Q = reqs[i]
        mis, une = oracle.scores(R, Q)
        es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
        assert np.array_equal(got[i][0], es) and np.array_equal(got[i][1], ei)


def test_budget_limits_slots(env):
    s, db, R, thr, seed = env
    srv = Server(s.ctx, db, 8, hbm_budget_bytes=1, max_wave=256, max_slots=4)
    assert len(srv.slots) == 1  # the budget admits one slot at a time
    rng = np.random.default_rng(2)
    reqs = _requests(R, thr, seed, 6, rng)
    futs = [srv.submit(p, m) for p, m, _ in reqs]
    for f in futs:
        f.result(timeout=60)
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit(reqs[0][0], reqs[0][1])


def test_device_condition_fails_its_wave(env):
    """A condition the device records (here a bounded wait that ran out,
    planted through fastid_wait_flag on the server's context while it is
    idle) fails the requests of the wave that reads it with FASTID_ETIMEOUT;
    the status word is cleared, and the next wave's results are delivered and
    equal the oracle's.  No GPU fault or hang is involved."""
    s, db, R, thr, seed = env
    reqs = _requests(R, thr, seed, 2, np.random.default_rng(11))
    srv = Server(s.ctx, db, 8, B.NO_THRESHOLD, hbm_budget_bytes=1 << 30, max_wave=512, max_slots=1)
    try:
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.fastid_wait_flag(s.ctx, flag, 50)  # nothing sets the flag: the wait runs out
        torch.cuda.synchronize()
        f = srv.submit(reqs[0][0], reqs[0][1])
        with pytest.raises(B.FastIDError) as e:
            f.result(timeout=120)
        assert e.value.status == B.ETIMEOUT
        sc, ix = srv.submit(reqs[1][0], reqs[1][1]).result(timeout=120)
        mis, une = oracle.scores(R, reqs[1][2])
        es, ei = oracle.topk(oracle.select(mis, une, reqs[1][1]), 8)
        assert np.array_equal(sc, es) and np.array_equal(ix, ei)
    finally:
        srv.close()
    assert B.fastid_sync_status(s.ctx) == B.OK
