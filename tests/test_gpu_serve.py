"""Continuous-batching servers: requests that arrive while others run are
coalesced into waves (on slots: Server; joining a running pass over the
database's parts: SweepServer), and every request's result equals its result
when run alone (and the oracle's)."""
import time
import threading

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher  # noqa: E402
from paper_1707_00516_gb300.serve import Server, SweepServer  # noqa: E402


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


def _alone(s, db, reqs, k, T):
    out = []
    for packed, modes, _ in reqs:
        q = torch.from_numpy(packed.view(np.int64)).cuda()
        sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), k, T)
        out.append((sc.cpu().numpy().view(np.uint32), ix.cpu().numpy()))
    return out


@pytest.mark.parametrize("form", [B.FORM_AUTO, B.FORM_TENSOR, B.FORM_PLAIN])
def test_sweep_alone_equal_mix(env, form):
    """SweepServer: 48 requests from four client threads, waves joining the
    running pass over three parts; each result equals the request alone and
    the oracle."""
    s, db, R, thr, seed = env
    B.fastid_set_form(s.ctx, form)
    k, T = 16, 200
    reqs = _requests(R, thr, seed, 48, np.random.default_rng(5))
    alone = _alone(s, db, reqs, k, T)
    srv = SweepServer(s.ctx, db, k, T, parts=3, capacity=1024, max_wave=256)
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
    B.fastid_set_form(s.ctx, B.FORM_TENSOR)
    assert st["requests"] == len(reqs) and st["waves"] < len(reqs)
    for (a_sc, a_ix), (g_sc, g_ix) in zip(alone, got):
        assert np.array_equal(a_sc, g_sc) and np.array_equal(a_ix, g_ix)
    for i in (0, 23, 47):
        _, modes, Q = reqs[i]
        mis, une = oracle.scores(R, Q)
        es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
        assert np.array_equal(got[i][0], es) and np.array_equal(got[i][1], ei)


def test_sweep_waves_share_launches(env):
    """A second burst of requests submitted while the first wave is still in
    its pass joins the running pass: some steps (one comparison launch each)
    serve both waves, and by the device timestamps of the steps the second
    wave's work starts before the first wave's work ends.  Results equal the
    oracle."""
    s, db, R, thr, seed = env
    k, T = 8, B.NO_THRESHOLD
    reqs = _requests(R, thr, seed, 8, np.random.default_rng(9))
    srv = SweepServer(s.ctx, db, k, T, parts=16, capacity=1024, max_wave=256)
    srv.trace = []
    first = [srv.submit(p, m) for p, m, _ in reqs[:4]]
    t0 = time.perf_counter()
    while srv.steps < 1 and time.perf_counter() - t0 < 30:
        time.sleep(0.0002)
    second = [srv.submit(p, m) for p, m, _ in reqs[4:]]
    got = [f.result(timeout=120) for f in first + second]
    trace = list(srv.trace)
    srv.close()
    torch.cuda.synchronize()
    waves = []  # wave ids in the order they first appear
    for _, _, ids in trace:
        for w in ids:
            if w not in waves:
                waves.append(w)
    assert len(waves) >= 2
    shared = [ids for _, _, ids in trace if waves[0] in ids and waves[1] in ids]
    assert shared, "no launch served both waves"
    base = trace[0][0]
    span = {w: (min(base.elapsed_time(a) for a, _, ids in trace if w in ids),
                max(base.elapsed_time(b) for _, b, ids in trace if w in ids)) for w in waves[:2]}
    assert span[waves[1]][0] < span[waves[0]][1]  # overlapping on the device
    for i, (_, modes, Q) in enumerate(reqs):
        mis, une = oracle.scores(R, Q)
        es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
        assert np.array_equal(got[i][0], es) and np.array_equal(got[i][1], ei), i


def test_sweep_ring_admission(env):
    """A ring that holds one full wave: requests wait for rows, the ring
    wraps, and every result is still the request's result alone."""
    s, db, R, thr, seed = env
    k, T = 4, 150
    reqs = _requests(R, thr, seed, 20, np.random.default_rng(13))
    alone = _alone(s, db, reqs, k, T)
    srv = SweepServer(s.ctx, db, k, T, parts=2, capacity=100, max_wave=64)
    with pytest.raises(ValueError):
        srv.submit(np.zeros((65, srv.words), np.uint64), np.zeros(65, np.uint8))
    futs = [srv.submit(p, m) for p, m, _ in reqs]
    got = [f.result(timeout=120) for f in futs]
    srv.close()
    for (a_sc, a_ix), (g_sc, g_ix) in zip(alone, got):
        assert np.array_equal(a_sc, g_sc) and np.array_equal(a_ix, g_ix)


def test_sweep_device_condition_fails_its_wave(env):
    """As for Server: a planted bounded-wait timeout fails the wave that reads
    it with FASTID_ETIMEOUT, and the next wave is delivered, equal to the
    oracle.  No GPU fault or hang is involved."""
    s, db, R, thr, seed = env
    reqs = _requests(R, thr, seed, 2, np.random.default_rng(17))
    srv = SweepServer(s.ctx, db, 8, B.NO_THRESHOLD, parts=3, capacity=512, max_wave=256)
    try:
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.fastid_wait_flag(s.ctx, flag, 50)
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
