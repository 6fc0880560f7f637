"""Parity at full size for the batched and serving workloads, in the launch
configurations bench.py times:

  * batched: 256 batches of 1-512 queries over four loci panels (N = 512,
    2048, 8192, 16384) of 4,000,000 references each, top-16, one persistent
    launch per run (the autotuned plan variant, graph replay);
  * serving: Poisson arrivals of 1-256-query requests against 20,000,000
    references at N = 2048, top-16, through the server with the bench's
    defaults (one wave in flight, waves of at most 256 queries).

The oracle cannot score every pair here, so for every query list:
  * each returned (query, reference) score equals the oracle's, pair by pair;
  * the list is sorted by (score, reference), and empty slots come last;
  * no reference of a seeded sample beats the list's k-th entry, and every
    sampled reference that belongs in the list is in it;
  * every planted contributor (score 0) is found.
Serving also has to return, for every request, exactly what the same request
returns alone through fastid_topk (which the 20M-reference parity test covers
against the oracle). The batched plan's host-buffer path has to return what its
device path returns.

The reference rows the checks need are regenerated by the seeded generator's
device form. A few rows of every set are compared with the host form
(gen.allele_rows), so the oracle's inputs are the generator's published
draws.
"""
import time

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher  # noqa: E402

UINT32_MAX = 0xFFFFFFFF


def _rows(seed, thr, thr_dev, rows, stream=gen.STREAM_DB):
    """Allele rows (uint8 [len(rows), n_loci]) of a generator stream, made on
    the device; three of them are checked against the host generator."""
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    n_loci = thr.shape[0]
    if rows.size == 0:
        return np.zeros((0, n_loci), np.uint8)
    out = torch.empty((rows.size, n_loci), dtype=torch.uint8, device="cuda")
    gen.allele_rows_device(seed, stream, thr_dev, out, rows_dev=torch.from_numpy(rows).cuda())
    R = out.cpu().numpy()
    pos = np.unique([0, rows.size // 2, rows.size - 1])
    assert np.array_equal(R[pos], gen.allele_rows(seed, stream, rows[pos], thr))
    return R


def _query_alleles(rec, seed, thr, thr_dev):
    """Unpacked queries of a recipe: its contributors' rows, OR-ed per query by
    oracle.mix."""
    src = np.empty((max(rec.n_sources, 1), thr.shape[0]), np.uint8)
    for stream in (gen.STREAM_DB, gen.STREAM_FRESH):
        sel = np.nonzero(rec.src_stream == stream)[0]
        if sel.size:
            src[sel] = _rows(seed, thr, thr_dev, rec.src_row[sel], stream)
    return oracle.mix(src[:rec.n_sources], rec.offsets)


def _check_lists(sc, ix, Q, modes, planted, k, T, seed, thr, thr_dev, n_refs, n_sample, rng):
    """The checks of the module docstring for the lists (sc, ix) [n_q, k] of
    the queries Q (unpacked) with their modes."""
    valid = ix >= 0
    # 1. every returned pair, one at a time
    qi = np.nonzero(valid)[0]
    ri = ix[valid]
    uniq, inv = np.unique(ri, return_inverse=True)
    mis, une = oracle.score_pairs(_rows(seed, thr, thr_dev, uniq), Q, qi, inv)
    assert np.array_equal(sc[valid], np.where(modes[qi] == gen.MODE_MISMATCH, mis, une))
    # 2. sorted by (score, reference), empty slots last, within the threshold
    key = np.where(valid, sc.astype(np.uint64) << np.uint64(32) | ix.astype(np.uint64) & np.uint64(0xFFFFFFFF),
                   np.uint64(0xFFFFFFFFFFFFFFFF))
    assert np.all(key[:, 1:] >= key[:, :-1])
    assert np.all(np.diff(key, axis=1)[valid[:, 1:]] > 0)
    if T != UINT32_MAX:
        assert np.all(sc[valid] <= T)
    # 3. sampled references
    sample = np.sort(rng.choice(n_refs, n_sample, replace=False))
    smis, sune = oracle.scores(_rows(seed, thr, thr_dev, sample), Q)
    ss = oracle.select(smis, sune, modes)
    skey = ss.astype(np.uint64) << np.uint64(32) | sample.astype(np.uint64)[None, :]
    ok_t = ss <= T if T != UINT32_MAX else np.ones_like(ss, dtype=bool)
    should = ok_t & (skey <= key[:, -1][:, None])
    for j in range(Q.shape[0]):
        need = set(sample[should[j]].tolist())
        assert need <= set(ix[j][valid[j]].tolist()), (j, sorted(need - set(ix[j].tolist()))[:5])
    # 4. planted contributors
    for j, rows in enumerate(planted):
        for r in rows:
            assert r in ix[j], (j, r)


def test_c4_batched_fullsize():
    import __graft_entry__
    import bench
    from paper_1707_00516_gb300.batched import BatchedSearch
    from paper_1707_00516_gb300.tune import Autotuner
    __graft_entry__.build()
    w = dict(bench.WORKLOADS["c4"])
    s = Searcher(0, B.FORM_TENSOR)
    seed, sizes, panels = bench._c4_batches(w)
    dbs, thrs, thr_devs = [], [], []
    for p, n_loci in enumerate(w["panels"]):
        db, thr = bench.build_db(s, seed + 10 * p, w["n_refs"], n_loci, B.REFS_TENSOR | B.REFS_FP4, chunk=(1 << 28) // n_loci)
        dbs.append(db)
        thrs.append(thr)
        thr_devs.append(torch.from_numpy(thr.view(np.int32)).cuda())
    bs = BatchedSearch(s.ctx, dbs, panels, sizes, w["k"], w["threshold"], tuner=Autotuner())
    recs, host_q, host_m = [], [], []
    for b, (n, p) in enumerate(zip(sizes, panels)):
        rec = bench._c4_recipe(w, b, int(n), int(p), seed)
        q, m = bench.device_queries(s, seed + 10 * p, rec, thr_devs[p], w["panels"][p])
        bs.set_queries(b, q, m)
        recs.append(rec)
        host_q.append(q.cpu().numpy().view(np.uint64))
        host_m.append(m.cpu().numpy())
    for _ in range(2):  # graph replays, as the bench's steps
        bs.run_device()
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    res = [tuple(t.cpu().numpy().copy() for t in bs.results(b)) for b in range(len(sizes))]
    # the host-buffer path returns the same lists
    h_sc, h_ix, _, _ = bs.run_host(host_q, host_m)
    for b in range(len(sizes)):
        assert np.array_equal(np.asarray(h_sc[b]).view(np.uint32), res[b][0].view(np.uint32)), b
        assert np.array_equal(np.asarray(h_ix[b]), res[b][1]), b
    bs.close()
    for d in dbs:
        d.close()
    s.ctx.close()
    rng = np.random.default_rng(seed + 4)
    for p, n_loci in enumerate(w["panels"]):
        bsel = [b for b in range(len(sizes)) if panels[b] == p and sizes[b] > 0]
        if not bsel:
            continue
        sc = np.concatenate([res[b][0].view(np.uint32) for b in bsel])
        ix = np.concatenate([res[b][1] for b in bsel])
        Q = np.concatenate([_query_alleles(recs[b], seed + 10 * p, thrs[p], thr_devs[p]) for b in bsel])
        modes = np.concatenate([recs[b].modes for b in bsel])
        planted = [recs[b].planted(j) for b in bsel for j in range(recs[b].n_queries)]
        # fewer sampled references on the widest panels keeps the oracle to seconds
        n_sample = 4096 if n_loci <= 2048 else 1024
        _check_lists(sc, ix, Q, modes, planted, w["k"], w["threshold"], seed + 10 * p, thrs[p], thr_devs[p],
                     w["n_refs"], n_sample, rng)


SERVE_SECONDS = 1.5


def test_c5_serving_fullsize():
    import __graft_entry__
    import bench
    __graft_entry__.build()
    w = dict(bench.WORKLOADS["c5"])
    n_refs, n_loci, k, T = w["n_refs"], w["n_loci"], w["k"], w["threshold"]
    s = Searcher(0, B.FORM_AUTO)
    seed = gen.config_seed(w["cfg"])
    db, thr = bench.build_db(s, seed, n_refs, n_loci, B.REFS_FP4)
    thr_dev = torch.from_numpy(thr.view(np.int32)).cuda()
    arrivals, sizes, rec = bench.c5_requests(w, seed, SERVE_SECONDS)
    q, m = bench.device_queries(s, seed, rec, thr_dev, n_loci)
    hq = q.cpu().numpy().view(np.uint64)
    hm = m.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    d = bench.C5_DEFAULTS
    srv = bench.make_server(d["server"], s.ctx, db, k, T, d["parts"], d["slots"], d["max_wave"], d["hbm_budget"])
    futs = []
    t0 = time.perf_counter()
    for i in range(arrivals.size):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(srv.submit(hq[offs[i]:offs[i + 1]], hm[offs[i]:offs[i + 1]]))
    got = [f.result(timeout=600) for f in futs]
    waves = srv.stats()["waves"]
    srv.close()
    assert waves < arrivals.size  # requests were coalesced
    # each request alone, through fastid_topk
    for i in range(arrivals.size):
        a_sc, a_ix = s.topk(db, q[offs[i]:offs[i + 1]], m[offs[i]:offs[i + 1]], k, T)
        assert np.array_equal(a_sc.cpu().numpy().view(np.uint32), got[i][0]), i
        assert np.array_equal(a_ix.cpu().numpy(), got[i][1]), i
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    db.close()
    s.ctx.close()
    sc = np.concatenate([g[0] for g in got])
    ix = np.concatenate([g[1] for g in got])
    Q = _query_alleles(rec, seed, thr, thr_dev)
    planted = [rec.planted(j) for j in range(rec.n_queries)]
    _check_lists(sc, ix, Q, rec.modes, planted, k, T, seed, thr, thr_dev, n_refs, 2048,
                 np.random.default_rng(seed + 5))
