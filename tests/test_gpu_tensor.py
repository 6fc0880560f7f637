"""Tensor form (tcgen05, e4m3 operands, FP32 accumulation): exactness at the
largest loci counts and form selection, for both reference operands -- the
database's FP8 copy and the packed rows expanded on chip.  Scores are
integers; the test is equality with the oracle."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402


TENSOR_FORMS = {"fp8": B.FORM_TENSOR, "packed": B.FORM_TENSOR_PACKED, "fp4": B.FORM_TENSOR_FP4,
                "fp4packed": B.FORM_TENSOR_FP4_PACKED}


@pytest.fixture(scope="module", params=list(TENSOR_FORMS))
def ts(request):
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, TENSOR_FORMS[request.param])
    yield s
    s.ctx.close()


def _full(s, R, Q, modes, n_loci, dtype=torch.int32):
    db = s.load_refs_alleles(torch.from_numpy(np.ascontiguousarray(R)).cuda(), n_loci)
    q = torch.empty((Q.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), n_loci, q)
    out = s.scores(db, q, torch.from_numpy(modes).cuda(), dtype)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    db.close()
    return out.cpu().numpy().view(np.uint32 if dtype == torch.int32 else np.uint16)


def test_tiny(ts):
    rng = np.random.default_rng(0)
    R = (rng.random((5, 200)) < 0.5).astype(np.uint8)
    Q = (rng.random((3, 200)) < 0.5).astype(np.uint8)
    modes = np.array([0, 1, 0], np.uint8)
    mis, une = oracle.scores(R, Q)
    assert np.array_equal(_full(ts, R, Q, modes, 200), oracle.select(mis, une, modes))


@pytest.mark.parametrize("n_loci", [16384, 65536])
def test_extreme_counts_exact(ts, n_loci):
    """All-ones / all-zero / alternating profiles drive the accumulators to
    +-N, the largest magnitudes the FP32 accumulation must hold exactly."""
    R = np.zeros((6, n_loci), np.uint8)
    R[0] = 1
    R[2, ::2] = 1
    R[3, 1::2] = 1
    R[4, : n_loci // 3] = 1
    R[5] = 1
    R[5, -1] = 0
    Q = np.stack([R[0], R[1], R[2], R[5], R[0], R[1]])
    modes = np.array([0, 0, 0, 1, 1, 1], np.uint8)
    mis, une = oracle.scores(R, Q)
    got = _full(ts, R, Q, modes, n_loci)
    assert np.array_equal(got, oracle.select(mis, une, modes))
    assert got.max() == n_loci  # reached the extreme


@pytest.mark.parametrize("n_loci,p", [(16384, 0.5), (32768, 0.3), (65536, 0.7)])
def test_random_large_n_exact(ts, n_loci, p):
    rng = np.random.default_rng(n_loci)
    R = (rng.random((37, n_loci)) < p).astype(np.uint8)
    Q = (rng.random((9, n_loci)) < p).astype(np.uint8)
    modes = (np.arange(9) % 2).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    assert np.array_equal(_full(ts, R, Q, modes, n_loci), oracle.select(mis, une, modes))


def test_uint16_scores(ts):
    rng = np.random.default_rng(3)
    R = (rng.random((300, 1024)) < 0.4).astype(np.uint8)
    Q = (rng.random((129, 1024)) < 0.4).astype(np.uint8)
    modes = (np.arange(129) % 3 == 0).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    exp = oracle.select(mis, une, modes).astype(np.uint16)
    assert np.array_equal(_full(ts, R, Q, modes, 1024, torch.int16), exp)


def test_tensor_form_on_packed_only_database(ts):
    """A database loaded without its FP8 copy still takes the tensor form: the
    packed rows are expanded on chip."""
    rng = np.random.default_rng(3)
    R = (rng.random((700, 300)) < 0.4).astype(np.uint8)
    Q = (rng.random((9, 300)) < 0.4).astype(np.uint8)
    modes = np.array([0, 1] * 4 + [1], np.uint8)
    db = ts.load_refs_alleles(torch.from_numpy(R).cuda(), 300, flags=0)
    assert db.info()["flags"] == 0
    q = torch.empty((9, words64(300)), dtype=torch.int64, device="cuda")
    B.fastid_pack(ts.ctx, torch.from_numpy(Q).cuda(), 300, q)
    sc, ix = ts.topk(db, q, torch.from_numpy(modes).cuda(), 5)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), 5, B.NO_THRESHOLD)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)
    db.close()
    db2 = ts.load_refs_alleles(torch.from_numpy(R).cuda(), 300, flags=B.REFS_TENSOR)
    assert db2.info()["flags"] == B.REFS_TENSOR
    db2.close()


@pytest.mark.parametrize("n_q,n_refs,k", [(600, 7000, 32), (1024, 20000, 32), (513, 3000, 32), (600, 7000, 16),
                                         (513, 3000, 9)])
def test_paired_launch_parity(ts, n_q, n_refs, k):
    """Enough query tiles for the paired (2-CTA cluster, multicast) launch,
    including an odd tile count (a padding tile in the last pair), with the
    32-slot (k > 16) and 16-slot top-k lists."""
    import gen
    n_loci, seed = 1536, 77 + n_q
    thr = gen.maf_thresholds(seed, n_loci)
    R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
    rec = gen.concat_recipes(gen.recipe_individuals(n_q // 2, n_refs, n_loci, seed, n_planted=50),
                             gen.recipe_mixtures(n_q - n_q // 2, n_refs, n_loci, seed, 2, 5))
    Q = oracle.mix(gen.source_alleles(rec, thr), rec.offsets)
    db = ts.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
    q = torch.empty((n_q, words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(ts.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
    modes = torch.from_numpy(rec.modes).cuda()
    mis, une = oracle.scores(R, Q)
    exp = oracle.select(mis, une, rec.modes)
    sc, ix = ts.topk(db, q, modes, k, 300)
    es, ei = oracle.topk(exp, k, 300)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)
    full = ts.scores(db, q, modes, torch.int32)
    assert np.array_equal(full.cpu().numpy().view(np.uint32), exp)
    hq, hr, hs, hc = ts.hits(db, q, modes, 20, 1 << 20)
    oq, orr, osc = oracle.hits(exp, 20)
    n = int(hc.item())
    assert n == oq.size and np.array_equal(hq[:n].cpu().numpy(), oq) and np.array_equal(hr[:n].cpu().numpy(), orr)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(ts.ctx) == B.OK
    db.close()


@pytest.mark.parametrize("n_q,k", [(100, 12), (128, 12), (129, 12), (256, 12), (257, 12), (300, 12), (600, 12),
                                   (128, 32), (129, 32)])
def test_auto_form_both_operands(n_q, k):
    """FASTID_FORM_AUTO takes the FP4 form: the packed rows up to 128 queries and
    the database's FP4 copy above (paired from two query tiles on; 300 queries
    pad to four tiles): results equal the oracle on both sides of the switch."""
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, B.FORM_AUTO)
    rng = np.random.default_rng(n_q)
    R = (rng.random((3000, 700)) < 0.3).astype(np.uint8)
    Q = (rng.random((n_q, 700)) < 0.3).astype(np.uint8)
    modes = (rng.random(n_q) < 0.5).astype(np.uint8)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), 700)
    assert db.info()["flags"] == B.REFS_FP4
    q = torch.empty((n_q, words64(700)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), 700, q)
    sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), k, 400)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k, 400)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)
    db.close()
    s.ctx.close()


def test_schedule_tail_exact():
    """2048 queries x 100,000 references at N = 96 (words ragged), top-16. The
    schedule is 8 tile pairs on 76 clusters: an 8 x 9 grid over the first 374
    reference tiles plus a tail of 4 clusters x 2 pairs over the last 17. The
    unpaired packed form gets a 16 x 9 grid plus 8 x 2; the FP4 forms (224
    references a tile) get their own grids and tails. Every form's lists equal
    the oracle's element by element, so every tail slot is written and merged."""
    import __graft_entry__
    __graft_entry__.build()
    n_refs, n_loci, n_q, k = 100_000, 96, 2048, 16
    rng = np.random.default_rng(2024)
    thr = gen.maf_thresholds(31, n_loci)
    R = gen.allele_rows(31, gen.STREAM_DB, np.arange(n_refs), thr)
    Q = (rng.random((n_q, n_loci)) < 0.35).astype(np.uint8)
    Q[:64] = R[rng.integers(0, n_refs, 64)]
    modes = (rng.random(n_q) < 0.5).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k)
    for form in (B.FORM_TENSOR, B.FORM_TENSOR_PACKED, B.FORM_TENSOR_FP4, B.FORM_TENSOR_FP4_PACKED):
        s = Searcher(0, form)
        db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
        q = torch.empty((n_q, words64(n_loci)), dtype=torch.int64, device="cuda")
        B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
        sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), k)
        torch.cuda.synchronize()
        assert B.fastid_sync_status(s.ctx) == B.OK
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), es), form
        assert np.array_equal(ix.cpu().numpy(), ei), form
        db.close()
        s.ctx.close()
