"""Host-streamed references (fastid_topk_streamed): the known profiles stay in
host memory and pass through the device in blocks.  The result must equal
the oracle's top-k (and fastid_topk on the same references loaded whole),
element by element, for every block size -- one block, ragged last blocks,
blocks of one tile, a block larger than the database -- both compute forms,
and pinned or pageable host memory."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402


FORMS = {"plain": B.FORM_PLAIN, "tensor": B.FORM_TENSOR, "packed": B.FORM_TENSOR_PACKED,
         "fp4packed": B.FORM_TENSOR_FP4}  # streamed FP4 blocks are expanded on chip


@pytest.fixture(scope="module", params=sorted(FORMS))
def searcher(request):
    """plain: padded rows per block; tensor: each block expanded to FP8;
    packed: padded rows per block, expanded on chip by the compare kernel."""
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, FORMS[request.param])
    s.form_name = request.param
    yield s
    s.ctx.close()


def _case(n_refs, n_loci, n_ind, n_mix, seed):
    thr = gen.maf_thresholds(seed, n_loci)
    R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
    rec = gen.concat_recipes(gen.recipe_individuals(n_ind, n_refs, n_loci, seed, n_planted=n_ind // 2),
                             gen.recipe_mixtures(n_mix, n_refs, n_loci, seed, 2, 5))
    Q = oracle.mix(gen.source_alleles(rec, thr), rec.offsets)
    return R, Q, rec.modes


def _pack_host(s, A, n_loci, pinned, pad_words=0):
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    w = words64(n_loci) + pad_words
    out = torch.zeros((A.shape[0], w), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, a, n_loci, out[:, :words64(n_loci)])
    h = out.cpu()
    return h.pin_memory() if pinned else h


def _flags(s):
    return B.REFS_TENSOR if s.form_name == "tensor" else 0


def _q(s, Q, n_loci):
    a = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    out = torch.empty((Q.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, a, n_loci, out)
    return out


@pytest.mark.parametrize("block", [5000, 1777, 256, 1, 100000])
@pytest.mark.parametrize("k,T", [(16, B.NO_THRESHOLD), (32, 120)])
def test_streamed_matches_oracle(searcher, block, k, T):
    n_refs, n_loci = 5000, 333
    if block == 1:
        n_refs = 300  # one reference per block: 300 blocks
    R, Q, modes = _case(n_refs, n_loci, 70, 60, seed=4242 + n_refs)
    refs = _pack_host(searcher, R, n_loci, pinned=True)
    q = _q(searcher, Q, n_loci)
    sc, ix = searcher.topk_streamed(refs, n_loci, q, torch.from_numpy(modes).cuda(), k, T, block_refs=block,
                                    flags=_flags(searcher))
    torch.cuda.synchronize()
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)


def test_streamed_pageable_and_row_stride(searcher):
    """Pageable host memory and a host row stride wider than the packed row."""
    n_refs, n_loci = 3000, 1031
    R, Q, modes = _case(n_refs, n_loci, 40, 40, seed=99)
    refs = _pack_host(searcher, R, n_loci, pinned=False, pad_words=3)
    q = _q(searcher, Q, n_loci)
    sc, ix = searcher.topk_streamed(refs, n_loci, q, torch.from_numpy(modes).cuda(), 8, block_refs=700,
                                    flags=_flags(searcher))
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), 8, B.NO_THRESHOLD)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)


def test_streamed_k_above_n_refs(searcher):
    R, Q, modes = _case(20, 64, 3, 3, seed=5)
    refs = _pack_host(searcher, R, 64, pinned=True)
    sc, ix = searcher.topk_streamed(refs, 64, _q(searcher, Q, 64), torch.from_numpy(modes).cuda(), 32,
                                    block_refs=7, flags=_flags(searcher))
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), 32, B.NO_THRESHOLD)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(ix.cpu().numpy(), ei)
    assert (ix.cpu().numpy()[:, 20:] == -1).all()


def test_streamed_equals_resident(searcher):
    """A larger database (several blocks of many tiles): identical to
    fastid_topk on the same references loaded whole."""
    n_refs, n_loci, n_q = 200_000, 1024, 600
    seed = 31337
    thr = gen.maf_thresholds(seed, n_loci)
    thr_dev = torch.from_numpy(thr.view(np.int32)).cuda()
    alle = torch.empty((n_refs, n_loci), dtype=torch.uint8, device="cuda")
    gen.allele_rows_device(seed, gen.STREAM_DB, thr_dev, alle)
    packed = torch.empty((n_refs, words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(searcher.ctx, alle, n_loci, packed)
    rec = gen.concat_recipes(gen.recipe_individuals(n_q // 2, n_refs, n_loci, seed, n_planted=40),
                             gen.recipe_mixtures(n_q - n_q // 2, n_refs, n_loci, seed, 2, 4))
    src = torch.from_numpy(gen.source_alleles(rec, thr)).cuda()
    q = searcher.build_queries(src, torch.from_numpy(rec.offsets).cuda(), n_loci)
    modes = torch.from_numpy(rec.modes).cuda()
    db = B.fastid_load_refs(searcher.ctx, packed, n_loci, _flags(searcher))
    sc0, ix0 = searcher.topk(db, q, modes, 16, B.NO_THRESHOLD)
    host = packed.cpu().pin_memory()
    sc1, ix1 = searcher.topk_streamed(host, n_loci, q, modes, 16, block_refs=65_536, flags=_flags(searcher))
    torch.cuda.synchronize()
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    assert torch.equal(sc0, sc1) and torch.equal(ix0, ix1)
    for j in range(n_q):  # planted rows are found
        for r in rec.planted(j):
            assert r in ix1[j].tolist()
    db.close()


def test_streamed_argument_errors(searcher):
    refs = torch.zeros((10, 1), dtype=torch.int64)
    q = torch.zeros((2, 1), dtype=torch.int64, device="cuda")
    m = torch.zeros(2, dtype=torch.uint8, device="cuda")
    sc = torch.empty((2, 4), dtype=torch.int32, device="cuda")
    ix = torch.empty((2, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(B.FastIDError):
        B.fastid_topk_streamed(searcher.ctx, refs, 64, 0, 0, q, m, 4, B.NO_THRESHOLD, sc, ix)  # block 0
    with pytest.raises(B.FastIDError):
        B.fastid_topk_streamed(searcher.ctx, refs, 64, 0, 4, q, m, 0, B.NO_THRESHOLD,
                               sc[:, :0], ix[:, :0])  # k = 0
    with pytest.raises(TypeError):
        B.fastid_topk_streamed(searcher.ctx, refs.cuda(), 64, 0, 4, q, m, 4, B.NO_THRESHOLD, sc, ix)


@pytest.mark.parametrize("block", [5000, 1777, 256])
def test_streamed_hits_match_oracle(searcher, block):
    """Hit lists over host-resident references: every (q, r) with score <= T,
    sorted by (q, r), reference indices global."""
    n_refs, n_loci, T = 5000, 333, 120
    R, Q, modes = _case(n_refs, n_loci, 50, 40, seed=777)
    refs = _pack_host(searcher, R, n_loci, pinned=True)
    q = _q(searcher, Q, n_loci)
    hq, hr, hs, hc = searcher.hits_streamed(refs, n_loci, q, torch.from_numpy(modes).cuda(), T, 1 << 20,
                                            block_refs=block, flags=_flags(searcher))
    torch.cuda.synchronize()
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    mis, une = oracle.scores(R, Q)
    oq, orr, osc = oracle.hits(oracle.select(mis, une, modes), T)
    n = int(hc.item())
    assert n == oq.size
    assert np.array_equal(hq[:n].cpu().numpy(), oq) and np.array_equal(hr[:n].cpu().numpy(), orr)
    assert np.array_equal(hs[:n].cpu().numpy().view(np.uint32), osc)


def test_streamed_hits_overflow(searcher):
    """More hits than capacity: the true count, a sorted valid subset, and
    FASTID_EOVERFLOW from the next status read."""
    n_refs, n_loci, T = 3000, 64, 40
    R, Q, modes = _case(n_refs, n_loci, 8, 8, seed=31)
    refs = _pack_host(searcher, R, n_loci, pinned=True)
    q = _q(searcher, Q, n_loci)
    mis, une = oracle.scores(R, Q)
    oq, orr, osc = oracle.hits(oracle.select(mis, une, modes), T)
    cap = oq.size // 3
    assert cap > 0
    hq, hr, hs, hc = searcher.hits_streamed(refs, n_loci, q, torch.from_numpy(modes).cuda(), T, cap, block_refs=700,
                                            flags=_flags(searcher))
    assert B.fastid_sync_status(searcher.ctx) == B.EOVERFLOW
    assert int(hc.item()) == oq.size
    got = set(zip(hq.cpu().tolist(), hr.cpu().tolist()))
    assert len(got) == cap and got <= set(zip(oq.tolist(), orr.tolist()))
    keys = hq.cpu().numpy() * n_refs + hr.cpu().numpy()
    assert np.all(np.diff(keys) > 0)
