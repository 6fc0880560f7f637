"""GPU parity: every kernel result through the C ABI equals the CPU oracle's,
element by element (integers: zero tolerance), for both compute forms."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402


FORMS = {"plain": B.FORM_PLAIN, "tensor": B.FORM_TENSOR, "packed": B.FORM_TENSOR_PACKED, "fp4": B.FORM_TENSOR_FP4,
         "fp4packed": B.FORM_TENSOR_FP4_PACKED}


@pytest.fixture(scope="module", params=sorted(FORMS))
def searcher(request):
    """One searcher per compute form; databases are loaded with the flags
    the form needs (the e4m3 or e2m1 operand copy of the tensor forms; none
    for the plain form and for the tensor forms over packed rows)."""
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, FORMS[request.param])
    yield s
    s.ctx.close()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def make_case(n_refs, n_loci, n_ind, n_mix, seed, planted=None, low_entropy=False):
    if low_entropy:
        rng = np.random.default_rng(seed)
        R = (rng.random((n_refs, n_loci)) < 0.5).astype(np.uint8)
        Q = (rng.random((n_ind + n_mix, n_loci)) < 0.5).astype(np.uint8)
        modes = np.array([0] * n_ind + [1] * n_mix, np.uint8)
        return R, Q, modes, None, None
    thr = gen.maf_thresholds(seed, n_loci)
    R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
    parts = []
    if n_ind:
        parts.append(gen.recipe_individuals(n_ind, n_refs, n_loci, seed,
                                            n_planted=min(n_ind, n_refs) // 2 if planted is None else planted))
    if n_mix:
        parts.append(gen.recipe_mixtures(n_mix, n_refs, n_loci, seed, 2, 5))
    rec = parts[0] if len(parts) == 1 else gen.concat_recipes(*parts)
    src = gen.source_alleles(rec, thr)
    Q = oracle.mix(src, rec.offsets)
    return R, Q, rec.modes, src, rec


def load(s, R, n_loci):
    return s.load_refs_alleles(torch.from_numpy(np.ascontiguousarray(R)).cuda(), n_loci)


def pack_dev(s, A, n_loci):
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    out = torch.empty((A.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, a, n_loci, out)
    return out


# ---- pack / mix ----------------------------------------------------------------

@pytest.mark.parametrize("n_loci", [1, 7, 63, 64, 65, 333, 1024, 2048, 4097])
def test_pack_parity(searcher, n_loci):
    rng = np.random.default_rng(n_loci)
    A = (rng.random((257, n_loci)) < 0.37).astype(np.uint8)
    A[rng.random(A.shape) < 0.05] *= 7  # any nonzero byte is an allele
    ld = words64(n_loci) + 3
    a = torch.from_numpy(A).cuda()
    out = torch.full((257, ld), -1, dtype=torch.int64, device="cuda")
    norms = torch.empty(257, dtype=torch.int32, device="cuda")
    B.fastid_pack(searcher.ctx, a, n_loci, out, norms)
    exp = oracle.pack(A, ld_words=ld)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), exp)
    _, une = oracle.scores(A, np.zeros((1, n_loci), np.uint8))
    assert np.array_equal(u32(norms), une[0])


def test_pack_strided_rows(searcher):
    rng = np.random.default_rng(5)
    big = (rng.random((50, 300)) < 0.5).astype(np.uint8)
    a = torch.from_numpy(big).cuda()[:, 10:210]  # row stride 300, 200 loci, unaligned start
    out = torch.empty((50, 4), dtype=torch.int64, device="cuda")
    B.fastid_pack(searcher.ctx, a, 200, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), oracle.pack(big[:, 10:210], ld_words=4))


def test_mix_parity(searcher):
    n_loci = 777
    thr = gen.maf_thresholds(3, n_loci)
    rec = gen.recipe_mixtures(60, 500, n_loci, 3, 1, 5)
    src = gen.source_alleles(rec, thr)
    q = searcher.build_queries(torch.from_numpy(src).cuda(), torch.from_numpy(rec.offsets).cuda(), n_loci)
    exp = oracle.pack(oracle.mix(src, rec.offsets))
    assert np.array_equal(q.cpu().numpy().view(np.uint64), exp)


# ---- full score matrix -----------------------------------------------------------

def test_scores_c1_full_config(searcher):
    """64 individuals (8 database copies) x 10,000 refs, N = 1024: both full
    uint16 matrices."""
    rec = gen.recipe_c1()
    n_loci, n_refs = rec.n_loci, rec.n_refs
    thr = gen.maf_thresholds(rec.seed, n_loci)
    R = gen.allele_rows(rec.seed, gen.STREAM_DB, np.arange(n_refs), thr)
    src = gen.source_alleles(rec, thr)
    Q = oracle.mix(src, rec.offsets)
    db = load(searcher, R, n_loci)
    q = pack_dev(searcher, Q, n_loci)
    mis, une = oracle.scores(R, Q)
    for mode, exp in ((0, mis), (1, une)):
        modes = torch.full((64,), mode, dtype=torch.uint8, device="cuda")
        out16 = searcher.scores(db, q, modes, torch.int16)
        out32 = searcher.scores(db, q, modes, torch.int32)
        assert np.array_equal(out16.cpu().numpy().view(np.uint16), exp.astype(np.uint16))
        assert np.array_equal(u32(out32), exp)
    for j in range(64):
        for r in rec.planted(j):
            assert mis[j, r] == 0
    db.close()


@pytest.mark.parametrize("n_refs,n_loci,n_q", [(1, 1, 1), (129, 64, 3), (1000, 333, 257), (300, 4096, 130)])
def test_scores_ragged(searcher, n_refs, n_loci, n_q):
    R, Q, modes, _, _ = make_case(n_refs, n_loci, n_q // 2, n_q - n_q // 2, 77 + n_refs, low_entropy=True)
    db = load(searcher, R, n_loci)
    q = pack_dev(searcher, Q, n_loci)
    out = searcher.scores(db, q, torch.from_numpy(modes).cuda(), torch.int32)
    mis, une = oracle.scores(R, Q)
    assert np.array_equal(u32(out), oracle.select(mis, une, modes))
    db.close()


# ---- top-k -------------------------------------------------------------------------

TOPK_CASES = [
    # n_refs, n_loci, n_ind, n_mix, k, threshold, low_entropy
    (1, 64, 1, 1, 1, B.NO_THRESHOLD, False),
    (20, 64, 3, 3, 32, B.NO_THRESHOLD, False),        # k > n_refs
    (3000, 333, 100, 200, 16, B.NO_THRESHOLD, False),  # 3 query tiles, ragged
    (5000, 1031, 60, 70, 32, 400, False),
    (4000, 8, 40, 40, 32, B.NO_THRESHOLD, True),       # N = 8: massive ties
    (6000, 12, 10, 10, 7, 3, True),                    # ties + threshold
    (20000, 256, 64, 64, 32, B.NO_THRESHOLD, False),   # several CTAs per query tile
]


@pytest.mark.parametrize("case", TOPK_CASES)
def test_topk_parity(searcher, case):
    n_refs, n_loci, n_ind, n_mix, k, T, le = case
    R, Q, modes, _, _ = make_case(n_refs, n_loci, n_ind, n_mix, 1000 + n_refs, low_entropy=le)
    db = load(searcher, R, n_loci)
    q = pack_dev(searcher, Q, n_loci)
    sc, ix = searcher.topk(db, q, torch.from_numpy(modes).cuda(), k, T)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
    assert np.array_equal(u32(sc), es)
    assert np.array_equal(ix.cpu().numpy(), ei)
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    db.close()


def test_topk_planted_recovery(searcher):
    R, Q, modes, src, rec = make_case(8000, 2048, 32, 32, 31)
    db = load(searcher, R, 2048)
    q = pack_dev(searcher, Q, 2048)
    sc, ix = searcher.topk(db, q, torch.from_numpy(modes).cuda(), 32, 512)
    sc, ix = u32(sc), ix.cpu().numpy()
    for j in range(rec.n_queries):
        for r in rec.planted(j):
            pos = np.nonzero(ix[j] == r)[0]
            assert pos.size == 1 and sc[j, pos[0]] == 0
    db.close()


# ---- hit list ------------------------------------------------------------------------

@pytest.mark.parametrize("T", [0, 2, 5])
def test_hits_parity(searcher, T):
    R, Q, modes, _, _ = make_case(3000, 10, 50, 50, 5 + T, low_entropy=True)
    db = load(searcher, R, 10)
    q = pack_dev(searcher, Q, 10)
    hq, hr, hs, hc = searcher.hits(db, q, torch.from_numpy(modes).cuda(), T, 1 << 18)
    mis, une = oracle.scores(R, Q)
    oq, orr, osc = oracle.hits(oracle.select(mis, une, modes), T)
    n = int(hc.item())
    assert n == oq.size
    assert np.array_equal(hq[:n].cpu().numpy(), oq)
    assert np.array_equal(hr[:n].cpu().numpy(), orr)
    assert np.array_equal(u32(hs[:n]), osc)
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    db.close()


def test_hits_overflow(searcher):
    R, Q, modes, _, _ = make_case(2000, 6, 20, 20, 9, low_entropy=True)
    db = load(searcher, R, 6)
    q = pack_dev(searcher, Q, 6)
    cap = 100
    hq, hr, hs, hc = searcher.hits(db, q, torch.from_numpy(modes).cuda(), 2, cap)
    mis, une = oracle.scores(R, Q)
    sel = oracle.select(mis, une, modes)
    oq, orr, osc = oracle.hits(sel, 2)
    assert oq.size > cap
    assert int(hc.item()) == oq.size
    assert B.fastid_sync_status(searcher.ctx) == B.EOVERFLOW
    # what was kept are valid hits, sorted by (q, r)
    hq, hr, hs = hq.cpu().numpy(), hr.cpu().numpy(), u32(hs)
    assert np.all(sel[hq, hr] == hs) and np.all(hs <= 2)
    keys = hq * (1 << 32) + hr
    assert np.all(np.diff(keys) > 0)
    db.close()


def test_hits_count_only(searcher):
    R, Q, modes, _, _ = make_case(500, 6, 5, 5, 19, low_entropy=True)
    db = load(searcher, R, 6)
    q = pack_dev(searcher, Q, 6)
    hc = torch.zeros(1, dtype=torch.int64, device="cuda")
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    B.fastid_compare(searcher.ctx, db, q, torch.from_numpy(modes).cuda(), 1, e, e,
                     torch.empty(0, dtype=torch.int32, device="cuda"), hc)
    mis, une = oracle.scores(R, Q)
    assert int(hc.item()) == int((oracle.select(mis, une, modes) <= 1).sum())
    st = B.fastid_sync_status(searcher.ctx)
    assert st in (B.OK, B.EOVERFLOW)
    db.close()


# ---- edge cases and argument errors ----------------------------------------------------

def test_zero_queries(searcher):
    R = np.ones((10, 64), np.uint8)
    db = load(searcher, R, 64)
    q = torch.empty((0, 1), dtype=torch.int64, device="cuda")
    m = torch.empty(0, dtype=torch.uint8, device="cuda")
    sc = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    ix = torch.empty((0, 4), dtype=torch.int64, device="cuda")
    B.fastid_topk(searcher.ctx, db, q, m, 4, B.NO_THRESHOLD, sc, ix)
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    db.close()


def test_all_ones_and_zeros(searcher):
    n_loci = 4096
    R = np.zeros((300, n_loci), np.uint8)
    R[::2] = 1
    Q = np.stack([np.ones(n_loci, np.uint8), np.zeros(n_loci, np.uint8)] * 3)
    modes = np.array([0, 0, 1, 1, 0, 1], np.uint8)
    db = load(searcher, R, n_loci)
    q = pack_dev(searcher, Q, n_loci)
    out = searcher.scores(db, q, torch.from_numpy(modes).cuda(), torch.int32)
    mis, une = oracle.scores(R, Q)
    assert np.array_equal(u32(out), oracle.select(mis, une, modes))
    db.close()


def test_invalid_arguments(searcher):
    R = np.ones((10, 64), np.uint8)
    db = load(searcher, R, 64)
    q = pack_dev(searcher, R[:2], 64)
    m = torch.zeros(2, dtype=torch.uint8, device="cuda")
    for k in (0, B.MAX_K + 1):
        sc = torch.empty((2, max(k, 1)), dtype=torch.int32, device="cuda")
        ix = torch.empty((2, max(k, 1)), dtype=torch.int64, device="cuda")
        with pytest.raises((B.FastIDError, ValueError)):
            B.fastid_topk(searcher.ctx, db, q, m, k, 0, sc, ix)
    with pytest.raises(B.FastIDError) as e:
        B.fastid_load_refs(searcher.ctx, q, 0)
    assert e.value.status == B.EINVAL
    db.close()


# ---- host in, host out -----------------------------------------------------------

def test_search_host_inputs(searcher):
    """Searcher.search_host from numpy arrays (staged), from pinned CPU tensors
    (copied directly) and from unpinned CPU tensors: the same lists, equal to
    the oracle's; a tensor of the wrong dtype is refused."""
    n_refs, n_loci, k, T = 2500, 555, 10, 300
    R, Q, modes, src, rec = make_case(n_refs, n_loci, 40, 60, seed=77)
    db = load(searcher, R, n_loci)
    off = rec.offsets.astype(np.int32)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
    inputs = {
        "numpy": (src, off, modes),
        "pinned": tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (src, off, modes)),
        "unpinned": tuple(torch.from_numpy(np.ascontiguousarray(a)) for a in (src, off, modes)),
    }
    for name, (a, o, m) in inputs.items():
        sc, ix, h2d, d2h = searcher.search_host(db, a, o, m, k, T)
        assert np.array_equal(sc, es) and np.array_equal(ix, ei), name
        assert h2d == src.nbytes + off.nbytes + modes.nbytes and d2h == 12 * k * Q.shape[0], name
    with pytest.raises(ValueError):
        searcher.search_host(db, torch.from_numpy(src.astype(np.int32)), off, modes, k, T)
    assert B.fastid_sync_status(searcher.ctx) == B.OK
    db.close()
