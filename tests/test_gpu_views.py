"""Row-range views of a database and the fold of per-part top-k lists
(fastid_topk_fold, and fastid_topk_accumulate which fuses the two): the
parts of one pass, compared in any order and folded, give exactly the
oracle's top-k over the whole database, in every compute form."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402

FORMS = {"plain": B.FORM_PLAIN, "fp8": B.FORM_TENSOR, "fp8packed": B.FORM_TENSOR_PACKED, "fp4": B.FORM_TENSOR_FP4,
         "fp4packed": B.FORM_TENSOR_FP4_PACKED}


@pytest.fixture(scope="module")
def case():
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(515)
    n_refs, n_loci, n_q = 10_000, 700, 300
    R = (rng.random((n_refs, n_loci)) < 0.3).astype(np.uint8)
    Q = (rng.random((n_q, n_loci)) < 0.3).astype(np.uint8)
    Q[:20] = R[rng.integers(0, n_refs, 20)]
    # equal scores across part boundaries: the order of ties must not depend on the part order
    R[3071] = R[3072] = R[9999] = Q[25]
    modes = (rng.random(n_q) < 0.5).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    return R, Q, modes, oracle.select(mis, une, modes), n_loci


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("k,T", [(1, B.NO_THRESHOLD), (16, 250), (32, B.NO_THRESHOLD)])
def test_views_folded_equal_whole(case, form, k, T):
    R, Q, modes, exp, n_loci = case
    s = Searcher(0, FORMS[form])
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci, flags=B.REFS_TENSOR | B.REFS_FP4)
    q = torch.empty((Q.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
    m = torch.from_numpy(modes).cuda()
    bounds = [(0, 3072), (3072, 4096), (7168, 2832)]
    views = [B.fastid_refs_view(s.ctx, db, r0, n) for r0, n in bounds]
    n_q = Q.shape[0]
    run_s = torch.full((n_q, k), -1, dtype=torch.int32, device="cuda")
    run_i = torch.full((n_q, k), -1, dtype=torch.int64, device="cuda")
    acc_s = run_s.clone()
    acc_i = run_i.clone()
    for p in (2, 0, 1):
        sc, ix = s.topk(views[p], q, m, k, T)
        B.fastid_topk_fold(s.ctx, run_s, run_i, sc, ix, bounds[p][0])
    for p in (1, 2, 0):  # the fused form, another order
        B.fastid_topk_accumulate(s.ctx, views[p], bounds[p][0], q, m, k, T, acc_s, acc_i)
    whole_s, whole_i = s.topk(db, q, m, k, T)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    es, ei = oracle.topk(exp, k, T)
    assert np.array_equal(run_s.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(run_i.cpu().numpy(), ei)
    assert np.array_equal(acc_s.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(acc_i.cpu().numpy(), ei)
    assert np.array_equal(whole_s.cpu().numpy().view(np.uint32), es)
    assert np.array_equal(whole_i.cpu().numpy(), ei)
    # a view's own hit list and full matrix, indices relative to the view
    full = s.scores(views[1], q, m, torch.int32)
    assert np.array_equal(full.cpu().numpy().view(np.uint32), exp[:, 3072:7168])
    for v in views:
        v.close()
    db.close()
    s.ctx.close()


def test_view_arguments(case):
    R, Q, modes, exp, n_loci = case
    s = Searcher(0, B.FORM_AUTO)
    db = s.load_refs_alleles(torch.from_numpy(R[:1000]).cuda(), n_loci, flags=0)
    for r0, n in [(100, 10), (0, 1001), (768, 300), (-256, 10), (0, 0)]:
        with pytest.raises(B.FastIDError) as e:
            B.fastid_refs_view(s.ctx, db, r0, n)
        assert e.value.status == B.EINVAL
    v = B.fastid_refs_view(s.ctx, db, 768, 232)
    assert v.info() == {"n_refs": 232, "n_loci": n_loci, "flags": 0, "device_bytes": 0}
    v.close()
    db.close()
    s.ctx.close()
