"""Order invariance of the tensor calls, which spread their input queries over
the operand's tiles: the same queries in another order give the same per-query
results (top-k, hit list, full matrix), equal to the oracle's, in every tensor
form, with the queries grouped by kind (every mismatch-count query before every
Eq. 1 query) and shuffled."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402

FORMS = {"fp8": B.FORM_TENSOR, "fp8packed": B.FORM_TENSOR_PACKED, "fp4": B.FORM_TENSOR_FP4,
         "fp4packed": B.FORM_TENSOR_FP4_PACKED}


@pytest.fixture(scope="module")
def case():
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(1707)
    n_refs, n_loci, n_q = 4000, 600, 390  # 390 queries: 4 tiles, the last one ragged
    R = (rng.random((n_refs, n_loci)) < 0.3).astype(np.uint8)
    Q = (rng.random((n_q, n_loci)) < 0.45).astype(np.uint8)
    Q[:30] = R[rng.integers(0, n_refs, 30)]
    modes = np.zeros(n_q, np.uint8)
    modes[n_q // 2:] = 1  # grouped by kind, as a caller may pass them
    mis, une = oracle.scores(R, Q)
    return R, Q, modes, oracle.select(mis, une, modes), n_loci, rng.permutation(n_q)


def run(s, db, Q, modes, n_loci, k, T):
    q = torch.empty((Q.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), n_loci, q)
    m = torch.from_numpy(np.ascontiguousarray(modes)).cuda()
    sc, ix = s.topk(db, q, m, k, T)
    hq, hr, hs, hc = s.hits(db, q, m, 70, 200_000)
    full = s.scores(db, q, m)
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    n = int(hc.item())
    # scores as uint32, the library's type (empty top-k slots hold 2^32 - 1)
    return (sc.cpu().numpy().view(np.uint32), ix.cpu().numpy(),
            (hq[:n].cpu().numpy(), hr[:n].cpu().numpy(), hs[:n].cpu().numpy().view(np.uint32)),
            full.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("form", sorted(FORMS))
def test_results_do_not_depend_on_query_order(case, form):
    R, Q, modes, exp, n_loci, perm = case
    s = Searcher(0, FORMS[form])
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci, flags=B.REFS_TENSOR | B.REFS_FP4)
    k, T = 16, 200
    a_s, a_i, a_h, a_f = run(s, db, Q, modes, n_loci, k, T)
    b_s, b_i, b_h, b_f = run(s, db, Q[perm], modes[perm], n_loci, k, T)
    es, ei = oracle.topk(exp, k, T)
    assert np.array_equal(a_s, es) and np.array_equal(a_i, ei)
    assert np.array_equal(b_s, es[perm]) and np.array_equal(b_i, ei[perm])
    assert np.array_equal(a_f, exp) and np.array_equal(b_f, exp[perm])
    hq, hr, hsc = oracle.hits(exp, 70)
    assert 0 < hq.size < 200_000
    assert np.array_equal(a_h[0], hq) and np.array_equal(a_h[1], hr) and np.array_equal(a_h[2], hsc)
    # the permuted call's hits, mapped back to input order and re-sorted, are the same set
    bq = perm[b_h[0]]
    order = np.lexsort((b_h[1], bq))
    assert np.array_equal(bq[order], hq) and np.array_equal(b_h[1][order], hr) and np.array_equal(b_h[2][order], hsc)
