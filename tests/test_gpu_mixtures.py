"""Mixture-to-mixture comparison through the C ABI: a database of known
mixtures searched with unknown mixtures.  The score is Eq. 1 with the known
mixture in the reference role (oracle.mixture_vs_mixture), so it runs on the
same kernels; every form must equal the oracle, and an unknown mixture that
carries every contributor of a known one must find it at score 0."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402

FORMS = {"plain": B.FORM_PLAIN, "fp8": B.FORM_TENSOR, "fp4": B.FORM_TENSOR_FP4,
         "fp4packed": B.FORM_TENSOR_FP4_PACKED}


@pytest.fixture(scope="module")
def case():
    import __graft_entry__
    __graft_entry__.build()
    seed, n_loci, n_pool, n_known, n_unknown = 4711, 1500, 800, 5000, 150
    thr = gen.maf_thresholds(seed, n_loci)
    pool = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_pool), thr)
    rng = np.random.default_rng(seed)
    known_sets = [rng.choice(n_pool, int(rng.integers(2, 4)), replace=False) for _ in range(n_known)]
    K = np.stack([np.bitwise_or.reduce(pool[s], axis=0) for s in known_sets])
    unknown_sets, planted = [], []
    for u in range(n_unknown):
        if u % 3 == 0:  # a superset of a known mixture's contributors
            kk = int(rng.integers(0, n_known))
            extra = rng.choice(n_pool, int(rng.integers(1, 3)), replace=False)
            unknown_sets.append(np.union1d(known_sets[kk], extra))
            planted.append(kk)
        else:
            unknown_sets.append(rng.choice(n_pool, int(rng.integers(2, 5)), replace=False))
            planted.append(-1)
    U = np.stack([np.bitwise_or.reduce(pool[s], axis=0) for s in unknown_sets])
    cont, mis = oracle.mixture_vs_mixture(K, U)
    return K, U, cont, mis, planted, n_loci


@pytest.mark.parametrize("form", sorted(FORMS))
def test_mixture_database_matches_oracle(case, form):
    K, U, cont, mis, planted, n_loci = case
    s = Searcher(0, FORMS[form])
    db = s.load_refs_alleles(torch.from_numpy(K).cuda(), n_loci, flags=B.REFS_TENSOR | B.REFS_FP4)
    q = torch.empty((U.shape[0], words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(U).cuda(), n_loci, q)
    for mode, exp in ((gen.MODE_UNEXPLAINED, cont), (gen.MODE_MISMATCH, mis)):
        m = torch.full((U.shape[0],), mode, dtype=torch.uint8, device="cuda")
        sc, ix = s.topk(db, q, m, 16)
        torch.cuda.synchronize()
        assert B.fastid_sync_status(s.ctx) == B.OK
        es, ei = oracle.topk(exp, 16)
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
        assert np.array_equal(ix.cpu().numpy(), ei)
        if mode == gen.MODE_UNEXPLAINED:
            got = ix.cpu().numpy()
            for u, kk in enumerate(planted):
                if kk >= 0:
                    assert cont[u, kk] == 0 and kk in got[u]
    hq, hr, hs, hc = s.hits(db, q, torch.full((U.shape[0],), gen.MODE_UNEXPLAINED, dtype=torch.uint8,
                                               device="cuda"), 0, 1 << 16)
    oq, orr, _ = oracle.hits(cont, 0)
    n = int(hc.item())
    assert n == oq.size and np.array_equal(hq[:n].cpu().numpy(), oq) and np.array_equal(hr[:n].cpu().numpy(), orr)
    db.close()
    s.ctx.close()
