"""Randomized parity sweep: seeded random shapes (references, loci, queries,
k, threshold, mode mix, allele density) through top-k, hit list and full score
matrix, in the three compute forms, each equal to the oracle element by
element.  The configurations are drawn once from a fixed seed, so the sweep is
the same on every run."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402

FORMS = {"plain": B.FORM_PLAIN, "tensor": B.FORM_TENSOR, "packed": B.FORM_TENSOR_PACKED, "fp4": B.FORM_TENSOR_FP4,
         "fp4packed": B.FORM_TENSOR_FP4_PACKED}


def _configs(n=48, seed=20251203):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_refs = int(rng.integers(1, 4000))
        n_loci = int(rng.choice([int(rng.integers(1, 200)), int(rng.integers(200, 2500))]))
        n_q = int(rng.integers(1, max(2, min(600, 600_000 // max(n_refs, 1)))))
        k = int(rng.integers(1, 33))
        T = B.NO_THRESHOLD if rng.random() < 0.4 else int(rng.integers(0, n_loci + 1))
        p_ref = float(rng.uniform(0.02, 0.6))
        p_q = float(rng.uniform(0.02, 0.6))
        out.append((i, n_refs, n_loci, n_q, k, T, p_ref, p_q))
    return out


CONFIGS = _configs()


@pytest.fixture(scope="module")
def searchers():
    import __graft_entry__
    __graft_entry__.build()
    ss = {name: Searcher(0, form) for name, form in FORMS.items()}
    yield ss
    for s in ss.values():
        s.ctx.close()


@pytest.mark.parametrize("cfg", CONFIGS, ids=[f"cfg{c[0]}" for c in CONFIGS])
def test_random_config(searchers, cfg):
    i, n_refs, n_loci, n_q, k, T, p_ref, p_q = cfg
    rng = np.random.default_rng(1000 + i)
    R = (rng.random((n_refs, n_loci)) < p_ref).astype(np.uint8)
    Q = (rng.random((n_q, n_loci)) < p_q).astype(np.uint8)
    # a few queries are exact copies of references (score 0 in both modes)
    for j in range(min(3, n_q)):
        Q[j] = R[rng.integers(0, n_refs)]
    modes = (rng.random(n_q) < 0.5).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    exp = oracle.select(mis, une, modes)
    es, ei = oracle.topk(exp, k, T)
    hit_T = T if T != B.NO_THRESHOLD else int(np.percentile(exp, 2))
    oq, orr, osc = oracle.hits(exp, hit_T)
    for name, s in searchers.items():
        flags = {"tensor": B.REFS_TENSOR, "fp4": B.REFS_FP4}.get(name, 0)
        db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci, flags=flags)
        q = torch.empty((n_q, words64(n_loci)), dtype=torch.int64, device="cuda")
        B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
        m = torch.from_numpy(modes).cuda()
        sc, ix = s.topk(db, q, m, k, T)
        hq, hr, hs, hc = s.hits(db, q, m, hit_T, max(1, oq.size))
        full = s.scores(db, q, m, torch.int32)
        torch.cuda.synchronize()
        assert B.fastid_sync_status(s.ctx) == B.OK, name
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), es), name
        assert np.array_equal(ix.cpu().numpy(), ei), name
        n = int(hc.item())
        assert n == oq.size, name
        assert np.array_equal(hq[:n].cpu().numpy(), oq) and np.array_equal(hr[:n].cpu().numpy(), orr), name
        assert np.array_equal(hs[:n].cpu().numpy().view(np.uint32), osc), name
        assert np.array_equal(full.cpu().numpy().view(np.uint32), exp), name
        db.close()
