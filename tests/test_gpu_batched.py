"""Batched persistent plans: many uneven query batches over several loci
panels in one launch, run directly and as a replayed CUDA graph; every batch's
top-k equals the oracle's for that batch against its panel."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402

PANELS = [(2000, 300), (5000, 1031), (3000, 2048)]  # (n_refs, n_loci)


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    s = Searcher(0, B.FORM_TENSOR)
    panels = []
    for i, (n_refs, n_loci) in enumerate(PANELS):
        seed = 900 + i
        thr = gen.maf_thresholds(seed, n_loci)
        R = gen.allele_rows(seed, gen.STREAM_DB, np.arange(n_refs), thr)
        db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci, flags=B.REFS_TENSOR | B.REFS_FP4)
        panels.append((R, db, thr, seed))
    yield s, panels
    for _, db, _, _ in panels:
        db.close()
    s.ctx.close()


def _make_batches(s, panels, sizes, k, salt, panel_ids=None):
    rng = np.random.default_rng(salt)
    out = []
    for b, n in enumerate(sizes):
        p = int(rng.integers(0, len(panels))) if panel_ids is None else panel_ids[b]
        R, db, thr, seed = panels[p]
        n_refs, n_loci = R.shape
        if n:
            rec = gen.recipe_mixtures(n, n_refs, n_loci, seed, 1, 4, fresh_base=(salt << 20) + b * 1000,
                                      salt=salt * 1000 + b)
            rec.modes[:] = rng.integers(0, 2, n).astype(np.uint8)
            Q = oracle.mix(gen.source_alleles(rec, thr), rec.offsets)
            modes = rec.modes
        else:
            Q = np.zeros((0, n_loci), np.uint8)
            modes = np.zeros(0, np.uint8)
        q = torch.zeros((max(n, 1), words64(n_loci)), dtype=torch.int64, device="cuda")[:n] if n else \
            torch.zeros((0, words64(n_loci)), dtype=torch.int64, device="cuda")
        if n:
            B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
        m = torch.from_numpy(modes).cuda() if n else torch.zeros(0, dtype=torch.uint8, device="cuda")
        sc = torch.full((n, k), 7, dtype=torch.int32, device="cuda")
        ix = torch.full((n, k), 7, dtype=torch.int64, device="cuda")
        out.append([p, q, m, sc, ix, Q, modes])
    return out


def _check(panels, batches, k, T):
    for p, q, m, sc, ix, Q, modes in batches:
        if Q.shape[0] == 0:
            continue
        R = panels[p][0]
        mis, une = oracle.scores(R, Q)
        es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), es)
        assert np.array_equal(ix.cpu().numpy(), ei)


@pytest.mark.parametrize("variant", [B.VARIANT_TENSOR_N256, B.VARIANT_TENSOR_N128, B.VARIANT_TENSOR_PAIR,
                                     B.VARIANT_TENSOR_FP4, B.VARIANT_TENSOR_FP4_PAIR, B.VARIANT_TENSOR_PAIR_2SM,
                                     B.VARIANT_TENSOR_FP4_PAIR_2SM])
@pytest.mark.parametrize("k,T", [(16, B.NO_THRESHOLD), (32, 40), (17, B.NO_THRESHOLD), (3, 25)])
def test_plan_run_matches_oracle(setup, variant, k, T):
    s, panels = setup
    sizes = [1, 0, 7, 130, 300, 2, 129, 57, 256]
    batches = _make_batches(s, panels, sizes, k, salt=11 + variant)
    plan = B.Plan(s.ctx, [p[1] for p in panels], [b[:5] for b in batches], k, T, variant)
    info = plan.info()
    assert info["n_queries"] == sum(sizes) and info["variant"] == variant
    plan.run()
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    _check(panels, batches, k, T)
    plan.close()


def test_plan_graph_replay_with_new_contents(setup):
    s, panels = setup
    k = 16
    sizes = [33, 200, 1, 90]
    batches = _make_batches(s, panels, sizes, k, salt=5)
    plan = B.Plan(s.ctx, [p[1] for p in panels], [b[:5] for b in batches], k)
    assert plan.info()["variant"] == B.VARIANT_TENSOR_FP4_PAIR  # AUTO: every panel has its FP4 copy
    plan.capture()
    plan.replay()
    torch.cuda.synchronize()
    _check(panels, batches, k, B.NO_THRESHOLD)
    # new query contents in the same buffers, then replay the same graph
    fresh = _make_batches(s, panels, sizes, k, salt=6, panel_ids=[b[0] for b in batches])
    for old, new in zip(batches, fresh):
        old[1].copy_(new[1])
        old[2].copy_(new[2])
        old[5], old[6] = new[5], new[6]
    plan.replay()
    torch.cuda.synchronize()
    assert B.fastid_sync_status(s.ctx) == B.OK
    _check(panels, batches, k, B.NO_THRESHOLD)
    plan.close()


def test_plan_needs_tensor_copy(setup):
    s, panels = setup
    R = panels[0][0]
    db_plain = s.load_refs_alleles(torch.from_numpy(R).cuda(), R.shape[1], flags=0)
    with pytest.raises(B.FastIDError) as e:
        B.Plan(s.ctx, [db_plain], [], 8)
    assert e.value.status == B.EUNSUPPORTED
    db_plain.close()
    db_fp8 = s.load_refs_alleles(torch.from_numpy(R).cuda(), R.shape[1], flags=B.REFS_TENSOR)
    for v in (B.VARIANT_TENSOR_FP4, B.VARIANT_TENSOR_FP4_PAIR):
        with pytest.raises(B.FastIDError) as e:
            B.Plan(s.ctx, [db_fp8], [], 8, variant=v)
        assert e.value.status == B.EUNSUPPORTED
    assert B.Plan(s.ctx, [db_fp8], [], 8).info()["variant"] == B.VARIANT_TENSOR_N256
    db_fp8.close()


def test_form_tuner_choice_is_exact(setup, tmp_path):
    """FormTuner times every form the database supports for these calls,
    caches the fastest, and the chosen form's results equal the oracle."""
    from paper_1707_00516_gb300.tune import FormTuner, forms_for
    s, panels = setup
    R, db, thr, seed = panels[2]
    k, T = 16, B.NO_THRESHOLD
    batches = _make_batches(s, panels, [300], k, salt=21, panel_ids=[2])
    _, q, m, sc, ix, Q, modes = batches[0]
    tuner = FormTuner(cache_path=str(tmp_path / "tune.json"))
    f = s.tune_form(db, q, m, k, T, tuner=tuner)
    assert set(tuner.last_timings) == set(forms_for(db)) and f == min(tuner.last_timings,
                                                                          key=tuner.last_timings.get)
    again = FormTuner(cache_path=str(tmp_path / "tune.json"))
    assert again.choose(s.ctx, db, q, m, k, T) == f and again.last_timings == {}  # from the cache
    got_s, got_i = s.topk(db, q, m, k, T)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), k, T)
    assert np.array_equal(got_s.cpu().numpy().view(np.uint32), es) and np.array_equal(got_i.cpu().numpy(), ei)
    B.fastid_set_form(s.ctx, B.FORM_TENSOR)
