"""Host logic of the autotuners (no GPU): which variants and forms a database
supports, the cache keys (query counts bucketed to powers of two), and that a
cached choice is returned without measuring, across tuner instances."""
import json
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300 import tune  # noqa: E402


def _db(n_loci, n_refs, flags):
    return SimpleNamespace(n_loci=n_loci, n_refs=n_refs, flags=flags)


def test_bucket_is_next_power_of_two():
    assert [tune._bucket(n) for n in (0, 1, 2, 3, 4, 5, 127, 128, 129, 2048)] == [0, 1, 2, 4, 4, 8, 128, 128, 256,
                                                                                    2048]


def test_variants_need_their_operand_copies():
    fp8, fp4, both = _db(512, 10, B.REFS_TENSOR), _db(512, 10, B.REFS_FP4), _db(512, 10, B.REFS_TENSOR | B.REFS_FP4)
    for v in tune.CANDIDATES:
        is_fp4 = v in tune.FP4_VARIANTS
        assert tune.supported(v, [both, both])
        assert tune.supported(v, [fp4]) == is_fp4
        assert tune.supported(v, [fp8]) == (not is_fp4)
        assert not tune.supported(v, [fp8, fp4])  # every panel must hold the copy


def test_forms_a_database_supports():
    assert set(tune.forms_for(_db(64, 1, 0))) == {B.FORM_PLAIN, B.FORM_TENSOR_PACKED, B.FORM_TENSOR_FP4_PACKED}
    assert B.FORM_TENSOR in tune.forms_for(_db(64, 1, B.REFS_TENSOR))
    assert B.FORM_TENSOR_FP4 not in tune.forms_for(_db(64, 1, B.REFS_TENSOR))
    assert set(tune.forms_for(_db(64, 1, B.REFS_TENSOR | B.REFS_FP4))) == set(tune.FORM_NEEDS)


def test_cached_choices_are_reused_without_measuring(tmp_path, monkeypatch):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FAKE GPU")
    path = str(tmp_path / "tune.json")
    dbs = [_db(512, 4_000_000, B.REFS_FP4), _db(2048, 4_000_000, B.REFS_FP4)]
    # batches: (panel, queries, ...); 100 + 30 queries on panel 0, 5 on panel 1
    batches = [(0, torch.zeros(100, 8)), (0, torch.zeros(30, 8)), (1, torch.zeros(5, 32))]
    at = tune.Autotuner(path)
    key = at.key(dbs, batches, 16)
    assert key == (f"FAKE GPU|k16|512x4000000f{B.REFS_FP4}:256,2048x4000000f{B.REFS_FP4}:8")
    db1 = _db(2048, 20_000_000, B.REFS_FP4)
    fkey = tune.FormTuner.key(db1, 100, 32, 512)
    assert fkey == f"FAKE GPU|topk|N2048|R33554432|f{B.REFS_FP4}|q128|k32|T1"
    assert tune.FormTuner.key(db1, 100, 32, B.NO_THRESHOLD).endswith("|T0")
    with open(path, "w") as f:
        json.dump({key: {"variant": B.VARIANT_TENSOR_FP4_PAIR_2SM, "ms": {}},
                   fkey: {"form": B.FORM_TENSOR_FP4_PACKED, "ms": {}}}, f)

    def no_measuring(*a, **kw):
        raise AssertionError("a cached choice was measured again")

    monkeypatch.setattr(B, "Plan", no_measuring)
    monkeypatch.setattr(B, "fastid_topk", no_measuring)
    # fresh instances read the file
    assert tune.Autotuner(path).choose(None, dbs, batches, 16) == B.VARIANT_TENSOR_FP4_PAIR_2SM
    q = torch.zeros(100, 32)
    assert tune.FormTuner(path).choose(None, db1, q, torch.zeros(100), 32, 512) == B.FORM_TENSOR_FP4_PACKED
