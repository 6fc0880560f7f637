"""Plausible mistakes planted in a copy of the C oracle must each be caught
by the pins (compiled on the CPU into a temporary directory; the real
oracle is untouched)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

MUTANTS = {
    "and_with_query": ("uint8_t y = (uint8_t)(x & a);", "uint8_t y = (uint8_t)(x & b);"),
    "xor_count_uses_and": ("m += x;", "m += y;"),
    "msb_first_packing": ("row[l / 64] |= (uint64_t)1 << (l % 64);",
                          "row[l / 64] |= (uint64_t)1 << (63 - l % 64);"),
    "dropped_last_locus": ("for (int32_t l = 0; l < n_loci; ++l) {\n        uint8_t a",
                           "for (int32_t l = 0; l + 1 < n_loci; ++l) {\n        uint8_t a"),
    "mix_intersection": ("v = (uint8_t)(v | (src", "v = (uint8_t)(v & (src"),
    "transposed_output": ("if (mis) mis[q * n_r + r] = m;", "if (mis) mis[r * n_q + q] = m;"),
}


def _pins_pass(golden_dir):
    """A compact run of the pins; False as soon as one fails."""
    import test_oracle_pins as P
    checks = [
        lambda: P.test_worked_example_packing(golden_dir),
        lambda: P.test_eq1_hand_worked(golden_dir),
        lambda: P.test_closed_forms_over_all_profiles(3),
        lambda: P.test_pack_matches_numpy_packbits(65),
        lambda: P.test_mix_is_union(),
        lambda: P.test_against_torch_int64_matmul(),
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, golden_dir, monkeypatch):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", str(path), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    real = oracle._load()
    for fname in ("oracle_pack", "oracle_mix", "oracle_scores", "oracle_score_pairs"):
        f = getattr(lib, fname)
        f.argtypes = getattr(real, fname).argtypes
        f.restype = None
    monkeypatch.setattr(oracle, "_lib", lib)
    assert not _pins_pass(golden_dir), f"mutant {name} survived the pins"


def test_unmutated_passes(golden_dir):
    assert _pins_pass(golden_dir)


# The oracle's Python steps (mode selection, top-k, hit list), mutated in a
# copy of the module's source; the pins of those steps must catch each one.
PY_MUTANTS = {
    "threshold_exclusive": ("keep = np.nonzero(s[q] <= threshold)[0]", "keep = np.nonzero(s[q] < threshold)[0]"),
    "ties_by_descending_ref": ("order = keep[np.lexsort((ids[keep], s[q, keep]))][:k]",
                               "order = keep[np.lexsort((-ids[keep], s[q, keep]))][:k]"),
    "modes_swapped": ("return np.where(m, une, mis).astype(np.uint32)",
                      "return np.where(m, mis, une).astype(np.uint32)"),
    "hits_by_ref_first": ("order = np.lexsort((rid, qid))", "order = np.lexsort((qid, rid))"),
}


def _py_pins_pass():
    import test_oracle_pins as P
    checks = [P.test_topk_ties_and_threshold, P.test_topk_against_python_sorted, P.test_hits_against_python,
              P.test_planted_recovery]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_is_caught(name, monkeypatch):
    import types
    src = open(oracle.__file__).read()
    old, new = PY_MUTANTS[name]
    assert src.count(old) == 1, name
    mut = types.ModuleType("oracle_mutant")
    mut.__file__ = oracle.__file__  # the C library resolves next to the real module
    exec(compile(src.replace(old, new), oracle.__file__, "exec"), mut.__dict__)
    for fname in ("select", "topk", "hits"):
        monkeypatch.setattr(oracle, fname, getattr(mut, fname))
    assert not _py_pins_pass(), f"mutant {name} survived the pins"


def test_python_unmutated_passes():
    assert _py_pins_pass()
