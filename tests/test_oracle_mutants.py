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
