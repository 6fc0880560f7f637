"""Autotuner for batched plans: picks the compare kernel's variant -- operand
encoding (FP8 or block-scaled FP4 copy) and tile shape (128 x 256, 128 x 128,
2-CTA pairs sharing reference stages by multicast or as one 2-SM MMA; FP4
128 x 224 single or paired either way) -- by timing each candidate plan
the panels support on the device, and caches the winner.

The cache is a JSON file keyed by the GPU name, the panels' loci counts,
reference counts and operand copies, a power-of-two bucket of each panel's
query count, and k.
It lives at $FASTID_TUNE_CACHE or ~/.cache/fastid_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding as B

CANDIDATES = (B.VARIANT_TENSOR_N256, B.VARIANT_TENSOR_N128, B.VARIANT_TENSOR_PAIR, B.VARIANT_TENSOR_FP4,
              B.VARIANT_TENSOR_FP4_PAIR, B.VARIANT_TENSOR_PAIR_2SM, B.VARIANT_TENSOR_FP4_PAIR_2SM)
FP4_VARIANTS = (B.VARIANT_TENSOR_FP4, B.VARIANT_TENSOR_FP4_PAIR, B.VARIANT_TENSOR_FP4_PAIR_2SM)


def supported(variant: int, dbs) -> bool:
    """Whether every panel holds the operand copy the variant reads."""
    need = B.REFS_FP4 if variant in FP4_VARIANTS else B.REFS_TENSOR
    return all(d.flags & need for d in dbs)


def _bucket(n: int) -> int:
    return 0 if n <= 0 else 1 << math.ceil(math.log2(n))


class Autotuner:
    def __init__(self, cache_path: str | None = None, candidates=CANDIDATES, reps: int = 3):
        self.path = cache_path or os.environ.get("FASTID_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "fastid_gb300", "tune.json")
        self.candidates = tuple(candidates)
        self.reps = reps
        self._lock = threading.Lock()
        self._cache = self._load()
        self.last_timings: dict[int, float] = {}

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(self._cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except OSError:
            pass

    def key(self, dbs, batches, k: int) -> str:
        per_panel = {}
        for (panel, q, *_rest) in batches:
            per_panel[panel] = per_panel.get(panel, 0) + q.size(0)
        parts = [f"{d.n_loci}x{d.n_refs}f{d.flags}:{_bucket(per_panel.get(i, 0))}" for i, d in enumerate(dbs)]
        return f"{torch.cuda.get_device_name()}|k{k}|" + ",".join(parts)

    def choose(self, ctx: B.Context, dbs, batches, k: int, threshold: int = B.NO_THRESHOLD) -> int:
        """Variant for this workload: cached, else measured now."""
        key = self.key(dbs, batches, k)
        with self._lock:
            hit = self._cache.get(key)
        if hit is not None:
            return int(hit["variant"])
        timings = {}
        for v in [c for c in self.candidates if supported(c, dbs)]:
            plan = B.Plan(ctx, dbs, batches, k, threshold, v)
            try:
                plan.run()  # warm-up (module load, caches)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(self.reps):
                    plan.run()
                e1.record()
                torch.cuda.synchronize()
                timings[v] = e0.elapsed_time(e1) / self.reps
            finally:
                plan.close()
        best = min(timings, key=timings.get)
        self.last_timings = timings
        with self._lock:
            self._cache[key] = {"variant": best, "ms": {str(v): t for v, t in timings.items()}}
            self._save()
        return best


# ---------------------------------------------------------------------------
# Compute form of single comparison calls
# ---------------------------------------------------------------------------

# FASTID_FORM_* and the database copy each one needs (0: the packed rows).
FORM_NEEDS = {B.FORM_PLAIN: 0, B.FORM_TENSOR: B.REFS_TENSOR, B.FORM_TENSOR_PACKED: 0,
              B.FORM_TENSOR_FP4: B.REFS_FP4, B.FORM_TENSOR_FP4_PACKED: 0}


def forms_for(db) -> list[int]:
    """The forms a database supports: every form whose operand copy it holds."""
    return [f for f, need in FORM_NEEDS.items() if (db.flags & need) == need]


class FormTuner:
    """Chooses the compute form and reference operand of fastid_topk calls --
    plain AND + POPC, FP8 or FP4 tensor form over the database's copy or over
    its packed rows expanded on chip -- by timing each form the database
    supports on the caller's queries, and caches the fastest.  The cache (same
    file as Autotuner's) is keyed by the GPU name, N, a power-of-two bucket of
    the reference count, the database's copies, a bucket of the query count,
    k and whether a threshold applies.  FASTID_FORM_AUTO is the library's fixed
    rule from one such sweep; this is the same choice measured per workload."""

    def __init__(self, cache_path: str | None = None, forms=tuple(FORM_NEEDS), reps: int = 2):
        self._tuner = Autotuner(cache_path)
        self.forms = tuple(forms)
        self.reps = reps
        self.last_timings: dict[int, float] = {}

    @staticmethod
    def key(db, n_q: int, k: int, threshold: int) -> str:
        return (f"{torch.cuda.get_device_name()}|topk|N{db.n_loci}|R{_bucket(db.n_refs)}|f{db.flags}|"
                f"q{_bucket(n_q)}|k{k}|T{int(threshold != B.NO_THRESHOLD)}")

    def choose(self, ctx: B.Context, db, queries: torch.Tensor, modes: torch.Tensor, k: int,
               threshold: int = B.NO_THRESHOLD) -> int:
        """FASTID_FORM_* for these calls: cached, else measured now (a
        measurement leaves the context's form at FASTID_FORM_AUTO)."""
        t = self._tuner
        key = self.key(db, queries.size(0), k, threshold)
        with t._lock:
            hit = t._cache.get(key)
        if hit is not None:
            return int(hit["form"])
        n_q = queries.size(0)
        sc = torch.empty((n_q, k), dtype=torch.int32, device=queries.device)
        ix = torch.empty((n_q, k), dtype=torch.int64, device=queries.device)
        timings = {}
        for f in [f for f in self.forms if f in forms_for(db)]:
            B.fastid_set_form(ctx, f)
            B.fastid_topk(ctx, db, queries, modes, k, threshold, sc, ix)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(self.reps):
                B.fastid_topk(ctx, db, queries, modes, k, threshold, sc, ix)
            e1.record()
            torch.cuda.synchronize()
            timings[f] = e0.elapsed_time(e1) / self.reps
        B.fastid_set_form(ctx, B.FORM_AUTO)
        best = min(timings, key=timings.get)
        self.last_timings = timings
        with t._lock:
            t._cache[key] = {"form": best, "ms": {str(f): v for f, v in timings.items()}}
            t._save()
        return best
