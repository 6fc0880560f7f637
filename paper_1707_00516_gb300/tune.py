"""Autotuner for batched plans: picks the compare kernel's tile variant by
timing each candidate plan on the device, and caches the winner.

The cache is a JSON file keyed by the GPU name, the panels' loci counts and
reference counts, a power-of-two bucket of each panel's query count, and k.
It lives at $FASTID_TUNE_CACHE or ~/.cache/fastid_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding as B

CANDIDATES = (B.VARIANT_TENSOR_N256, B.VARIANT_TENSOR_N128, B.VARIANT_TENSOR_PAIR)


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
        parts = [f"{d.n_loci}x{d.n_refs}:{_bucket(per_panel.get(i, 0))}" for i, d in enumerate(dbs)]
        return f"{torch.cuda.get_device_name()}|k{k}|" + ",".join(parts)

    def choose(self, ctx: B.Context, dbs, batches, k: int, threshold: int = B.NO_THRESHOLD) -> int:
        """Variant for this workload: cached, else measured now."""
        key = self.key(dbs, batches, k)
        with self._lock:
            hit = self._cache.get(key)
        if hit is not None:
            return int(hit["variant"])
        timings = {}
        for v in self.candidates:
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
