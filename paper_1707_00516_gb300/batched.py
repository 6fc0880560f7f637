"""Batched search over several loci panels with one persistent launch per run
(fastid_plan_*), captured once into a CUDA graph and replayed.

A BatchedSearch owns the device buffers of every batch (packed queries,
modes, results), so a run needs no allocation.  `run_host` is the host-buffer
path: it copies each batch's packed queries and modes in through pinned
memory, replays the graph and copies the results out.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .tune import Autotuner


class BatchedSearch:
    def __init__(self, ctx: B.Context, dbs, batch_panels, batch_sizes, k: int, threshold: int = B.NO_THRESHOLD,
                 variant: int | None = None, tuner: Autotuner | None = None, device: int = 0):
        self.ctx, self.dbs, self.k, self.threshold = ctx, list(dbs), k, threshold
        dev = torch.device("cuda", device)
        self.batches = []
        for p, n in zip(batch_panels, batch_sizes):
            w = (self.dbs[p].n_loci + 63) // 64
            self.batches.append((int(p),
                                 torch.zeros((n, w), dtype=torch.int64, device=dev),
                                 torch.zeros(n, dtype=torch.uint8, device=dev),
                                 torch.zeros((n, k), dtype=torch.int32, device=dev),
                                 torch.zeros((n, k), dtype=torch.int64, device=dev)))
        if variant is None:
            variant = (tuner or Autotuner()).choose(ctx, self.dbs, self.batches, k, threshold)
        self.variant = variant
        self.plan = B.Plan(ctx, self.dbs, self.batches, k, threshold, variant)
        self.plan.capture()
        total_words = sum(b[1].numel() for b in self.batches)
        total_q = sum(b[1].size(0) for b in self.batches)
        # pinned staging: all batches' words, modes, and results, contiguous
        self._h_words = torch.empty(max(total_words, 1), dtype=torch.int64, pin_memory=True)
        self._h_modes = torch.empty(max(total_q, 1), dtype=torch.uint8, pin_memory=True)
        self._h_sc = torch.empty(max(total_q * k, 1), dtype=torch.int32, pin_memory=True)
        self._h_ix = torch.empty(max(total_q * k, 1), dtype=torch.int64, pin_memory=True)

    @property
    def n_queries(self) -> int:
        return sum(b[1].size(0) for b in self.batches)

    def set_queries(self, i: int, packed: torch.Tensor, modes: torch.Tensor) -> None:
        """Copy device-resident packed queries/modes into batch i's buffers."""
        _, q, m, _, _ = self.batches[i]
        q.copy_(packed, non_blocking=True)
        m.copy_(modes, non_blocking=True)

    def run_device(self, stream=None) -> None:
        self.plan.replay(stream)

    def results(self, i: int):
        _, _, _, sc, ix = self.batches[i]
        return sc, ix

    def run_host(self, packed_list, modes_list):
        """Host arrays in, host arrays out.  Returns ([scores uint32 [n, k]],
        [idx int64 [n, k]], h2d bytes, d2h bytes)."""
        hw = self._h_words.numpy()
        hm = self._h_modes.numpy()
        ow, om = 0, 0
        for (_, q, m, _, _), pk, md in zip(self.batches, packed_list, modes_list):
            n, w = q.shape
            if n == 0:
                continue
            hw[ow:ow + n * w] = np.asarray(pk, dtype=np.uint64).view(np.int64).reshape(-1)
            hm[om:om + n] = md
            q.view(-1).copy_(self._h_words[ow:ow + n * w], non_blocking=True)
            m.copy_(self._h_modes[om:om + n], non_blocking=True)
            ow += n * w
            om += n
        self.plan.replay()
        os_, oi = 0, 0
        k = self.k
        for (_, q, _, sc, ix) in self.batches:
            n = q.size(0)
            if n == 0:
                continue
            self._h_sc[os_:os_ + n * k].copy_(sc.view(-1), non_blocking=True)
            self._h_ix[oi:oi + n * k].copy_(ix.view(-1), non_blocking=True)
            os_ += n * k
            oi += n * k
        # synchronises the stream; raises if the device recorded a condition
        # (a bounded wait that ran out): results are then not returned
        self.ctx.check(B.fastid_sync_status(self.ctx, torch.cuda.current_stream()))
        scores, idx = [], []
        off = 0
        for (_, q, _, _, _) in self.batches:
            n = q.size(0)
            scores.append(self._h_sc[off:off + n * k].numpy().view(np.uint32).reshape(n, k).copy())
            idx.append(self._h_ix[off:off + n * k].numpy().reshape(n, k).copy())
            off += n * k
        h2d = 8 * ow + om
        d2h = 12 * off
        return scores, idx, h2d, d2h

    def close(self):
        self.plan.close()
