"""User-facing search API over the C ABI: a resident reference database and
queries given as contributor allele rows, on the device or on the host.

The host path (`Searcher.search_host`) is what an application calls with
host inputs (numpy arrays, staged through pinned buffers, or pinned CPU
tensors, copied directly): it copies them to the device, runs pack -> mix ->
top-k in the library's kernels and copies the result back.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def words64(n_loci: int) -> int:
    return (n_loci + 63) // 64


class Searcher:
    def __init__(self, device: int = 0, form: int = B.FORM_AUTO):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.ctx = B.Context(device)
        self.form = form
        B.fastid_set_form(self.ctx, form)
        self._pinned: dict[str, torch.Tensor] = {}
        self._devbuf: dict[str, torch.Tensor] = {}

    # ---- database ------------------------------------------------------
    def load_refs_packed(self, packed: torch.Tensor, n_loci: int, flags: int = 0) -> B.RefDB:
        return B.fastid_load_refs(self.ctx, packed, n_loci, flags)

    def default_flags(self) -> int:
        """Database flags the chosen form needs (the operand copy it reads)."""
        if self.form == B.FORM_TENSOR:
            return B.REFS_TENSOR
        return B.REFS_FP4 if self.form in (B.FORM_TENSOR_FP4, B.FORM_AUTO) else 0

    def load_refs_alleles(self, alleles: torch.Tensor, n_loci: int, flags: int | None = None) -> B.RefDB:
        """Pack uint8 allele rows already on the device and load them."""
        if flags is None:
            flags = self.default_flags()
        packed = torch.empty((alleles.shape[0], words64(n_loci)), dtype=torch.int64, device=self.device)
        B.fastid_pack(self.ctx, alleles, n_loci, packed)
        db = B.fastid_load_refs(self.ctx, packed, n_loci, flags)
        torch.cuda.current_stream().synchronize()
        return db

    # ---- queries ---------------------------------------------------------
    def build_queries(self, src_alleles: torch.Tensor, offsets: torch.Tensor, n_loci: int) -> torch.Tensor:
        """Pack contributor rows and OR each group into one query profile."""
        n_src = src_alleles.shape[0]
        n_q = offsets.numel() - 1
        w = words64(n_loci)
        src_packed = self._buf("src_packed", (max(n_src, 1), w), torch.int64)[:n_src]
        B.fastid_pack(self.ctx, src_alleles, n_loci, src_packed)
        q = self._buf("queries", (max(n_q, 1), w), torch.int64)[:n_q]
        B.fastid_mix(self.ctx, src_packed, w, offsets, q)
        return q

    def tune_form(self, db: B.RefDB, queries: torch.Tensor, modes: torch.Tensor, k: int,
                  threshold: int = B.NO_THRESHOLD, tuner=None) -> int:
        """Measure (or recall) the fastest form for calls like this one and
        make it the context's form (tune.FormTuner)."""
        from .tune import FormTuner
        self.form = (tuner or FormTuner()).choose(self.ctx, db, queries, modes, k, threshold)
        B.fastid_set_form(self.ctx, self.form)
        return self.form

    def topk(self, db: B.RefDB, queries: torch.Tensor, modes: torch.Tensor, k: int,
             threshold: int = B.NO_THRESHOLD):
        n_q = queries.shape[0]
        sc = torch.empty((n_q, k), dtype=torch.int32, device=self.device)
        ix = torch.empty((n_q, k), dtype=torch.int64, device=self.device)
        B.fastid_topk(self.ctx, db, queries, modes, k, threshold, sc, ix)
        return sc, ix

    def topk_streamed(self, refs_host: torch.Tensor, n_loci: int, queries: torch.Tensor, modes: torch.Tensor,
                      k: int, threshold: int = B.NO_THRESHOLD, block_refs: int = 1 << 22,
                      flags: int = B.REFS_TENSOR):
        """Top-k against packed references kept in host memory (int64
        [n_refs][words]; pinned for overlapped copies), streamed in blocks."""
        n_q = queries.shape[0]
        sc = torch.empty((n_q, k), dtype=torch.int32, device=self.device)
        ix = torch.empty((n_q, k), dtype=torch.int64, device=self.device)
        B.fastid_topk_streamed(self.ctx, refs_host, n_loci, flags, block_refs, queries, modes, k, threshold, sc, ix)
        return sc, ix

    def hits_streamed(self, refs_host: torch.Tensor, n_loci: int, queries: torch.Tensor, modes: torch.Tensor,
                      threshold: int, capacity: int, block_refs: int = 1 << 22, flags: int = B.REFS_TENSOR):
        """Hit list against packed references kept in host memory."""
        hq = torch.empty(capacity, dtype=torch.int64, device=self.device)
        hr = torch.empty(capacity, dtype=torch.int64, device=self.device)
        hs = torch.empty(capacity, dtype=torch.int32, device=self.device)
        hc = torch.zeros(1, dtype=torch.int64, device=self.device)
        B.fastid_compare_streamed(self.ctx, refs_host, n_loci, flags, block_refs, queries, modes, threshold, hq, hr,
                                  hs, hc)
        return hq, hr, hs, hc

    def hits(self, db: B.RefDB, queries: torch.Tensor, modes: torch.Tensor, threshold: int, capacity: int):
        hq = torch.empty(capacity, dtype=torch.int64, device=self.device)
        hr = torch.empty(capacity, dtype=torch.int64, device=self.device)
        hs = torch.empty(capacity, dtype=torch.int32, device=self.device)
        hc = torch.zeros(1, dtype=torch.int64, device=self.device)
        B.fastid_compare(self.ctx, db, queries, modes, threshold, hq, hr, hs, hc)
        return hq, hr, hs, hc

    def scores(self, db: B.RefDB, queries: torch.Tensor, modes: torch.Tensor, dtype=torch.int32):
        out = torch.empty((queries.shape[0], db.n_refs), dtype=dtype, device=self.device)
        B.fastid_scores(self.ctx, db, queries, modes, out)
        return out

    # ---- host in, host out ---------------------------------------------
    def _buf(self, name, shape, dtype):
        t = self._devbuf.get(name)
        n = int(np.prod(shape))
        if t is None or t.numel() < n or t.dtype != dtype:
            t = torch.empty(n, dtype=dtype, device=self.device)
            self._devbuf[name] = t
        return t[:n].view(shape)

    def _pin(self, name, arr: np.ndarray) -> torch.Tensor:
        t = self._pinned.get(name)
        if t is None or t.numel() < arr.size or t.dtype != _TORCH[arr.dtype]:
            t = torch.empty(max(arr.size, 1), dtype=_TORCH[arr.dtype], pin_memory=True)
            self._pinned[name] = t
        v = t[:arr.size].view(arr.shape)
        v.numpy()[...] = arr
        return v

    def _host_input(self, name, x, dtype: np.dtype) -> torch.Tensor:
        """A pinned host tensor holding x: x itself when it already is a
        contiguous pinned CPU tensor of that dtype, else a staged copy."""
        if isinstance(x, torch.Tensor):
            if x.device.type != "cpu" or x.dtype != _TORCH[np.dtype(dtype)]:
                raise ValueError(f"{name}: expected a CPU tensor of {np.dtype(dtype)}")
            if x.is_pinned() and x.is_contiguous():
                return x
            x = x.numpy()
        return self._pin(name, np.ascontiguousarray(x, dtype))

    def search_host(self, db: B.RefDB, src_alleles, offsets, modes, k: int, threshold: int = B.NO_THRESHOLD):
        """Top-k for queries given on the host as contributor rows.

        src_alleles uint8 [n_src, N]; offsets int32 [n_q + 1]; modes uint8 [n_q]:
        numpy arrays (staged through pinned buffers) or pinned CPU tensors
        (copied to the device directly).  Returns numpy (scores uint32
        [n_q, k], idx int64 [n_q, k]) and the bytes copied each way.
        """
        n_loci = src_alleles.shape[1]
        h_src = self._host_input("src", src_alleles, np.uint8)
        h_off = self._host_input("off", offsets, np.int32)
        h_mod = self._host_input("mod", modes, np.uint8)
        d_src = self._buf("d_src", h_src.shape, torch.uint8)
        d_off = self._buf("d_off", h_off.shape, torch.int32)
        d_mod = self._buf("d_mod", h_mod.shape, torch.uint8)
        d_src.copy_(h_src, non_blocking=True)
        d_off.copy_(h_off, non_blocking=True)
        d_mod.copy_(h_mod, non_blocking=True)
        q = self.build_queries(d_src, d_off, n_loci)
        n_q = q.shape[0]
        sc = self._buf("d_sc", (n_q, k), torch.int32)
        ix = self._buf("d_ix", (n_q, k), torch.int64)
        B.fastid_topk(self.ctx, db, q, d_mod, k, threshold, sc, ix)
        o_sc = self._pin_out("o_sc", (n_q, k), torch.int32)
        o_ix = self._pin_out("o_ix", (n_q, k), torch.int64)
        o_sc.copy_(sc, non_blocking=True)
        o_ix.copy_(ix, non_blocking=True)
        # synchronises the stream; raises if the device recorded a condition
        # (a bounded wait that ran out): results are then not returned
        self.ctx.check(B.fastid_sync_status(self.ctx, torch.cuda.current_stream()))
        h2d = h_src.numel() + 4 * h_off.numel() + h_mod.numel()
        d2h = 4 * o_sc.numel() + 8 * o_ix.numel()
        return o_sc.numpy().view(np.uint32).copy(), o_ix.numpy().copy(), h2d, d2h

    def _pin_out(self, name, shape, dtype):
        t = self._pinned.get(name)
        n = int(np.prod(shape))
        if t is None or t.numel() < n or t.dtype != dtype:
            t = torch.empty(max(n, 1), dtype=dtype, pin_memory=True)
            self._pinned[name] = t
        return t[:n].view(shape)


_TORCH = {np.dtype(np.uint8): torch.uint8, np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64}
