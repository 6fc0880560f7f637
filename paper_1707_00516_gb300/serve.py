"""Continuous-batching server over a device-resident reference database.

Requests (a few packed query profiles each) arrive at any time.  A dispatcher
thread coalesces every waiting request, first come first served, into one
*wave* -- up to `max_wave` queries -- and runs it as one fastid_topk pass over
the database on a free *slot*.  A slot is a CUDA stream with its own pinned
host and device buffers; the number of slots is what the HBM budget admits,
so new requests are admitted as slots (and their memory) free up, and waves
on different slots overlap on the device (copies of one wave run under the
compare kernel of another).  A completion thread waits for each wave, splits
its results per request and resolves the requests' futures.

Each request's result depends only on its own queries (top-k is per query and
ties break by reference index), so it is the same whether it ran alone or in
a wave with others.  Only the dispatcher thread calls into the library.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from concurrent.futures import Future

import numpy as np
import torch

from . import binding as B


class _Request:
    __slots__ = ("packed", "modes", "n", "t_submit", "future")

    def __init__(self, packed, modes):
        self.packed = packed
        self.modes = modes
        self.n = packed.shape[0]
        self.t_submit = time.perf_counter()
        self.future = Future()


class _Slot:
    def __init__(self, device, max_wave, words, k):
        self.stream = torch.cuda.Stream(device=device)
        self.h_q = torch.empty((max_wave, words), dtype=torch.int64, pin_memory=True)
        self.h_m = torch.empty(max_wave, dtype=torch.uint8, pin_memory=True)
        self.h_sc = torch.empty((max_wave, k), dtype=torch.int32, pin_memory=True)
        self.h_ix = torch.empty((max_wave, k), dtype=torch.int64, pin_memory=True)
        self.d_q = torch.empty((max_wave, words), dtype=torch.int64, device=device)
        self.d_m = torch.empty(max_wave, dtype=torch.uint8, device=device)
        self.d_sc = torch.empty((max_wave, k), dtype=torch.int32, device=device)
        self.d_ix = torch.empty((max_wave, k), dtype=torch.int64, device=device)
        self.done = torch.cuda.Event()


def slot_device_bytes(n_loci: int, max_wave: int, k: int, tensor: bool, sms: int = 152) -> int:
    """Device memory one slot can hold at once: its buffers plus the scratch
    fastid_topk takes for a full wave."""
    words = (n_loci + 63) // 64
    kpad = (n_loci + 127) // 128 * 128
    n_pad = (max_wave + 127) // 128 * 128
    buffers = max_wave * (8 * words + 1 + 12 * k)
    scratch = n_pad * (kpad + 4 if tensor else 8 * words + 8) + sms * 3 * 128 * k * 8
    return buffers + scratch


class Server:
    def __init__(self, ctx: B.Context, db: B.RefDB, k: int, threshold: int = B.NO_THRESHOLD,
                 hbm_budget_bytes: int = 1 << 30, max_wave: int = 4096, max_slots: int = 3, device: int = 0):
        self.ctx, self.db, self.k, self.threshold = ctx, db, k, threshold
        self.device = torch.device("cuda", device)
        self.words = (db.n_loci + 63) // 64
        self.max_wave = max_wave
        per_slot = slot_device_bytes(db.n_loci, max_wave, k, bool(db.flags & B.REFS_TENSOR))
        n_slots = max(1, min(max_slots, hbm_budget_bytes // per_slot))
        self.slot_bytes = per_slot
        self.slots = [_Slot(self.device, max_wave, self.words, k) for _ in range(n_slots)]
        self._free: queue.Queue = queue.Queue()
        for s in self.slots:
            self._free.put(s)
        self._pending: collections.deque = collections.deque()
        self._cv = threading.Condition()
        # a context is used by one host thread at a time: the dispatcher's
        # launches and the completion thread's status reads take turns
        self._lib = threading.Lock()
        self._inflight: queue.Queue = queue.Queue()
        self._stop = False
        self.latencies: list[float] = []
        self.records: list[tuple[float, float]] = []  # (submit time, latency) per request
        self.waves = 0
        self.queries = 0
        self.wave_sizes: list[int] = []
        self._disp = threading.Thread(target=self._dispatch, name="fastid-dispatch", daemon=True)
        self._comp = threading.Thread(target=self._complete, name="fastid-complete", daemon=True)
        self._disp.start()
        self._comp.start()

    # ---- public --------------------------------------------------------------
    def submit(self, packed: np.ndarray, modes: np.ndarray) -> Future:
        """Queue one request: packed uint64 [n, words], modes uint8 [n].
        The future resolves to (scores uint32 [n, k], idx int64 [n, k])."""
        packed = np.ascontiguousarray(packed).view(np.uint64)
        modes = np.ascontiguousarray(modes, dtype=np.uint8)
        if packed.ndim != 2 or packed.shape[1] != self.words or modes.shape != (packed.shape[0],):
            raise ValueError("packed must be [n, words] with one mode per query")
        if packed.shape[0] > self.max_wave:
            raise ValueError(f"request of {packed.shape[0]} queries exceeds max_wave {self.max_wave}")
        r = _Request(packed, modes)
        with self._cv:
            if self._stop:
                raise RuntimeError("server stopped")
            self._pending.append(r)
            self._cv.notify()
        return r.future

    def close(self, timeout: float = 60.0):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._disp.join(timeout)
        self._inflight.put(None)
        self._comp.join(timeout)

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "queries": self.queries, "waves": self.waves,
                "slots": len(self.slots), "slot_bytes": self.slot_bytes,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_wave": float(np.mean(self.wave_sizes)) if self.wave_sizes else 0.0}

    # ---- threads ----------------------------------------------------------------
    def _dispatch(self):
        torch.cuda.set_device(self.device)
        while True:
            slot = self._free.get()
            with self._cv:
                while not self._pending and not self._stop:
                    self._cv.wait()
                if not self._pending and self._stop:
                    self._free.put(slot)
                    return
                wave, n = [], 0
                while self._pending and n + self._pending[0].n <= self.max_wave:
                    r = self._pending.popleft()
                    wave.append(r)
                    n += r.n
            try:
                self._launch(slot, wave, n)
            except Exception as e:  # report to every request of the wave
                for r in wave:
                    r.future.set_exception(e)
                self._free.put(slot)
                continue
            self._inflight.put((slot, wave, n))

    def _launch(self, slot: _Slot, wave, n: int):
        hq, hm = slot.h_q.numpy(), slot.h_m.numpy()
        o = 0
        for r in wave:
            hq[o:o + r.n] = r.packed.view(np.int64)
            hm[o:o + r.n] = r.modes
            o += r.n
        with torch.cuda.stream(slot.stream):
            slot.d_q[:n].copy_(slot.h_q[:n], non_blocking=True)
            slot.d_m[:n].copy_(slot.h_m[:n], non_blocking=True)
            with self._lib:
                B.fastid_topk(self.ctx, self.db, slot.d_q[:n], slot.d_m[:n], self.k, self.threshold,
                              slot.d_sc[:n], slot.d_ix[:n], stream=slot.stream)
            slot.h_sc[:n].copy_(slot.d_sc[:n], non_blocking=True)
            slot.h_ix[:n].copy_(slot.d_ix[:n], non_blocking=True)
            slot.done.record(slot.stream)

    def _complete(self):
        while True:
            item = self._inflight.get()
            if item is None:
                return
            slot, wave, n = item
            try:
                slot.done.synchronize()
                # conditions the device recorded (a bounded wait that ran out):
                # the wave's results are not delivered.  The status word is the
                # context's, so with several waves in flight a condition fails
                # the wave whose completion reads it first.
                with self._lib:
                    self.ctx.check(B.fastid_sync_status(self.ctx, slot.stream))
                sc = slot.h_sc[:n].numpy().view(np.uint32)
                ix = slot.h_ix[:n].numpy()
                now = time.perf_counter()
                o = 0
                for r in wave:
                    r.future.set_result((sc[o:o + r.n].copy(), ix[o:o + r.n].copy()))
                    self.latencies.append(now - r.t_submit)
                    self.records.append((r.t_submit, now - r.t_submit))
                    o += r.n
                self.waves += 1
                self.queries += n
                self.wave_sizes.append(n)
            except Exception as e:  # report to every request of the wave
                for r in wave:
                    if not r.future.done():
                        r.future.set_exception(e)
            self._free.put(slot)
