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
    fastid_topk takes for a full wave: the query operand and the per-segment
    top-k lists, at most 4 x SMs lists of 128 queries (the plain kernel's two
    CTAs an SM, each over at most two query tiles for waves up to 38,912
    queries; the tensor kernel's slots are fewer)."""
    words = (n_loci + 63) // 64
    kpad = (n_loci + 127) // 128 * 128
    n_pad = (max_wave + 127) // 128 * 128
    buffers = max_wave * (8 * words + 1 + 12 * k)
    scratch = n_pad * (kpad + 4 if tensor else 8 * words + 8) + sms * 4 * 128 * k * 8
    return buffers + scratch


class Server:
    def __init__(self, ctx: B.Context, db: B.RefDB, k: int, threshold: int = B.NO_THRESHOLD,
                 hbm_budget_bytes: int = 1 << 30, max_wave: int = 4096, max_slots: int = 3, device: int = 0):
        self.ctx, self.db, self.k, self.threshold = ctx, db, k, threshold
        self.device = torch.device("cuda", device)
        self.words = (db.n_loci + 63) // 64
        self.max_wave = max_wave
        per_slot = slot_device_bytes(db.n_loci, max_wave, k, True)  # any tensor operand (the largest scratch)
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


# ---------------------------------------------------------------------------
# Continuous batching over a running pass: waves share every launch
# ---------------------------------------------------------------------------

class _SweepWave:
    __slots__ = ("reqs", "off", "n", "j_first", "j_end", "epoch", "done", "error")

    def __init__(self, reqs, off, n, j, parts, epoch):
        self.reqs, self.off, self.n = reqs, off, n
        self.j_first, self.j_end = j, j + parts - 1
        self.epoch = epoch
        self.done = None
        self.error = None


class SweepServer:
    """Continuous batching whose waves overlap on the device.

    The database is split into `parts` row ranges (fastid_refs_view).  While
    any request is in flight, a dispatcher thread runs one *step* after
    another on its stream: a step compares ONE part against the queries of
    every active wave -- one fastid_topk_accumulate over the ring rows they
    occupy: one comparison launch, whose merge folds the part's lists into
    each query's running list (an exact (score, reference) merge).  Requests that
    arrive meanwhile are admitted together, as one new wave, into the next
    step, whichever part that is: a pass may start at any part boundary and
    wrap round.  A wave leaves after `parts` steps, having met every part
    once, and its running lists are then exactly fastid_topk over the whole
    database.  So the waves in flight share the launches of their common
    steps (their work overlaps on the device), and a request waits about one
    part, not a whole pass, for its first comparison.

    Admission is by memory: a wave takes contiguous rows of a fixed ring of
    `capacity` query rows (packed queries, modes and running lists on the
    device, pinned staging on the host) and is admitted only when its rows
    are free; rows are released in order as waves complete.  At most
    `lookahead` steps are queued on the device, so an arriving request joins
    within a step or two.

    A request's result depends only on its own queries (top-k is per query,
    ties break by reference index, and the fold is order-free), so it is the
    same alone and in a mix.  A condition recorded on the device (a bounded
    wait that ran out) fails the wave that reads it and every wave in flight
    with it.  Only this object's threads call into the library, one at a
    time.
    """

    def __init__(self, ctx: B.Context, db: B.RefDB, k: int, threshold: int = B.NO_THRESHOLD, parts: int = 4,
                 capacity: int = 2048, max_wave: int = 256, lookahead: int = 2, device: int = 0):
        if parts < 1 or capacity < max_wave or lookahead < 1:
            raise ValueError("need parts >= 1, capacity >= max_wave and lookahead >= 1")
        self.ctx, self.db, self.k, self.threshold = ctx, db, k, threshold
        self.device = torch.device("cuda", device)
        self.words = (db.n_loci + 63) // 64
        self.max_wave, self.capacity, self.lookahead = max_wave, capacity, lookahead
        per = -(-db.n_refs // parts)
        per = -(-per // B.VIEW_ALIGN) * B.VIEW_ALIGN
        self.bounds = [(r0, min(per, db.n_refs - r0)) for r0 in range(0, db.n_refs, per)]
        self.parts = len(self.bounds)
        self.views = [B.fastid_refs_view(ctx, db, r0, n) for r0, n in self.bounds]
        C, dev = capacity, self.device
        self.d_q = torch.zeros((C, self.words), dtype=torch.int64, device=dev)
        self.d_m = torch.zeros(C, dtype=torch.uint8, device=dev)
        self.run_s = torch.empty((C, k), dtype=torch.int32, device=dev)
        self.run_i = torch.empty((C, k), dtype=torch.int64, device=dev)
        self.h_q = torch.empty((C, self.words), dtype=torch.int64, pin_memory=True)
        self.h_m = torch.empty(C, dtype=torch.uint8, pin_memory=True)
        self.h_s = torch.empty((C, k), dtype=torch.int32, pin_memory=True)
        self.h_i = torch.empty((C, k), dtype=torch.int64, pin_memory=True)
        self.stream = torch.cuda.Stream(device=dev)
        self.status_stream = torch.cuda.Stream(device=dev)
        self._pending: collections.deque = collections.deque()
        self._active: list[_SweepWave] = []
        self._alloc: collections.deque = collections.deque()  # (off, n) of waves holding rows, in order
        self._head = self._tail = 0
        self._cv = threading.Condition()
        self._lib = threading.Lock()
        self._done_q: queue.Queue = queue.Queue()
        self._stop = False
        self._epoch = 0
        self.latencies: list[float] = []
        self.records: list[tuple[float, float]] = []
        self.waves = 0
        self.queries = 0
        self.wave_sizes: list[int] = []
        self.steps = 0
        # per step: (start event, end event, ids of the waves it served), while tracing
        self.trace: list[tuple[torch.cuda.Event, torch.cuda.Event, tuple[int, ...]]] | None = None
        self._disp = threading.Thread(target=self._dispatch, name="fastid-sweep", daemon=True)
        self._comp = threading.Thread(target=self._complete, name="fastid-sweep-complete", daemon=True)
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
        self._done_q.put(None)
        self._comp.join(timeout)
        for v in self.views:
            v.close()
        self.views = []

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "queries": self.queries, "waves": self.waves,
                "slots": f"{self.parts} parts, {self.capacity}-query ring", "steps": self.steps,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_wave": float(np.mean(self.wave_sizes)) if self.wave_sizes else 0.0}

    # ---- ring of query rows (caller holds self._cv) -------------------------------
    def _ring_alloc(self, n: int):
        C = self.capacity
        if not self._alloc:
            self._head = self._tail = 0
        head, tail = self._head, self._tail
        if not self._alloc or tail > head:  # free: [tail, C) and [0, head)
            off = tail if tail + n <= C else (0 if n <= head else None)
        else:  # wrapped: free [tail, head)
            off = tail if tail + n <= head else None
        if off is not None:
            self._alloc.append((off, n))
            self._tail = off + n
        return off

    def _ring_release(self):
        self._alloc.popleft()
        self._head = self._alloc[0][0] if self._alloc else self._tail

    def _admit_locked(self, j: int):
        """One new wave from the pending requests (first come, first served,
        up to max_wave queries) if its rows are free."""
        reqs, n = [], 0
        for r in self._pending:
            if n + r.n > self.max_wave:
                break
            reqs.append(r)
            n += r.n
        if not reqs:
            return None
        off = self._ring_alloc(n)
        if off is None:
            return None
        for _ in reqs:
            self._pending.popleft()
        w = _SweepWave(reqs, off, n, j, self.parts, self._epoch)
        self._active.append(w)
        return w

    # ---- threads ----------------------------------------------------------------
    def _spans(self, active):
        spans = []
        for w in active:
            if spans and spans[-1][1] == w.off:
                spans[-1][1] = w.off + w.n
            else:
                spans.append([w.off, w.off + w.n])
        return spans

    def _stage(self, w: _SweepWave):
        hq, hm = self.h_q.numpy(), self.h_m.numpy()
        o = w.off
        for r in w.reqs:
            hq[o:o + r.n] = r.packed.view(np.int64)
            hm[o:o + r.n] = r.modes
            o += r.n
        a, b = w.off, w.off + w.n
        self.d_q[a:b].copy_(self.h_q[a:b], non_blocking=True)
        self.d_m[a:b].copy_(self.h_m[a:b], non_blocking=True)
        self.run_s[a:b].fill_(-1)  # empty lists: (0xFFFFFFFF, -1)
        self.run_i[a:b].fill_(-1)

    def _dispatch(self):
        torch.cuda.set_device(self.device)
        j = 0
        queued: collections.deque = collections.deque()
        while True:
            with self._cv:
                while not self._stop and not self._pending and not self._active:
                    self._cv.wait()
                if self._stop and not self._pending and not self._active:
                    return
                failed = [w for w in self._active if w.epoch < self._epoch]
                for w in failed:
                    self._active.remove(w)
                new = self._admit_locked(j)
                active = list(self._active)
                if not active and not failed:
                    # nothing to run: the pending wave waits for rows that
                    # waves still completing hold (released with a notify)
                    self._cv.wait(0.05)
                    continue
            for w in failed:  # a device condition was seen while they were in flight
                w.error = B.FastIDError(B.ETIMEOUT, "device condition recorded while the wave was in flight")
                self._done_q.put(w)
            if not active:
                continue
            part = j % self.parts
            r0 = self.bounds[part][0]
            finishing = [w for w in active if w.j_end == j]
            try:
                with torch.cuda.stream(self.stream), self._lib:
                    if new is not None:
                        self._stage(new)
                    ev0 = torch.cuda.Event(enable_timing=True) if self.trace is not None else None
                    if ev0 is not None:
                        ev0.record(self.stream)
                    for a, b in self._spans(active):
                        B.fastid_topk_accumulate(self.ctx, self.views[part], r0, self.d_q[a:b], self.d_m[a:b],
                                                 self.k, self.threshold, self.run_s[a:b], self.run_i[a:b],
                                                 stream=self.stream)
                    ev = torch.cuda.Event(enable_timing=self.trace is not None)
                    ev.record(self.stream)
                    if ev0 is not None:
                        self.trace.append((ev0, ev, tuple(id(w) for w in active)))
                    for w in finishing:
                        a, b = w.off, w.off + w.n
                        self.h_s[a:b].copy_(self.run_s[a:b], non_blocking=True)
                        self.h_i[a:b].copy_(self.run_i[a:b], non_blocking=True)
                        w.done = torch.cuda.Event()
                        w.done.record(self.stream)
            except Exception as e:  # fail every wave of the step
                with self._cv:
                    for w in active:
                        self._active.remove(w)
                for w in active:
                    w.error = e
                    self._done_q.put(w)
                continue
            self.steps += 1
            with self._cv:
                for w in finishing:
                    self._active.remove(w)
            for w in finishing:
                self._done_q.put(w)
            j += 1
            queued.append(ev)
            while len(queued) >= self.lookahead:
                queued.popleft().synchronize()

    def _complete(self):
        while True:
            w = self._done_q.get()
            if w is None:
                return
            try:
                if w.error is not None:
                    raise w.error
                w.done.synchronize()
                with self._lib:
                    self.status_stream.wait_event(w.done)
                    st = B.fastid_sync_status(self.ctx, self.status_stream)
                if st != B.OK or w.epoch < self._epoch:
                    if st != B.OK:
                        with self._cv:
                            self._epoch += 1
                    raise B.FastIDError(st if st != B.OK else B.ETIMEOUT,
                                        "device condition recorded while the wave was in flight")
                a, b = w.off, w.off + w.n
                sc = self.h_s[a:b].numpy().view(np.uint32)
                ix = self.h_i[a:b].numpy()
                now = time.perf_counter()
                o = 0
                for r in w.reqs:
                    r.future.set_result((sc[o:o + r.n].copy(), ix[o:o + r.n].copy()))
                    self.latencies.append(now - r.t_submit)
                    self.records.append((r.t_submit, now - r.t_submit))
                    o += r.n
                self.waves += 1
                self.queries += w.n
                self.wave_sizes.append(w.n)
            except Exception as e:  # report to every request of the wave
                for r in w.reqs:
                    if not r.future.done():
                        r.future.set_exception(e)
            with self._cv:
                self._ring_release()
                self._cv.notify_all()
