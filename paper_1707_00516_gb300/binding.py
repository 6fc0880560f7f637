"""Python binding of the C ABI in ``include/fastid.h``.

Argument marshalling only: every function here checks tensor placement and
dtype, turns tensors into device pointers and calls the entry point of the
same name in ``libfastid.so``.  Unsigned buffers travel in signed tensors of
the same width (uint64 words in int64, uint32 scores in int32, uint16 scores
in int16): the bits are the C ABI's, only the dtype label differs.  PyTorch supplies device memory and streams;
no step of the comparison runs in Python or on the CPU.  If the compiled
library is missing, loading it raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfastid.so")

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEOUT, EUNSUPPORTED, EDEVICE = range(8)
MODE_MISMATCH, MODE_UNEXPLAINED = 0, 1
FORM_AUTO, FORM_PLAIN, FORM_TENSOR, FORM_TENSOR_PACKED, FORM_TENSOR_FP4, FORM_TENSOR_FP4_PACKED = range(6)
REFS_TENSOR, REFS_FP4 = 1, 2
MAX_K = 32
MAX_LOCI = 65536
NO_THRESHOLD = 0xFFFFFFFF
NOALLOC_SCRATCH_BYTES = 32 << 20
VIEW_ALIGN = 256
(VARIANT_AUTO, VARIANT_TENSOR_N256, VARIANT_TENSOR_N128, VARIANT_TENSOR_PAIR, VARIANT_TENSOR_FP4,
 VARIANT_TENSOR_FP4_PAIR, VARIANT_TENSOR_PAIR_2SM, VARIANT_TENSOR_FP4_PAIR_2SM) = range(8)

_lib = None
_lock = threading.Lock()


class FastIDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_STATUS_NAMES = {0: "FASTID_OK", 1: "FASTID_EINVAL", 2: "FASTID_ENOMEM", 3: "FASTID_ECUDA",
                 4: "FASTID_EOVERFLOW", 5: "FASTID_ETIMEOUT", 6: "FASTID_EUNSUPPORTED",
                 7: "FASTID_EDEVICE"}

_P, _I64, _I32, _U32, _U8 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint8

_PROTOS = {
    "fastid_version": (_I32, []),
    "fastid_status_string": (ctypes.c_char_p, [_I32]),
    "fastid_create": (_I32, [ctypes.POINTER(_P), _I32]),
    "fastid_destroy": (_I32, [_P]),
    "fastid_last_error": (ctypes.c_char_p, [_P]),
    "fastid_memory_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "fastid_set_form": (_I32, [_P, _I32]),
    "fastid_sync_status": (_I32, [_P, _P]),
    "fastid_profile": (_I32, [_P, _I32]),
    "fastid_profile_read": (_I32, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_I64), _I32]),
    "fastid_pack": (_I32, [_P, _P, _I64, _I32, _I64, _P, _I64, _P, _P]),
    "fastid_mix": (_I32, [_P, _P, _I64, _I32, _P, _I64, _P, _I64, _P, _P]),
    "fastid_load_refs": (_I32, [_P, _P, _I64, _I32, _I64, _U32, ctypes.POINTER(_P), _P]),
    "fastid_free_refs": (_I32, [_P, _P]),
    "fastid_refs_view": (_I32, [_P, _P, _I64, _I64, ctypes.POINTER(_P)]),
    "fastid_topk_fold": (_I32, [_P, _P, _P, _P, _P, _I64, _I64, _I32, _P]),
    "fastid_topk_accumulate": (_I32, [_P, _P, _I64, _P, _I64, _I64, _P, _I32, _U32, _P, _P, _P]),
    "fastid_refs_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.POINTER(_U32),
                                ctypes.POINTER(_I64)]),
    "fastid_scores": (_I32, [_P, _P, _P, _I64, _I64, _P, _P, _I32, _I64, _P]),
    "fastid_topk": (_I32, [_P, _P, _P, _I64, _I64, _P, _I32, _U32, _P, _P, _P]),
    "fastid_compare": (_I32, [_P, _P, _P, _I64, _I64, _P, _U32, _I64, _P, _P, _P, _P, _P]),
    "fastid_topk_noalloc": (_I32, [_P, _P, _P, _I64, _I64, _P, _I32, _U32, _P, _P, _P]),
    "fastid_topk_streamed": (_I32, [_P, _P, _I64, _I32, _I64, _U32, _I64, _P, _I64, _I64, _P, _I32, _U32, _P, _P,
                                    _P]),
    "fastid_compare_streamed": (_I32, [_P, _P, _I64, _I32, _I64, _U32, _I64, _P, _I64, _I64, _P, _U32, _I64, _P,
                                       _P, _P, _P, _P]),
    "fastid_wait_flag": (_I32, [_P, _P, _I32, _P]),
    "fastid_save_refs": (_I32, [_P, _P, ctypes.c_char_p]),
    "fastid_load_refs_file": (_I32, [_P, ctypes.c_char_p, _U32, _P, _P]),
    "fastid_plan_create": (_I32, [_P, _P, _I32, _P, _I32, _I32, _U32, _I32, ctypes.POINTER(_P)]),
    "fastid_plan_run": (_I32, [_P, _P]),
    "fastid_plan_capture": (_I32, [_P, _P]),
    "fastid_plan_replay": (_I32, [_P, _P]),
    "fastid_plan_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                                ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "fastid_plan_destroy": (_I32, [_P]),
}

# Every symbol the header declares (checked by the CPU tests).
EXPORTS = tuple(_PROTOS)


def load_library(path: str | None = None):
    """Load libfastid.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library {p} is missing: run __graft_entry__.build() or "
                                   "python -m paper_1707_00516_gb300.build")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _PROTOS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _dev(t: torch.Tensor | None, dtype: torch.dtype, name: str, ndim: int | None = None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")
    if ndim == 2:
        if t.stride(1) != 1:
            raise ValueError(f"{name} rows must be contiguous")
    elif not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _ld(t: torch.Tensor) -> int:
    return t.stride(0) if t.size(0) > 1 else t.size(1)


class Context:
    """Owns a fastid_ctx (C handle in .handle)."""

    def __init__(self, device: int | None = None):
        lib = load_library()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = _P()
        st = lib.fastid_create(ctypes.byref(h), self.device)
        if st != OK:
            raise FastIDError(st, "fastid_create failed")
        self.handle = h
        self._lib = lib

    def check(self, st: int):
        if st != OK:
            msg = self._lib.fastid_last_error(self.handle)
            raise FastIDError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fastid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class RefDB:
    """Owns a fastid_refdb loaded through fastid_load_refs."""

    def __init__(self, ctx: Context, handle, n_refs: int, n_loci: int, flags: int):
        self.ctx, self.handle, self.n_refs, self.n_loci, self.flags = ctx, handle, n_refs, n_loci, flags

    def info(self):
        n, l, f, b = _I64(), _I32(), _U32(), _I64()
        self.ctx.check(load_library().fastid_refs_info(self.handle, ctypes.byref(n), ctypes.byref(l),
                                                       ctypes.byref(f), ctypes.byref(b)))
        return {"n_refs": n.value, "n_loci": l.value, "flags": f.value, "device_bytes": b.value}

    def close(self):
        if getattr(self, "handle", None) and self.ctx.handle:
            load_library().fastid_free_refs(self.ctx.handle, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- entry points, same names as the C ABI ----------------------------------

def fastid_version() -> int:
    return int(load_library().fastid_version())


def fastid_set_form(ctx: Context, form: int) -> None:
    ctx.check(load_library().fastid_set_form(ctx.handle, form))


def fastid_profile(ctx: Context, enable: bool) -> None:
    ctx.check(load_library().fastid_profile(ctx.handle, 1 if enable else 0))


def fastid_profile_read(ctx: Context, reset: bool = True) -> dict:
    """{'main_ms', 'main_launches', 'all_launches'} since the last reset."""
    ms, ml, al = ctypes.c_double(), _I64(), _I64()
    ctx.check(load_library().fastid_profile_read(ctx.handle, ctypes.byref(ms), ctypes.byref(ml),
                                                 ctypes.byref(al), 1 if reset else 0))
    return {"main_ms": ms.value, "main_launches": ml.value, "all_launches": al.value}


def fastid_memory_info(ctx: Context) -> dict:
    """{'pool_allocs', 'pool_used_bytes', 'pool_reserved_bytes'} of the context."""
    a, u, r = _I64(), _I64(), _I64()
    ctx.check(load_library().fastid_memory_info(ctx.handle, ctypes.byref(a), ctypes.byref(u), ctypes.byref(r)))
    return {"pool_allocs": a.value, "pool_used_bytes": u.value, "pool_reserved_bytes": r.value}


def fastid_save_refs(ctx: Context, db: RefDB, path: str) -> None:
    ctx.check(load_library().fastid_save_refs(ctx.handle, db.handle, os.fsencode(path)))


def fastid_load_refs_file(ctx: Context, path: str, flags: int = 0, stream=None) -> RefDB:
    h = _P()
    ctx.check(load_library().fastid_load_refs_file(ctx.handle, os.fsencode(path), flags, ctypes.byref(h),
                                                   _stream_ptr(stream)))
    n, l, f, b = _I64(), _I32(), _U32(), _I64()
    ctx.check(load_library().fastid_refs_info(h, ctypes.byref(n), ctypes.byref(l), ctypes.byref(f), ctypes.byref(b)))
    return RefDB(ctx, h, n.value, l.value, f.value)


def fastid_wait_flag(ctx: Context, flag: torch.Tensor, wait_ms: int, stream=None) -> None:
    """Bounded device wait on flag (int32, one element, device) -- see fastid.h."""
    f = _dev(flag, torch.int32, "flag", 1)
    ctx.check(load_library().fastid_wait_flag(ctx.handle, f, wait_ms, _stream_ptr(stream)))


def fastid_sync_status(ctx: Context, stream=None) -> int:
    """Returns the status code (does not raise on EOVERFLOW / ETIMEOUT / EDEVICE)."""
    return int(load_library().fastid_sync_status(ctx.handle, _stream_ptr(stream)))


def fastid_pack(ctx: Context, alleles: torch.Tensor, n_loci: int, packed: torch.Tensor,
                norms: torch.Tensor | None = None, stream=None) -> None:
    a = _dev(alleles, torch.uint8, "alleles", 2)
    p = _dev(packed, torch.int64, "packed", 2)
    nm = _dev(norms, torch.int32, "norms")
    n = alleles.size(0)
    if packed.size(0) != n:
        raise ValueError("packed must have one row per allele row")
    ctx.check(load_library().fastid_pack(ctx.handle, a, n, n_loci, _ld(alleles), p, _ld(packed), nm,
                                         _stream_ptr(stream)))


def fastid_mix(ctx: Context, src: torch.Tensor, n_words: int, offsets: torch.Tensor, out: torch.Tensor,
               norms: torch.Tensor | None = None, stream=None) -> None:
    s = _dev(src, torch.int64, "src", 2)
    o = _dev(offsets, torch.int32, "offsets", 1)
    d = _dev(out, torch.int64, "out", 2)
    nm = _dev(norms, torch.int32, "norms")
    n_mix = offsets.numel() - 1
    if out.size(0) != n_mix:
        raise ValueError("out must have one row per mixture")
    ctx.check(load_library().fastid_mix(ctx.handle, s, _ld(src), n_words, o, n_mix, d, _ld(out), nm,
                                        _stream_ptr(stream)))


def fastid_load_refs(ctx: Context, packed: torch.Tensor, n_loci: int, flags: int = 0, stream=None) -> RefDB:
    p = _dev(packed, torch.int64, "packed", 2)
    h = _P()
    ctx.check(load_library().fastid_load_refs(ctx.handle, p, packed.size(0), n_loci, _ld(packed), flags,
                                              ctypes.byref(h), _stream_ptr(stream)))
    return RefDB(ctx, h, packed.size(0), n_loci, flags)


def fastid_refs_view(ctx: Context, db: RefDB, r_begin: int, n_refs: int) -> RefDB:
    """Rows [r_begin, r_begin + n_refs) of db as a database of their own
    (shared memory; r_begin a multiple of VIEW_ALIGN).  The view keeps a
    reference to db; close the view before db."""
    h = _P()
    ctx.check(load_library().fastid_refs_view(ctx.handle, db.handle, r_begin, n_refs, ctypes.byref(h)))
    v = RefDB(ctx, h, n_refs, db.n_loci, db.flags)
    v.parent, v.r_begin = db, r_begin
    return v


def fastid_topk_fold(ctx: Context, run_scores: torch.Tensor, run_idx: torch.Tensor, blk_scores: torch.Tensor,
                     blk_idx: torch.Tensor, ref_offset: int, stream=None) -> None:
    """Merge blk's [n_q][k] lists (indices + ref_offset) into run's, in place."""
    rs = _dev(run_scores, torch.int32, "run_scores", 2)
    ri = _dev(run_idx, torch.int64, "run_idx", 2)
    bs = _dev(blk_scores, torch.int32, "blk_scores", 2)
    bi = _dev(blk_idx, torch.int64, "blk_idx", 2)
    n_q, k = run_scores.shape
    for t in (run_idx, blk_scores, blk_idx):
        if tuple(t.shape) != (n_q, k):
            raise ValueError("fold lists must all be [n_q][k]")
    for t in (run_scores, run_idx, blk_scores, blk_idx):
        if n_q > 1 and t.stride(0) != k:
            raise ValueError("fold lists must be contiguous [n_q][k]")
    ctx.check(load_library().fastid_topk_fold(ctx.handle, rs, ri, bs, bi, ref_offset, n_q, k, _stream_ptr(stream)))


def fastid_topk_accumulate(ctx: Context, db: RefDB, ref_offset: int, queries: torch.Tensor, modes: torch.Tensor,
                           k: int, threshold: int, run_scores: torch.Tensor, run_idx: torch.Tensor,
                           stream=None) -> None:
    """fastid_topk against db merged into run's [n_q][k] lists (indices +
    ref_offset), in place."""
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    s = _dev(run_scores, torch.int32, "run_scores", 2)
    i = _dev(run_idx, torch.int64, "run_idx", 2)
    n_q = queries.size(0)
    if modes.numel() != n_q or tuple(run_scores.shape) != (n_q, k) or tuple(run_idx.shape) != (n_q, k):
        raise ValueError("modes / running lists do not match n_q x k")
    for t in (run_scores, run_idx):
        if n_q > 1 and t.stride(0) != k:
            raise ValueError("running lists must be contiguous [n_q][k]")
    ctx.check(load_library().fastid_topk_accumulate(ctx.handle, db.handle, ref_offset, q, _ld(queries), n_q, m, k,
                                                    threshold, s, i, _stream_ptr(stream)))


def fastid_scores(ctx: Context, db: RefDB, queries: torch.Tensor, modes: torch.Tensor, out: torch.Tensor,
                  stream=None) -> None:
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    if out.dtype == torch.int16:
        ob = 2
    elif out.dtype == torch.int32:
        ob = 4
    else:
        raise TypeError("out must be int16 (uint16 scores) or int32 (uint32 scores)")
    o = _dev(out, out.dtype, "out", 2)
    n_q = queries.size(0)
    if modes.numel() != n_q or out.size(0) != n_q:
        raise ValueError("modes/out must have one entry/row per query")
    ctx.check(load_library().fastid_scores(ctx.handle, db.handle, q, _ld(queries), n_q, m, o, ob, _ld(out),
                                           _stream_ptr(stream)))


def fastid_topk(ctx: Context, db: RefDB, queries: torch.Tensor, modes: torch.Tensor, k: int,
                threshold: int, out_scores: torch.Tensor, out_idx: torch.Tensor, stream=None) -> None:
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    s = _dev(out_scores, torch.int32, "out_scores", 2)
    i = _dev(out_idx, torch.int64, "out_idx", 2)
    n_q = queries.size(0)
    if modes.numel() != n_q or tuple(out_scores.shape) != (n_q, k) or tuple(out_idx.shape) != (n_q, k):
        raise ValueError("modes / outputs do not match n_q x k")
    ctx.check(load_library().fastid_topk(ctx.handle, db.handle, q, _ld(queries), n_q, m, k, threshold, s, i,
                                         _stream_ptr(stream)))


def fastid_topk_streamed(ctx: Context, refs_host: torch.Tensor, n_loci: int, flags: int, block_refs: int,
                         queries: torch.Tensor, modes: torch.Tensor, k: int, threshold: int,
                         out_scores: torch.Tensor, out_idx: torch.Tensor, stream=None) -> None:
    """refs_host: int64 [n_refs][ld_words] packed references in host memory
    (pin it for overlapped copies); it must outlive the stream's work."""
    if not isinstance(refs_host, torch.Tensor) or refs_host.is_cuda or refs_host.dtype != torch.int64:
        raise TypeError("refs_host must be a host int64 torch.Tensor")
    if refs_host.dim() != 2 or refs_host.stride(1) != 1:
        raise ValueError("refs_host must be 2-D with contiguous rows")
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    s = _dev(out_scores, torch.int32, "out_scores", 2)
    i = _dev(out_idx, torch.int64, "out_idx", 2)
    n_q = queries.size(0)
    if modes.numel() != n_q or tuple(out_scores.shape) != (n_q, k) or tuple(out_idx.shape) != (n_q, k):
        raise ValueError("modes / outputs do not match n_q x k")
    ctx.check(load_library().fastid_topk_streamed(ctx.handle, refs_host.data_ptr(), refs_host.size(0), n_loci,
                                                  _ld(refs_host), flags, block_refs, q, _ld(queries), n_q, m, k,
                                                  threshold, s, i, _stream_ptr(stream)))


def fastid_compare_streamed(ctx: Context, refs_host: torch.Tensor, n_loci: int, flags: int, block_refs: int,
                            queries: torch.Tensor, modes: torch.Tensor, threshold: int, hit_q: torch.Tensor,
                            hit_r: torch.Tensor, hit_score: torch.Tensor, hit_count: torch.Tensor,
                            stream=None) -> None:
    """Hit list over packed references in host memory (see fastid_topk_streamed)."""
    if not isinstance(refs_host, torch.Tensor) or refs_host.is_cuda or refs_host.dtype != torch.int64:
        raise TypeError("refs_host must be a host int64 torch.Tensor")
    if refs_host.dim() != 2 or refs_host.stride(1) != 1:
        raise ValueError("refs_host must be 2-D with contiguous rows")
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    hq = _dev(hit_q, torch.int64, "hit_q", 1)
    hr = _dev(hit_r, torch.int64, "hit_r", 1)
    hs = _dev(hit_score, torch.int32, "hit_score", 1)
    hc = _dev(hit_count, torch.int64, "hit_count", 1)
    cap = hit_q.numel()
    if hit_r.numel() != cap or hit_score.numel() != cap:
        raise ValueError("hit buffers differ in length")
    n_q = queries.size(0)
    if modes.numel() != n_q:
        raise ValueError("modes do not match n_q")
    ctx.check(load_library().fastid_compare_streamed(ctx.handle, refs_host.data_ptr(), refs_host.size(0), n_loci,
                                                     _ld(refs_host), flags, block_refs, q, _ld(queries), n_q, m,
                                                     threshold, cap, hq, hr, hs, hc, _stream_ptr(stream)))


def fastid_compare(ctx: Context, db: RefDB, queries: torch.Tensor, modes: torch.Tensor, threshold: int,
                   hit_q: torch.Tensor, hit_r: torch.Tensor, hit_score: torch.Tensor,
                   hit_count: torch.Tensor, stream=None) -> None:
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    hq = _dev(hit_q, torch.int64, "hit_q", 1)
    hr = _dev(hit_r, torch.int64, "hit_r", 1)
    hs = _dev(hit_score, torch.int32, "hit_score", 1)
    hc = _dev(hit_count, torch.int64, "hit_count", 1)
    cap = hit_q.numel()
    if hit_r.numel() != cap or hit_score.numel() != cap:
        raise ValueError("hit buffers differ in length")
    n_q = queries.size(0)
    ctx.check(load_library().fastid_compare(ctx.handle, db.handle, q, _ld(queries), n_q, m, threshold, cap,
                                            hq, hr, hs, hc, _stream_ptr(stream)))


def fastid_topk_noalloc(ctx: Context, db: RefDB, queries: torch.Tensor, modes: torch.Tensor, k: int,
                        threshold: int, out_scores: torch.Tensor, out_idx: torch.Tensor, stream=None) -> None:
    """fastid_topk without device allocation: scratch comes from a fixed array
    of NOALLOC_SCRATCH_BYTES inside the library (see include/fastid.h)."""
    q = _dev(queries, torch.int64, "queries", 2)
    m = _dev(modes, torch.uint8, "modes", 1)
    s = _dev(out_scores, torch.int32, "out_scores", 2)
    i = _dev(out_idx, torch.int64, "out_idx", 2)
    n_q = queries.size(0)
    if modes.numel() != n_q or tuple(out_scores.shape) != (n_q, k) or tuple(out_idx.shape) != (n_q, k):
        raise ValueError("modes / outputs do not match n_q x k")
    ctx.check(load_library().fastid_topk_noalloc(ctx.handle, db.handle, q, _ld(queries), n_q, m, k, threshold,
                                                 s, i, _stream_ptr(stream)))


class FastIDBatch(ctypes.Structure):
    """Mirror of the C struct fastid_batch."""
    _fields_ = [("panel", ctypes.c_int32), ("queries_dev", ctypes.c_void_p), ("ld_q", ctypes.c_int64),
                ("n_q", ctypes.c_int64), ("modes_dev", ctypes.c_void_p), ("out_scores_dev", ctypes.c_void_p),
                ("out_idx_dev", ctypes.c_void_p)]


class Plan:
    """A fastid_plan: fixed panels and batches, reusable runs and graph replays.

    batches: list of (panel, queries int64 [n_q, ld], modes uint8 [n_q],
    out_scores int32 [n_q, k], out_idx int64 [n_q, k]) CUDA tensors.  The
    tensors must stay alive (and at the same addresses) for the plan's life.
    """

    def __init__(self, ctx: Context, dbs, batches, k: int, threshold: int = NO_THRESHOLD,
                 variant: int = VARIANT_AUTO):
        lib = load_library()
        self.ctx, self._lib = ctx, lib
        self._keep = [dbs, batches]
        arr = (FastIDBatch * max(1, len(batches)))()
        for i, (panel, q, m, sc, ix) in enumerate(batches):
            n = q.size(0)
            if n:
                _dev(q, torch.int64, "queries", 2)
                _dev(m, torch.uint8, "modes", 1)
                _dev(sc, torch.int32, "out_scores", 2)
                _dev(ix, torch.int64, "out_idx", 2)
                if tuple(sc.shape) != (n, k) or tuple(ix.shape) != (n, k) or m.numel() != n:
                    raise ValueError("batch outputs must be [n_q, k]")
            arr[i] = FastIDBatch(panel, q.data_ptr() if n else None, _ld(q) if n else dbs[panel].n_loci // 64 + 1,
                                 n, m.data_ptr() if n else None, sc.data_ptr() if n else None,
                                 ix.data_ptr() if n else None)
        self._arr = arr
        handles = (_P * len(dbs))(*[d.handle.value for d in dbs])
        h = _P()
        ctx.check(lib.fastid_plan_create(ctx.handle, handles, len(dbs), arr, len(batches), k, threshold, variant,
                                         ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        self.ctx.check(self._lib.fastid_plan_run(self.handle, _stream_ptr(stream)))

    def capture(self, stream=None):
        self.ctx.check(self._lib.fastid_plan_capture(self.handle, _stream_ptr(stream)))

    def replay(self, stream=None):
        self.ctx.check(self._lib.fastid_plan_replay(self.handle, _stream_ptr(stream)))

    def info(self) -> dict:
        nq, nu, g, v, wb = _I64(), _I64(), _I32(), _I32(), _I64()
        self.ctx.check(self._lib.fastid_plan_info(self.handle, ctypes.byref(nq), ctypes.byref(nu), ctypes.byref(g),
                                                  ctypes.byref(v), ctypes.byref(wb)))
        return {"n_queries": nq.value, "n_units": nu.value, "grid": g.value, "variant": v.value,
                "workspace_bytes": wb.value}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fastid_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
