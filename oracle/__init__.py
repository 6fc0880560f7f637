"""CPU oracle for the FastID all-pairs comparison (arXiv:1707.00516).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports, links or runs anything in this package, and this package imports
nothing from the product.

What it computes, with the passage each function follows:

* ``pack``      Sec. II-A: alleles to unsigned words (locus l -> bit l mod 64
                of word l // 64, least significant bit first).
* ``mix``       Sec. I / II-A: a mixture carries every minor allele of every
                contributor (per-locus OR).
* ``scores``    Eq. 1 and Algorithm 2, per locus on unpacked 0/1 alleles:
                ``une[q, r] = sum_l AND(XOR(R_r[l], Q_q[l]), R_r[l])`` and the
                XOR-only mismatch ``mis[q, r] = sum_l XOR(R_r[l], Q_q[l])``.
* ``select``    per-query choice of the two counts (mode 0 = mismatch,
                mode 1 = Eq. 1).
* ``topk``      the k smallest scores per query ordered by (score, reference
                index), restricted to score <= threshold; empty slots are
                (2^32 - 1, -1).  The paper returns the full matrix (Sec. III-C);
                the reduction is the one it proposes in Sec. IV.
* ``hits``      every (q, r, score) with score <= threshold, in (q, r) order.

The C part (``fastid_oracle.c``) is compiled by ``build()`` with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastid_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

UINT32_MAX = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            lib.oracle_pack.argtypes = [P, i64, i32, i64, P, i64]
            lib.oracle_mix.argtypes = [P, i32, P, i64, P]
            lib.oracle_scores.argtypes = [P, i64, P, i64, i32, P, P, i32]
            lib.oracle_score_pairs.argtypes = [P, P, i32, P, P, i64, P, P, i32]
            lib.oracle_max_threads.restype = i32
            for f in (lib.oracle_pack, lib.oracle_mix, lib.oracle_scores, lib.oracle_score_pairs):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def words_for(n_loci: int) -> int:
    """Number of 64-bit words that hold n_loci bits."""
    return (n_loci + 63) // 64


def pack(alleles: np.ndarray, ld_words: int | None = None) -> np.ndarray:
    """Sec. II-A packing: uint8 [n, N] (0/1) -> uint64 [n, ld_words]."""
    a = np.ascontiguousarray(alleles, dtype=np.uint8)
    n, n_loci = a.shape
    ld = words_for(n_loci) if ld_words is None else int(ld_words)
    if ld < words_for(n_loci):
        raise ValueError("ld_words too small")
    out = np.empty((n, ld), dtype=np.uint64)
    _load().oracle_pack(_ptr(a), n, n_loci, n_loci, _ptr(out), ld)
    return out


def mix(src: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Per-locus OR of the source rows offsets[m]..offsets[m+1]-1."""
    s = np.ascontiguousarray(src, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    n_mix = off.shape[0] - 1
    out = np.empty((n_mix, s.shape[1]), dtype=np.uint8)
    _load().oracle_mix(_ptr(s), s.shape[1], _ptr(off), n_mix, _ptr(out))
    return out


def scores(R: np.ndarray, Q: np.ndarray, threads: int = 0):
    """(mis, une), each uint32 [n_q, n_r], per Eq. 1 / Algorithm 2."""
    R = np.ascontiguousarray(R, dtype=np.uint8)
    Q = np.ascontiguousarray(Q, dtype=np.uint8)
    if R.shape[1] != Q.shape[1]:
        raise ValueError("loci counts differ")
    mis = np.empty((Q.shape[0], R.shape[0]), dtype=np.uint32)
    une = np.empty_like(mis)
    _load().oracle_scores(_ptr(R), R.shape[0], _ptr(Q), Q.shape[0], R.shape[1],
                          _ptr(mis), _ptr(une), threads)
    return mis, une


def score_pairs(R: np.ndarray, Q: np.ndarray, qi, ri, threads: int = 0):
    """(mis, une) for the pairs (Q[qi[p]], R[ri[p]])."""
    R = np.ascontiguousarray(R, dtype=np.uint8)
    Q = np.ascontiguousarray(Q, dtype=np.uint8)
    qi = np.ascontiguousarray(qi, dtype=np.int64)
    ri = np.ascontiguousarray(ri, dtype=np.int64)
    mis = np.empty(qi.shape[0], dtype=np.uint32)
    une = np.empty_like(mis)
    _load().oracle_score_pairs(_ptr(R), _ptr(Q), R.shape[1], _ptr(qi), _ptr(ri), qi.shape[0],
                               _ptr(mis), _ptr(une), threads)
    return mis, une


def select(mis: np.ndarray, une: np.ndarray, modes: np.ndarray) -> np.ndarray:
    """Per query: mode 0 -> mismatch count, mode 1 -> Eq. 1 count."""
    m = np.asarray(modes).reshape(-1, *([1] * (mis.ndim - 1))).astype(bool)
    return np.where(m, une, mis).astype(np.uint32)


def topk(score_rows: np.ndarray, k: int, threshold: int = UINT32_MAX, ref_ids=None):
    """Per row: the k smallest (score, ref id) with score <= threshold.

    score_rows: uint32 [n_q, n_r]; ref_ids: int64 [n_r] global indices of the
    columns (default 0..n_r-1).  Returns (scores uint32 [n_q, k], idx int64
    [n_q, k]) with unused slots (2^32 - 1, -1).
    """
    s = np.asarray(score_rows, dtype=np.uint32)
    n_q, n_r = s.shape
    ids = np.arange(n_r, dtype=np.int64) if ref_ids is None else np.asarray(ref_ids, np.int64)
    out_s = np.full((n_q, k), UINT32_MAX, dtype=np.uint32)
    out_i = np.full((n_q, k), -1, dtype=np.int64)
    for q in range(n_q):
        keep = np.nonzero(s[q] <= threshold)[0]
        order = keep[np.lexsort((ids[keep], s[q, keep]))][:k]
        out_s[q, :order.size] = s[q, order]
        out_i[q, :order.size] = ids[order]
    return out_s, out_i


def hits(score_rows: np.ndarray, threshold: int, ref_ids=None, query_ids=None):
    """All (q, r, score) with score <= threshold, sorted by (q, r).

    Returns (q int64 [h], r int64 [h], score uint32 [h]).
    """
    s = np.asarray(score_rows, dtype=np.uint32)
    qq, rr = np.nonzero(s <= threshold)
    sc = s[qq, rr]
    qid = qq.astype(np.int64) if query_ids is None else np.asarray(query_ids, np.int64)[qq]
    rid = rr.astype(np.int64) if ref_ids is None else np.asarray(ref_ids, np.int64)[rr]
    order = np.lexsort((rid, qid))
    return qid[order], rid[order], sc[order]


def mixture_vs_mixture(known: np.ndarray, unknown: np.ndarray, threads: int = 0):
    """Mixture-to-mixture comparison.  Sec. I names comparing mixtures with
    mixtures as a use of the method but gives no score; the reading taken
    here applies Eq. 1 with the known mixture K in the reference role:

        containment[u, k] = sum_l AND(XOR(K_l, U_l), K_l)  (= popc(K AND NOT U))

    the known mixture's minor alleles the unknown mixture U does not carry --
    0 exactly when K's allele set lies inside U's, as it does whenever every
    contributor of K also contributed to U -- and the symmetric
    mismatch[u, k] = sum_l XOR(K_l, U_l) = containment(K, U) + containment(U, K).
    known uint8 [n_k, N], unknown uint8 [n_u, N] (0/1, mixtures or
    individuals).  Returns (containment, mismatch), uint32 [n_u, n_k]."""
    mis, une = scores(known, unknown, threads)
    return une, mis
