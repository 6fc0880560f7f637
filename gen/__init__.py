"""Seeded synthetic SNP profiles for tests and benchmarks.

This module only draws inputs.  It holds none of the comparison arithmetic
(no XOR, AND, popcount, no OR of mixtures): it produces unpacked 0/1 allele
rows and *recipes* that say which rows make up each query.  Both the CUDA
path and the CPU oracle consume what it returns; neither imports the other.

Bits come from a counter-based generator so that any row can be regenerated
on its own, on the host here or on the device by ``gen/gen_gpu.cu``, which
implements the same published function independently:

* ``splitmix64`` is the output function of SplitMix64 (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014): add the
  golden gamma 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds with
  0xBF58476D1CE4E5B9 and 0x94D049BB133111EB and a final xor-shift by 31.
* ``draw32(seed, stream, row, locus)`` =
  ``splitmix64(key(seed, stream) ^ (row << 24 | locus)) >> 32`` with
  ``key(seed, stream) = splitmix64(splitmix64(seed) ^ stream)``.

Population model (the workloads of the paper's Sec. IV, made synthetic):
per-locus minor-allele frequency ``p_l = 0.05 + 0.45 u_l`` with ``u_l``
uniform, genotypes in Hardy-Weinberg proportion, and one bit per locus set
when the genotype carries at least one minor allele, i.e. with probability
``P_l = 1 - (1 - p_l)^2``.  The host turns ``P_l`` into an integer threshold
``thr_l = floor(P_l * 2^32)`` once; a bit is then ``draw32(...) < thr_l``, an
integer test that both sides evaluate identically.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB

# Independent counter streams.
STREAM_MAF = 0      # per-locus allele frequencies (row 0)
STREAM_DB = 1       # reference (known) individuals: row = database index
STREAM_FRESH = 2    # individuals that are not in the database
STREAM_ALLELE_BASE = 16  # free-form allele streams used by tests

LOCUS_BITS = 24
MAX_LOCI = 1 << LOCUS_BITS


def splitmix64_scalar(x: int) -> int:
    """SplitMix64 output function on a Python int (mod 2^64)."""
    z = (x + GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MUL2) & MASK64
    return z ^ (z >> 31)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised SplitMix64 output function on uint64 arrays (wraps mod 2^64)."""
    z = np.asarray(x, dtype=np.uint64) + np.uint64(GAMMA)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MUL1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MUL2)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    return splitmix64_scalar(splitmix64_scalar(seed & MASK64) ^ (stream & MASK64))


def draw32(seed: int, stream: int, rows: np.ndarray, loci: np.ndarray) -> np.ndarray:
    """uint32 draws for every (row, locus) in the outer product rows x loci."""
    key = np.uint64(stream_key(seed, stream))
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1, 1)
    loci = np.asarray(loci, dtype=np.uint64).reshape(1, -1)
    ctr = (rows << np.uint64(LOCUS_BITS)) | loci
    return (splitmix64(key ^ ctr) >> np.uint64(32)).astype(np.uint32)


def maf_thresholds(seed: int, n_loci: int) -> np.ndarray:
    """thr_l = floor(P_l * 2^32), P_l = 1 - (1 - p_l)^2, p_l = 0.05 + 0.45 u_l."""
    if not (0 < n_loci <= MAX_LOCI):
        raise ValueError(f"n_loci must be in (0, {MAX_LOCI}]")
    u = draw32(seed, STREAM_MAF, np.zeros(1, np.uint64), np.arange(n_loci)).astype(np.float64)[0]
    u /= 2.0 ** 32
    p = 0.05 + 0.45 * u
    P = 1.0 - (1.0 - p) ** 2
    return np.floor(P * 2.0 ** 32).astype(np.uint32)


def allele_rows(seed: int, stream: int, rows, thr: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Unpacked 0/1 rows: out[i, l] = draw32(seed, stream, rows[i], l) < thr[l]."""
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    n_loci = thr.shape[0]
    out = np.empty((rows.shape[0], n_loci), dtype=np.uint8)
    loci = np.arange(n_loci)
    for s in range(0, rows.shape[0], chunk):
        d = draw32(seed, stream, rows[s:s + chunk], loci)
        out[s:s + chunk] = (d < thr[None, :]).astype(np.uint8)
    return out


# --------------------------------------------------------------------------
# Query recipes.  A query is a list of sources; a source is a database row
# (STREAM_DB) or a fresh individual (STREAM_FRESH).  An individual query has
# one source; a mixture query has its contributors.  Mode 0 asks for the XOR
# mismatch count, mode 1 for the Eq. 1 unexplained-allele count.
# --------------------------------------------------------------------------

MODE_MISMATCH = 0
MODE_UNEXPLAINED = 1


@dataclass
class QueryRecipe:
    n_refs: int
    n_loci: int
    seed: int
    src_stream: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))  # per source
    src_row: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))     # per source
    offsets: np.ndarray = field(default_factory=lambda: np.zeros(1, np.int32))     # [n_q + 1]
    modes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))       # [n_q]

    @property
    def n_queries(self) -> int:
        return int(self.modes.shape[0])

    @property
    def n_sources(self) -> int:
        return int(self.src_row.shape[0])

    def planted(self, q: int) -> list[int]:
        """Database rows that contribute to query q."""
        a, b = int(self.offsets[q]), int(self.offsets[q + 1])
        return [int(self.src_row[i]) for i in range(a, b) if self.src_stream[i] == STREAM_DB]

    def select(self, qs) -> "QueryRecipe":
        """Sub-recipe with the queries listed in qs (in that order)."""
        qs = np.asarray(qs, dtype=np.int64)
        st, rw, off = [], [], [0]
        for q in qs:
            a, b = int(self.offsets[q]), int(self.offsets[q + 1])
            st.append(self.src_stream[a:b]); rw.append(self.src_row[a:b]); off.append(off[-1] + b - a)
        return QueryRecipe(self.n_refs, self.n_loci, self.seed,
                           np.concatenate(st).astype(np.int32) if st else np.zeros(0, np.int32),
                           np.concatenate(rw).astype(np.int64) if rw else np.zeros(0, np.int64),
                           np.asarray(off, np.int32), self.modes[qs].copy())


def _build(n_refs, n_loci, seed, groups, modes) -> QueryRecipe:
    st = np.array([s for g in groups for (s, _) in g], dtype=np.int32)
    rw = np.array([r for g in groups for (_, r) in g], dtype=np.int64)
    off = np.zeros(len(groups) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(g) for g in groups])
    return QueryRecipe(n_refs, n_loci, seed, st, rw, off, np.asarray(modes, dtype=np.uint8))


def recipe_individuals(n_q: int, n_refs: int, n_loci: int, seed: int, n_planted: int,
                       fresh_base: int = 0) -> QueryRecipe:
    """n_q individuals; n_planted of them (at random positions) are exact database copies."""
    rng = np.random.default_rng([seed, 0xC1])
    pos = set(rng.choice(n_q, size=min(n_planted, n_q), replace=False).tolist())
    db_rows = rng.choice(n_refs, size=len(pos), replace=False) if pos else []
    groups, k = [], 0
    for j in range(n_q):
        if j in pos:
            groups.append([(STREAM_DB, int(db_rows[k]))]); k += 1
        else:
            groups.append([(STREAM_FRESH, fresh_base + j)])
    return _build(n_refs, n_loci, seed, groups, [MODE_MISMATCH] * n_q)


def recipe_mixtures(n_q: int, n_refs: int, n_loci: int, seed: int, cmin: int, cmax: int,
                    fresh_base: int = 1 << 30, salt: int = 0xC2) -> QueryRecipe:
    """n_q mixtures of cmin..cmax contributors.  Contributor 1 is always a
    database row; each further contributor is a database row with probability
    1/2 and a fresh individual otherwise."""
    rng = np.random.default_rng([seed, salt])
    groups, fresh = [], fresh_base
    for _ in range(n_q):
        c = int(rng.integers(cmin, cmax + 1))
        g = [(STREAM_DB, int(rng.integers(0, n_refs)))]
        for _ in range(c - 1):
            if rng.random() < 0.5:
                g.append((STREAM_DB, int(rng.integers(0, n_refs))))
            else:
                g.append((STREAM_FRESH, fresh)); fresh += 1
        groups.append(g)
    return _build(n_refs, n_loci, seed, groups, [MODE_UNEXPLAINED] * n_q)


def concat_recipes(a: QueryRecipe, b: QueryRecipe) -> QueryRecipe:
    assert a.n_refs == b.n_refs and a.n_loci == b.n_loci and a.seed == b.seed
    return QueryRecipe(a.n_refs, a.n_loci, a.seed,
                       np.concatenate([a.src_stream, b.src_stream]).astype(np.int32),
                       np.concatenate([a.src_row, b.src_row]).astype(np.int64),
                       np.concatenate([a.offsets, b.offsets[1:] + a.offsets[-1]]).astype(np.int32),
                       np.concatenate([a.modes, b.modes]).astype(np.uint8))


def source_alleles(recipe: QueryRecipe, thr: np.ndarray) -> np.ndarray:
    """Unpacked allele rows of every source of a recipe, in source order."""
    out = np.empty((recipe.n_sources, thr.shape[0]), dtype=np.uint8)
    for stream in (STREAM_DB, STREAM_FRESH):
        sel = np.nonzero(recipe.src_stream == stream)[0]
        if sel.size:
            out[sel] = allele_rows(recipe.seed, stream, recipe.src_row[sel], thr)
    return out


# --------------------------------------------------------------------------
# Workload configurations (sizes and mixes of the paper's Sec. IV experiments
# plus the batched and serving workloads).  Seeds are 0x170700516 + c.
# --------------------------------------------------------------------------

SEED_BASE = 0x170700516


def config_seed(c: int) -> int:
    return SEED_BASE + c


def recipe_c1(seed: int | None = None) -> QueryRecipe:
    """64 individuals (8 exact database copies) x 10,000 refs, N = 1024."""
    seed = config_seed(1) if seed is None else seed
    return recipe_individuals(64, 10_000, 1024, seed, n_planted=8)


def recipe_c2(seed: int | None = None, n_refs: int = 1_000_000, n_q: int = 2048,
              n_loci: int = 4096) -> QueryRecipe:
    """2048 mixtures of 2-4 contributors (>= 1 planted) x 1M refs, N = 4096."""
    seed = config_seed(2) if seed is None else seed
    return recipe_mixtures(n_q, n_refs, n_loci, seed, 2, 4)


def recipe_c3(seed: int | None = None, n_refs: int = 20_000_000, n_q: int = 2048,
              n_loci: int = 2048) -> QueryRecipe:
    """2048 unknowns (half individuals, half 2-5 person mixtures) x 20M refs, N = 2048."""
    seed = config_seed(3) if seed is None else seed
    half = n_q // 2
    ind = recipe_individuals(half, n_refs, n_loci, seed, n_planted=half // 2)
    mix = recipe_mixtures(n_q - half, n_refs, n_loci, seed, 2, 5)
    return concat_recipes(ind, mix)


def log_uniform_sizes(n: int, lo: int, hi: int, seed: int, salt: int) -> np.ndarray:
    """n integer sizes in [lo, hi], log-uniform: floor(exp(u ln(hi + 1))) clipped to [lo, hi]."""
    rng = np.random.default_rng([seed, salt])
    u = rng.random(n)
    s = np.floor(np.exp(u * np.log(hi + 1))).astype(np.int64)
    return np.clip(s, lo, hi)


# --------------------------------------------------------------------------
# Device generator (gen/gen_gpu.cu), for databases too large for the host.
# --------------------------------------------------------------------------

import ctypes as _ct
import os as _os
import subprocess as _sp

_GEN_DIR = _os.path.dirname(_os.path.abspath(__file__))
_GEN_SRC = _os.path.join(_GEN_DIR, "gen_gpu.cu")
_GEN_LIB = _os.path.join(_GEN_DIR, "libgen_gpu.so")
_gen_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile gen_gpu.cu for sm_103a into gen/libgen_gpu.so."""
    if (not force and _os.path.exists(_GEN_LIB)
            and _os.path.getmtime(_GEN_LIB) >= _os.path.getmtime(_GEN_SRC)):
        return _GEN_LIB
    nvcc = _os.path.join(_os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    tmp = _GEN_LIB + f".tmp{_os.getpid()}"
    _sp.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
             "-shared", _GEN_SRC, "-o", tmp], check=True)
    _os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _gpu():
    global _gen_lib
    if _gen_lib is None:
        if not _os.path.exists(_GEN_LIB):
            raise RuntimeError("gen/libgen_gpu.so is missing: call gen.build_gpu()")
        lib = _ct.CDLL(_GEN_LIB)
        lib.gen_alleles.restype = _ct.c_int
        lib.gen_alleles.argtypes = [_ct.c_uint64, _ct.c_uint64, _ct.c_void_p, _ct.c_int64, _ct.c_int64,
                                    _ct.c_void_p, _ct.c_int32, _ct.c_void_p, _ct.c_int64, _ct.c_void_p]
        _gen_lib = lib
    return _gen_lib


def allele_rows_device(seed: int, stream: int, thr_dev, out_dev, rows_dev=None, row0: int = 0,
                       cuda_stream=None) -> None:
    """Fill the uint8 CUDA tensor out_dev [n_rows, >= n_loci] with allele rows
    row0 .. row0 + n_rows - 1 (or the int64 CUDA tensor rows_dev) of a stream;
    thr_dev is the uint32 threshold table as an int32 CUDA tensor."""
    import torch
    n_rows = out_dev.shape[0]
    n_loci = thr_dev.shape[0]
    st = torch.cuda.current_stream() if cuda_stream is None else cuda_stream
    err = _gpu().gen_alleles(int(seed) & MASK64, int(stream), rows_dev.data_ptr() if rows_dev is not None else None,
                             row0, n_rows, thr_dev.data_ptr(), n_loci, out_dev.data_ptr(),
                             out_dev.stride(0), st.cuda_stream or None)
    if err != 0:
        raise RuntimeError(f"gen_alleles failed with cudaError {err}")
