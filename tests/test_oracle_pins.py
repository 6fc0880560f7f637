"""Pins for the CPU oracle: each test checks it against something other than
itself -- the paper's printed example, hand-worked instances of Eq. 1,
closed forms over all profiles of a few loci, a library matmul, a library
bit-packer, and invariants the method guarantees."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from gen import (MODE_MISMATCH, MODE_UNEXPLAINED, STREAM_DB, allele_rows, maf_thresholds,
                 recipe_individuals, recipe_mixtures, source_alleles)


def _golden_kv(path):
    kv = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            k, *v = line.split()
            kv[k] = v
    return kv


def _profile(s):
    return np.array([int(c) for c in s], dtype=np.uint8)


# --- packing (Sec. II-A) -----------------------------------------------------

def test_worked_example_packing(golden_dir):
    kv = _golden_kv(os.path.join(golden_dir, "worked_example.txt"))
    n = int(kv["n_loci"][0])
    a = np.zeros((1, n), np.uint8)
    a[0, [int(x) for x in kv["set_loci"]]] = 1
    w = oracle.pack(a)
    assert w.shape == (1, 1)
    low32 = int(w[0, 0]) & 0xFFFFFFFF
    assert low32 == int(kv["word_hex"][0], 16) == int(kv["word_dec"][0])
    assert int(w[0, 0]) >> 32 == 0
    # popcount of the profile = Eq. 1 of the profile against an empty query
    _, une = oracle.scores(a, np.zeros_like(a))
    assert une[0, 0] == int(kv["popcount"][0])


def test_512_snps_is_16_u32_words(golden_dir):
    kv = _golden_kv(os.path.join(golden_dir, "worked_example.txt"))
    a = np.ones((1, 512), np.uint8)
    w = oracle.pack(a)
    assert w.view(np.uint32).shape[1] == int(kv["snps_512_u32_words"][0])
    assert np.all(w.view(np.uint32) == 0xFFFFFFFF)


@pytest.mark.parametrize("n_loci", [1, 31, 32, 63, 64, 65, 200, 1024, 1031])
def test_pack_matches_numpy_packbits(n_loci):
    rng = np.random.default_rng(n_loci)
    a = (rng.random((37, n_loci)) < 0.4).astype(np.uint8)
    ld = oracle.words_for(n_loci) + 2  # padded rows
    w = oracle.pack(a, ld_words=ld)
    ref = np.zeros((37, ld * 8), np.uint8)
    pb = np.packbits(a, axis=1, bitorder="little")
    ref[:, :pb.shape[1]] = pb
    assert np.array_equal(w.view(np.uint8), ref)


# --- Eq. 1 and the XOR mismatch ----------------------------------------------

def test_eq1_hand_worked(golden_dir):
    for line in open(os.path.join(golden_dir, "eq1_hand.txt")):
        line = line.split("#", 1)[0].split(";", 1)[0].strip()
        if not line:
            continue
        r, q, mis, une = line.split()
        m, u = oracle.scores(_profile(r)[None], _profile(q)[None])
        assert (m[0, 0], u[0, 0]) == (int(mis), int(une)), line


@pytest.mark.parametrize("n_loci", [1, 2, 3, 5, 7])
def test_closed_forms_over_all_profiles(n_loci):
    """Over all 4^N ordered pairs of N-locus profiles: at each locus half the
    pairs differ and a quarter have (R, Q) = (1, 0), so
        sum mis = N 2^(2N-1),  sum une = N 2^(2N-2),
        #{une = j} = C(N, j) 3^(N-j),  #{mis = j} = C(N, j) 2^N."""
    P = np.array(list(itertools.product([0, 1], repeat=n_loci)), dtype=np.uint8)
    mis, une = oracle.scores(P, P)
    N = n_loci
    assert int(mis.astype(np.int64).sum()) == N * 2 ** (2 * N - 1)
    assert int(une.astype(np.int64).sum()) == N * 2 ** (2 * N - 2)
    hu = np.bincount(une.ravel(), minlength=N + 1)
    hm = np.bincount(mis.ravel(), minlength=N + 1)
    for j in range(N + 1):
        assert hu[j] == math.comb(N, j) * 3 ** (N - j)
        assert hm[j] == math.comb(N, j) * 2 ** N


def test_eq1_operand_is_the_reference():
    """une[q, r] counts alleles of reference r missing from query q: an
    all-ones query explains every reference, an all-zero query explains
    none; swapping the operands gives the other count."""
    rng = np.random.default_rng(7)
    R = (rng.random((9, 50)) < 0.5).astype(np.uint8)
    ones, zeros = np.ones((1, 50), np.uint8), np.zeros((1, 50), np.uint8)
    _, u1 = oracle.scores(R, ones)
    _, u0 = oracle.scores(R, zeros)
    assert np.all(u1 == 0)
    assert np.array_equal(u0[0], R.sum(1))


def test_against_torch_int64_matmul():
    """For 0/1 matrices G = R Q^T (library matmul); mis = |R| + |Q| - 2G and
    une = |R| - G."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    for n_loci in (1, 63, 64, 129, 777):
        R = (rng.random((41, n_loci)) < rng.random()).astype(np.uint8)
        Q = (rng.random((23, n_loci)) < rng.random()).astype(np.uint8)
        mis, une = oracle.scores(R, Q)
        tR = torch.from_numpy(R.astype(np.int64))
        tQ = torch.from_numpy(Q.astype(np.int64))
        G = (tQ @ tR.T).numpy()
        nR, nQ = R.sum(1).astype(np.int64), Q.sum(1).astype(np.int64)
        assert np.array_equal(mis, nR[None, :] + nQ[:, None] - 2 * G)
        assert np.array_equal(une, nR[None, :] - G)


def test_invariants_on_generated_profiles():
    thr = maf_thresholds(5, 300)
    A = allele_rows(5, STREAM_DB, np.arange(40), thr)
    mis, une = oracle.scores(A, A)
    assert np.all(np.diag(mis) == 0) and np.all(np.diag(une) == 0)   # self score 0
    assert np.array_equal(mis, mis.T)                                 # XOR symmetry
    assert np.array_equal(mis, une + une.T)                           # mis = une(R,Q)+une(Q,R)
    # popc(R & ~M) = |R| - popc(R & M)
    G = A.astype(np.int64) @ A.astype(np.int64).T
    assert np.array_equal(une.T, A.sum(1)[:, None] - G)


def test_score_pairs_matches_full():
    rng = np.random.default_rng(3)
    R = (rng.random((30, 70)) < 0.3).astype(np.uint8)
    Q = (rng.random((12, 70)) < 0.6).astype(np.uint8)
    mis, une = oracle.scores(R, Q)
    qi = rng.integers(0, 12, 200)
    ri = rng.integers(0, 30, 200)
    pm, pu = oracle.score_pairs(R, Q, qi, ri)
    assert np.array_equal(pm, mis[qi, ri]) and np.array_equal(pu, une[qi, ri])


# --- mixtures -----------------------------------------------------------------

def test_mix_is_union():
    rng = np.random.default_rng(4)
    src = (rng.random((10, 90)) < 0.2).astype(np.uint8)
    off = np.array([0, 1, 4, 4 + 3, 10], np.int32)
    m = oracle.mix(src, off)
    for i in range(4):
        assert np.array_equal(m[i], np.max(src[off[i]:off[i + 1]], axis=0))


def test_planted_recovery():
    """Planted database copies score 0 (mismatch); every database contributor
    of a mixture scores 0 (Eq. 1) against it."""
    n_refs, n_loci = 500, 256
    thr = maf_thresholds(21, n_loci)
    db = allele_rows(21, STREAM_DB, np.arange(n_refs), thr)
    ri = recipe_individuals(16, n_refs, n_loci, 21, n_planted=5)
    rm = recipe_mixtures(16, n_refs, n_loci, 21, 2, 5)
    for rec, mode in ((ri, MODE_MISMATCH), (rm, MODE_UNEXPLAINED)):
        q = oracle.mix(source_alleles(rec, thr), rec.offsets)
        mis, une = oracle.scores(db, q)
        s = oracle.select(mis, une, rec.modes)
        assert np.all(rec.modes == mode)
        n_planted = 0
        for j in range(rec.n_queries):
            for r in rec.planted(j):
                assert s[j, r] == 0
                n_planted += 1
        assert n_planted >= 5
        # a random reference is essentially never a perfect match
        assert np.mean(s == 0) < 0.05


# --- top-k and hits ------------------------------------------------------------

def test_topk_ties_and_threshold():
    s = np.array([[5, 3, 3, 9, 0, 3],
                  [7, 7, 7, 7, 7, 7],
                  [1, 2, 3, 4, 5, 6]], dtype=np.uint32)
    sc, ix = oracle.topk(s, 4)
    assert ix.tolist() == [[4, 1, 2, 5], [0, 1, 2, 3], [0, 1, 2, 3]]
    assert sc.tolist() == [[0, 3, 3, 3], [7, 7, 7, 7], [1, 2, 3, 4]]
    sc, ix = oracle.topk(s, 4, threshold=2)
    assert ix.tolist() == [[4, -1, -1, -1], [-1] * 4, [0, 1, -1, -1]]
    assert sc[0].tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]
    # k larger than the number of references
    sc, ix = oracle.topk(s[:, :2], 3)
    assert ix.tolist() == [[1, 0, -1], [0, 1, -1], [0, 1, -1]]


def test_topk_against_python_sorted():
    rng = np.random.default_rng(9)
    s = rng.integers(0, 6, size=(20, 50)).astype(np.uint32)
    ids = rng.permutation(1000)[:50].astype(np.int64)
    for k, T in ((1, 0xFFFFFFFF), (7, 0xFFFFFFFF), (16, 2), (60, 3)):
        sc, ix = oracle.topk(s, k, T, ref_ids=ids)
        for q in range(20):
            exp = sorted((int(s[q, j]), int(ids[j])) for j in range(50) if s[q, j] <= T)[:k]
            exp += [(0xFFFFFFFF, -1)] * (k - len(exp))
            assert list(zip(sc[q].tolist(), ix[q].tolist())) == exp


def test_hits_against_python():
    rng = np.random.default_rng(10)
    s = rng.integers(0, 8, size=(9, 40)).astype(np.uint32)
    q, r, v = oracle.hits(s, 1)
    exp = [(a, b, int(s[a, b])) for a in range(9) for b in range(40) if s[a, b] <= 1]
    assert list(zip(q.tolist(), r.tolist(), v.tolist())) == exp


# --- mixture to mixture (Sec. I; Eq. 1 with a known mixture as reference) ----

def test_mixture_pairs_hand_worked(golden_dir):
    for line in open(os.path.join(golden_dir, "mixture_pairs.txt")):
        line = line.split("#", 1)[0].split(";", 1)[0].strip()
        if not line:
            continue
        k, u, mis, cont = line.split()
        c, m = oracle.mixture_vs_mixture(_profile(k)[None], _profile(u)[None])
        assert (m[0, 0], c[0, 0]) == (int(mis), int(cont)), line


def test_mixture_containment_by_contributor_sets():
    """Brute force over every pair of contributor subsets of a small pool:
    whenever K's contributors are a subset of U's the containment score is 0;
    the mismatch is the two one-sided scores' sum."""
    rng = np.random.default_rng(77)
    pool = (rng.random((5, 40)) < 0.3).astype(np.uint8)
    subsets = [s for n in range(1, 6) for s in itertools.combinations(range(5), n)]
    mixes = np.stack([np.bitwise_or.reduce(pool[list(s)], axis=0) for s in subsets])
    cont, mis = oracle.mixture_vs_mixture(mixes, mixes)
    for iu, su in enumerate(subsets):
        for ik, sk in enumerate(subsets):
            if set(sk) <= set(su):
                assert cont[iu, ik] == 0
            assert mis[iu, ik] == cont[iu, ik] + cont[ik, iu]
            # brute force over loci
            assert cont[iu, ik] == int(np.sum((mixes[ik] == 1) & (mixes[iu] == 0)))
