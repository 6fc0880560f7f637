"""The seeded input generator: published SplitMix64 values, determinism,
row independence, allele frequencies and recipe structure."""
import numpy as np

import gen


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0 (Steele, Lea, Flood 2014): the first three
    outputs of the sequence x_{i+1} = x_i + gamma are these constants."""
    exp = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    x = 0
    for e in exp:
        assert gen.splitmix64_scalar(x) == e
        x = (x + gen.GAMMA) & gen.MASK64
    v = gen.splitmix64(np.array([0, gen.GAMMA, (2 * gen.GAMMA) & gen.MASK64], np.uint64))
    assert [int(t) for t in v] == exp


def test_draw32_scalar_vs_vector():
    key = gen.stream_key(123, 4)
    for row, locus in ((0, 0), (5, 77), (19_999_999, 16383)):
        z = gen.splitmix64_scalar(key ^ ((row << 24) | locus)) >> 32
        assert int(gen.draw32(123, 4, [row], [locus])[0, 0]) == z


def test_rows_are_independent_of_batch():
    thr = gen.maf_thresholds(1, 333)
    a = gen.allele_rows(1, gen.STREAM_DB, np.array([3, 9, 1_000_000]), thr)
    for i, r in enumerate([3, 9, 1_000_000]):
        assert np.array_equal(a[i], gen.allele_rows(1, gen.STREAM_DB, [r], thr)[0])
    assert np.array_equal(a, gen.allele_rows(1, gen.STREAM_DB, np.array([3, 9, 1_000_000]), thr))


def test_thresholds_and_frequencies():
    thr = gen.maf_thresholds(2, 4096)
    P = thr.astype(np.float64) / 2 ** 32
    # p in [0.05, 0.5] -> P = 1 - (1-p)^2 in [0.0975, 0.75]
    assert P.min() >= 0.0975 - 1e-9 and P.max() <= 0.75
    a = gen.allele_rows(2, gen.STREAM_DB, np.arange(400), thr)
    freq = a.mean(0)
    # binomial(400, P) per locus: mean over loci within a few standard errors
    assert abs(freq.mean() - P.mean()) < 0.01
    assert np.corrcoef(freq, P)[0, 1] > 0.9


def test_recipes():
    r = gen.recipe_c1()
    assert r.n_queries == 64 and r.n_refs == 10_000 and r.n_loci == 1024
    assert sum(len(r.planted(q)) for q in range(64)) == 8
    r3 = gen.recipe_c3(n_refs=1000, n_q=64)
    assert r3.n_queries == 64
    assert np.all(r3.modes[:32] == gen.MODE_MISMATCH) and np.all(r3.modes[32:] == gen.MODE_UNEXPLAINED)
    sizes = np.diff(r3.offsets)
    assert np.all(sizes[:32] == 1) and np.all((sizes[32:] >= 2) & (sizes[32:] <= 5))
    assert all(len(r3.planted(q)) >= 1 for q in range(32, 64))
    s = gen.log_uniform_sizes(1000, 1, 512, 5, 1)
    assert s.min() >= 1 and s.max() <= 512
