"""The serving and batched workloads (no GPU): the generators produce the
stated recipe -- Poisson arrivals at the configured rate, request sizes
log-uniform on 1-256 with mixtures of 1-5 contributors (one contributor is an
individual query in mismatch mode), and 256 batches of 1-512 queries with the
loci panel drawn uniformly -- and the same inputs for the same seed."""
import numpy as np

import bench
import gen


def test_serving_requests_follow_the_recipe():
    w = dict(bench.WORKLOADS["c5"])
    seed = gen.config_seed(w["cfg"])
    horizon = 20.0
    arrivals, sizes, rec = bench.c5_requests(w, seed, horizon)
    n = arrivals.size
    expect = w["rate"] * horizon
    assert abs(n - expect) < 5 * np.sqrt(expect)  # Poisson count
    assert np.all(np.diff(arrivals) >= 0) and 0 <= arrivals[0] and arrivals[-1] < horizon
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert abs(gaps.mean() * w["rate"] - 1) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05  # exponential gaps: coefficient of variation 1
    assert sizes.min() >= 1 and sizes.max() <= 256 and sizes.size == n
    # log-uniform: P(size <= s) = ln(s + 1) / ln(257)
    for s in (1, 15, 63):
        assert abs(np.mean(sizes <= s) - np.log(s + 1) / np.log(257)) < 0.03
    contrib = np.diff(rec.offsets)
    assert rec.n_queries == int(sizes.sum())
    assert contrib.min() == 1 and contrib.max() == 5
    for c in range(1, 6):
        assert abs(np.mean(contrib == c) - 0.2) < 0.02
    assert np.array_equal(rec.modes == gen.MODE_MISMATCH, contrib == 1)
    a2, s2, r2 = bench.c5_requests(w, seed, horizon)
    assert np.array_equal(a2, arrivals) and np.array_equal(s2, sizes) and np.array_equal(r2.offsets, rec.offsets)


def test_batched_workload_follows_the_recipe():
    w = bench.WORKLOADS["c4"]
    seed, sizes, panels = bench._c4_batches(w)
    assert len(sizes) == len(panels) == w["n_batches"] == 256
    assert min(sizes) >= 1 and max(sizes) <= 512
    counts = np.bincount(panels, minlength=len(w["panels"]))
    assert counts.size == 4 and np.all(np.abs(counts - 64) < 5 * np.sqrt(256 * 0.25 * 0.75))
    rec = bench._c4_recipe(w, 7, sizes[7], panels[7], seed)
    contrib = np.diff(rec.offsets)
    assert rec.n_queries == sizes[7] and contrib.min() >= 1 and contrib.max() <= 4
    assert np.array_equal(rec.modes == gen.MODE_MISMATCH, contrib == 1)
    assert bench._c4_batches(w) == (seed, sizes, panels)
