"""Tensor-core operand encodings, checked on one tile against an integer
matmul, and the roofline microbenchmarks.

The tensor forms rest on two encodings of 0/+1/-1 operands: e4m3 bytes for
tcgen05 kind::f8f6f4 and e2m1 nibbles with unit ue8m0 block scale factors for
kind::mxf4.  One stage of MMAs (128 queries x n references x one 128-byte
K atom) must return D = A B^T exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import peaks  # noqa: E402

CASES = [(False, 256, 128), (True, 224, 256), (True, 256, 256)]


@pytest.mark.parametrize("f4,n,K", CASES)
def test_mma_random_operands(f4, n, K):
    rng = np.random.default_rng(1707 + n + K)
    A = rng.integers(-1, 2, (128, K)).astype(np.int64)
    Bm = rng.integers(0, 2, (n, K)).astype(np.int64)
    D = peaks.mma_check(f4, n, A, Bm)
    assert np.array_equal(D.astype(np.int64), A @ Bm.T)


@pytest.mark.parametrize("f4,n,K", CASES)
def test_mma_extremes(f4, n, K):
    ones_a = np.ones((128, K), np.int64)
    ones_b = np.ones((n, K), np.int64)
    assert np.all(peaks.mma_check(f4, n, ones_a, ones_b) == K)
    assert np.all(peaks.mma_check(f4, n, -ones_a, ones_b) == -K)
    # row i of A and row j of B set on disjoint / shared locus sets
    A = np.zeros((128, K), np.int64)
    Bm = np.zeros((n, K), np.int64)
    for i in range(128):
        A[i, i % K] = 1
        A[i, (i * 7 + 3) % K] = -1
    for j in range(n):
        Bm[j, j % K] = 1
        Bm[j, (j * 5 + 1) % K] = 1
    assert np.array_equal(peaks.mma_check(f4, n, A, Bm).astype(np.int64), A @ Bm.T)


def test_measure_rates_positive():
    m = peaks.measure(target_ms=5.0)
    for key in ("fp8_f8f6f4", "fp4_mxf4_n224", "fp4_mxf4_n256"):
        assert m[key]["tflops"] > 0 and m[key]["flops_per_clk_sm"] > 0
    for key in ("popc", "lop3", "and_popc_add", "harley_seal", "carry_save8"):
        assert m[key]["per_s"] > 0 and m[key]["per_clk_sm"] > 0
    assert m["b1_and_popc"]["bit_macs_per_s"] > 0
