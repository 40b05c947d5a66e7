"""Pins for the oracle SpMM (CPU only): hand example, brute force, special
cases, 0% sparsity against dense GEMM, skip semantics and the normaliser."""
import json
import os

import numpy as np
import pytest

from oracle.spmm import spmm, spmm_int, normalized_error, flops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_example_product():
    with open(os.path.join(GOLDEN, "hand_example.json")) as f:
        g = json.load(f)
    C, D = spmm(np.array(g["A"], np.float32), np.array(g["B"], np.float32))
    assert C.tolist() == g["C"]


@pytest.mark.parametrize("M", [1, 2, 3, 5, 9, 17, 33])
@pytest.mark.parametrize("s", [0.0, 0.5, 0.9, 1.0])
def test_brute_force_small_integers(M, s):
    # small integer values: every product and partial sum is exact in FP64,
    # so the definition must equal the dense matrix product exactly
    rng = np.random.default_rng(M)
    K, N = (M * 7) % 11 + 1, (M * 5) % 9 + 1
    A = rng.integers(-4, 5, size=(M, K)).astype(np.float32)
    A[rng.random((M, K)) < s] = 0
    B = rng.integers(-4, 5, size=(K, N)).astype(np.float32)
    C, D = spmm(A, B)
    ref = [[sum(float(A[i, k]) * float(B[k, j]) for k in range(K)) for j in range(N)]
           for i in range(M)]
    assert C.tolist() == ref
    assert np.array_equal(D, np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))


@pytest.mark.parametrize("s", [0.0, 0.7, 0.95])
def test_against_dense_gemm_float(s):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 70)).astype(np.float32)
    A[rng.random(A.shape) < s] = 0
    B = rng.standard_normal((70, 23)).astype(np.float32)
    C, D = spmm(A, B)
    dense = A.astype(np.float64) @ B.astype(np.float64)
    assert normalized_error(C, dense, D) < 1e-14


def test_special_cases():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((6, 5)).astype(np.float32)
    Z = np.zeros((4, 6), np.float32)
    C, _ = spmm(Z, B)
    assert np.all(C == 0)
    C0 = rng.standard_normal((4, 5)).astype(np.float32)
    C, _ = spmm(Z, B, C0=C0)
    assert np.array_equal(C, C0.astype(np.float64))
    C, _ = spmm(np.eye(6, dtype=np.float32), B)
    assert np.array_equal(C, B.astype(np.float64))
    perm = rng.permutation(6)
    Pm = np.eye(6, dtype=np.float32)[perm]
    C, _ = spmm(Pm, B)
    assert np.array_equal(C, B[perm].astype(np.float64))
    e = np.array([-3, 0, 1, 5, 2, -1])
    Dg = np.diag(np.float32(2.0) ** e).astype(np.float32)
    C, _ = spmm(Dg, B)
    assert np.array_equal(C, (B.astype(np.float64) * (2.0 ** e)[:, None]))


def test_skip_semantics_with_nonfinite_b():
    # a zero of A skips its row entirely (Sec. 3): Inf in the untouched B row
    # must not leak into C, unlike a dense product (0 * Inf = NaN)
    A = np.array([[1.0, 0.0], [0.0, 2.0]], np.float32)
    B = np.array([[np.inf, 1.0], [3.0, 4.0]], np.float32)
    C, _ = spmm(A, B)
    assert C.tolist() == [[np.inf, 1.0], [6.0, 8.0]]
    with np.errstate(invalid="ignore"):
        assert np.isnan((A.astype(np.float64) @ B.astype(np.float64))[1, 0])


def test_rows_cols_subset_matches_full():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((20, 30)).astype(np.float32)
    A[rng.random(A.shape) < 0.8] = 0
    B = rng.standard_normal((30, 12)).astype(np.float32)
    C, D = spmm(A, B)
    rows, cols = [19, 0, 7], [11, 3]
    Cs, Ds = spmm(A, B, rows, cols)
    assert np.array_equal(Cs, C[np.ix_(rows, cols)]) and np.array_equal(Ds, D[np.ix_(rows, cols)])


def test_int_path():
    A = np.ones((5, 9), np.int8)
    A[1, :4] = 0
    A[3] = 0
    B = np.ones((9, 4), np.int8)
    C = spmm_int(A, B)
    assert C[:, 0].tolist() == [9, 5, 9, 0, 9]          # row nnz
    rng = np.random.default_rng(1)
    Aq = rng.integers(-127, 128, size=(13, 21)).astype(np.int8)
    Aq[rng.random(Aq.shape) < 0.6] = 0
    Bq = rng.integers(-127, 128, size=(21, 7)).astype(np.int8)
    assert np.array_equal(spmm_int(Aq, Bq), Aq.astype(np.int64) @ Bq.astype(np.int64))
    with pytest.raises(OverflowError):
        big = np.full((1, 140000), 127, np.int8)
        spmm_int(big, np.full((140000, 1), 127, np.int8))


def test_normalized_error_zero_denominator():
    assert normalized_error([[0.0, 1.0]], [[-0.0, 1.0]], [[0.0, 2.0]]) == 0.0
    assert normalized_error([[1e-30, 1.0]], [[0.0, 1.0]], [[0.0, 2.0]]) == float("inf")
    assert normalized_error([[1.5]], [[1.0]], [[2.0]]) == 0.25


def _count_macs(A, N):
    """Multiply-accumulates of the row-skipping product, counted one by one:
    every (i, k, j) with A[i, k] != 0 is one product a_ik * b_kj added into
    c_ij (Sec. 3); rows with a zero a_ik are skipped and cost nothing."""
    count = 0
    M, K = len(A), len(A[0])
    for i in range(M):
        for k in range(K):
            if A[i][k] != 0:
                for _ in range(N):
                    count += 1
    return count


def test_flops_against_counted_macs():
    # Sec. 5 counts one FLOP per multiply-accumulate (nnz * N); the metric
    # here counts the multiply and the add (2 * nnz * N).  The hand example
    # of tests/golden has 4 nonzeros and N = 2: 8 products, 16 flops.
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_example.json")) as f:
        ex = json.load(f)
    A = ex["A"]
    N = len(ex["B"][0])
    nnz = sum(1 for r in A for x in r if x != 0)
    assert _count_macs(A, N) == 8
    assert flops(nnz, N) == 2 * _count_macs(A, N) == 16
    # random shapes, including an all-zero row and an all-zero matrix
    rng = np.random.default_rng(11)
    for M, K, N in [(5, 7, 3), (1, 9, 4), (6, 2, 1), (3, 3, 5)]:
        Ar = np.where(rng.random((M, K)) < 0.4, rng.standard_normal((M, K)), 0.0)
        Ar[0] = 0.0
        nz = int(np.count_nonzero(Ar))
        assert flops(nz, N) == 2 * _count_macs(Ar.tolist(), N)
    assert flops(0, 17) == 2 * _count_macs([[0.0, 0.0]], 17) == 0
