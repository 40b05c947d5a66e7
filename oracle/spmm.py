"""Oracle: the SpMM C = A.B over the nonzeros of A.  Test infrastructure.

Sec. 3 states the method: the outer product of column k of A with row k of B
contributes a[m]*B[k, :] to row m of C, and a row whose a[m] is zero is
skipped.  Summed over k this is exactly the ordinary product restricted to
the nonzeros of A, so the oracle is that definition written out: for each row
i, for each k ascending with A[i, k] != 0, add A[i, k]*B[k, :] to C[i, :].
Alg. 2 loads C before accumulating ("accumulate in-place", Fig. 2), so an
optional initial C is added first.

FP values are accumulated in FP64 (exact products of FP32/BF16 inputs); integer
values in int64.  The normaliser D[i, j] = sum_k |A[i, k]| |B[k, j]| (same k
set) scales the error test max |C - C_ref| / D.
"""
from __future__ import annotations

import numpy as np

__all__ = ["spmm", "spmm_int", "normalized_error", "flops"]


def _index(x, n):
    if x is None:
        return np.arange(n)
    return np.asarray(x, dtype=np.int64)


def spmm(A, B, rows=None, cols=None, C0=None):
    """FP64 C = C0 + A.B restricted to nonzeros of A, for the given output rows
    and columns (default: all).  Returns (C, D) as float64 arrays of shape
    (len(rows), len(cols))."""
    A = np.asarray(A)
    B = np.asarray(B)
    M, K = A.shape
    assert B.shape[0] == K
    rows = _index(rows, M)
    cols = _index(cols, B.shape[1])
    C = np.zeros((rows.size, cols.size), dtype=np.float64)
    D = np.zeros_like(C)
    for out_i, i in enumerate(rows):
        acc = C[out_i]
        nrm = D[out_i]
        for k in np.flatnonzero(A[i] != 0):     # k ascending, zeros skipped
            a = np.float64(A[i, k])
            b = B[k, cols].astype(np.float64)
            acc += a * b
            nrm += abs(a) * np.abs(b)
    if C0 is not None:
        C += np.asarray(C0, dtype=np.float64)[np.ix_(rows, cols)]
    return C, D


def spmm_int(Aq, Bq, rows=None, cols=None, C0=None):
    """Integer C = C0 + A.B with int64 accumulation (INT8 x INT8 -> INT32
    path).  Raises if a result does not fit int32."""
    Aq = np.asarray(Aq)
    Bq = np.asarray(Bq)
    M, K = Aq.shape
    rows = _index(rows, M)
    cols = _index(cols, Bq.shape[1])
    C = np.zeros((rows.size, cols.size), dtype=np.int64)
    for out_i, i in enumerate(rows):
        acc = C[out_i]
        for k in np.flatnonzero(Aq[i] != 0):
            acc += np.int64(Aq[i, k]) * Bq[k, cols].astype(np.int64)
    if C0 is not None:
        C += np.asarray(C0, dtype=np.int64)[np.ix_(rows, cols)]
    lim = np.int64(2 ** 31)
    if C.size and (C.max() >= lim or C.min() < -lim):
        raise OverflowError("integer SpMM result does not fit int32")
    return C


def normalized_error(C, C_ref, D):
    """max over elements of |C - C_ref| / D.  Where D == 0 the element must be
    equal (then it counts as 0), else the error is infinite."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    diff = np.abs(C - C_ref)
    zero = D == 0
    if np.any(zero & (diff != 0)):
        return float("inf")
    with np.errstate(divide="ignore", invalid="ignore"):
        err = np.where(zero, 0.0, diff / np.where(zero, 1.0, D))
    return float(err.max()) if err.size else 0.0


def flops(nnz: int, N: int) -> int:
    """Algorithmic work of the SpMM: 2 flops per multiply-accumulate, one MAC
    per nonzero of A per column of B (Sec. 5 counts nnz*N MACs)."""
    return 2 * int(nnz) * int(N)
