"""Oracle: Rosko packing (Alg. 1, Sec. 4.1) and its inverse.  Test infrastructure.

Alg. 1 walks an M x K tile column by column (k ascending) and, inside a
column, row by row (m ascending).  Every nonzero value is appended to ``A_p``
and its row to ``loc_m``; a column that holds at least one nonzero appends its
index to ``col_ind`` and its count to ``nnz``.  Empty columns leave no trace.

Reading of the paper used here: a pack covers one row panel of ``m_r``
consecutive rows of A (Sec. 4.2 packs d*m_r x k_c tiles); ``loc_m`` is
relative to the panel; panels are stored one after another.  The zero test is
the IEEE comparison ``a != 0`` (so -0.0 is skipped and NaN/Inf are kept).
"""
from __future__ import annotations

import numpy as np

__all__ = ["pack_tile", "pack_panels", "unpack_panels", "PackedPanels"]


def pack_tile(A: np.ndarray):
    """Alg. 1 on one tile.  A is M x K (row-major in the paper: element
    A[k + m*K] is ``A[m, k]`` here).

    Returns (A_p, loc_m, col_ind, nnz) as numpy arrays; A_p keeps A's dtype.
    """
    A = np.asarray(A)
    M, K = A.shape
    A_p, loc_m, col_ind, nnz = [], [], [], []
    for k in range(K):                      # columns, ascending
        column = A[:, k]
        ms = np.flatnonzero(column != 0)    # rows m ascending with A != 0
        if ms.size != 0:                    # a non-empty column is recorded
            A_p.append(column[ms])
            loc_m.append(ms)
            col_ind.append(k)
            nnz.append(ms.size)
    if A_p:
        A_p = np.concatenate(A_p)
        loc_m = np.concatenate(loc_m)
    else:
        A_p = np.zeros(0, dtype=A.dtype)
        loc_m = np.zeros(0, dtype=np.int64)
    return (A_p.astype(A.dtype, copy=False), loc_m.astype(np.int64),
            np.asarray(col_ind, dtype=np.int64), np.asarray(nnz, dtype=np.int64))


class PackedPanels:
    """Per-panel Alg. 1 output concatenated in panel order.

    panel_cols[p]:panel_cols[p+1] indexes this panel's entries of col_ind/nnz;
    panel_nnz[p]:panel_nnz[p+1] indexes its entries of A_p/loc_m.
    """

    def __init__(self, M, K, m_r, A_p, loc_m, col_ind, nnz, panel_cols, panel_nnz):
        self.M, self.K, self.m_r = M, K, m_r
        self.A_p, self.loc_m, self.col_ind, self.nnz = A_p, loc_m, col_ind, nnz
        self.panel_cols, self.panel_nnz = panel_cols, panel_nnz

    @property
    def n_panels(self):
        return len(self.panel_cols) - 1


def pack_panels(A: np.ndarray, m_r: int) -> PackedPanels:
    """Apply Alg. 1 to each row panel A[p*m_r:(p+1)*m_r, :] (last panel ragged)."""
    A = np.asarray(A)
    M, K = A.shape
    P = (M + m_r - 1) // m_r
    parts = [pack_tile(A[p * m_r:min(M, (p + 1) * m_r), :]) for p in range(P)]
    panel_cols = np.zeros(P + 1, dtype=np.int64)
    panel_nnz = np.zeros(P + 1, dtype=np.int64)
    for p, (A_p, _, col_ind, _) in enumerate(parts):
        panel_cols[p + 1] = panel_cols[p] + col_ind.size
        panel_nnz[p + 1] = panel_nnz[p] + A_p.size

    def cat(i, dtype):
        if not parts:
            return np.zeros(0, dtype=dtype)
        return np.concatenate([q[i] for q in parts]).astype(dtype, copy=False)

    return PackedPanels(M, K, m_r, cat(0, A.dtype), cat(1, np.int64), cat(2, np.int64),
                        cat(3, np.int64), panel_cols, panel_nnz)


def unpack_panels(pk: PackedPanels) -> np.ndarray:
    """Inverse of pack_panels: scatter every packed value back to its (row, k)."""
    A = np.zeros((pk.M, pk.K), dtype=pk.A_p.dtype)
    for p in range(pk.n_panels):
        pos = pk.panel_nnz[p]
        for c in range(pk.panel_cols[p], pk.panel_cols[p + 1]):
            k = pk.col_ind[c]
            for _ in range(pk.nnz[c]):
                A[p * pk.m_r + pk.loc_m[pos], k] = pk.A_p[pos]
                pos += 1
    return A
