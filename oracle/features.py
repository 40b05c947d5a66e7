"""Oracle: input features of the learned schedule selector.  Test infrastructure.

The selector sees the problem sizes, the nonzero count, the row-nonzero
histogram and statistics of the row panels that Alg. 1 packs (the density the
sparsity-aware tiling of Sec. 4.2 is built on).  The feature vector (16
entries) is defined here in plain numpy:

  0 log2 M            1 log2 K            2 log2 N           3 density nnz/(M K)
  4 log2(1+nnz)       5 log2(1+mean row nnz)
  6 coefficient of variation of row nnz (population std / mean; 0 if mean 0)
  7 log2(1+max row nnz) - log2(1+mean row nnz)
  8..11 fraction of rows with row nnz r in the bins (integer tests on r, K):
        100 r < K | 20 r < K <= 100 r | 5 r < K <= 20 r | K <= 5 r
  12 mean over panels of (non-empty columns of the panel) / K
  13 coefficient of variation of panel nnz
  14 log2(1 + nnz / total non-empty panel columns)  (mean nonzeros per packed column)
  15 fraction of panels holding no nonzero
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 16
__all__ = ["N_FEATURES", "features"]


def _cv(x):
    x = np.asarray(x, dtype=np.float64)
    m = x.mean() if x.size else 0.0
    if m == 0:
        return 0.0
    return float(np.sqrt(np.mean((x - m) ** 2)) / m)


def features(A, m_r: int, N: int) -> np.ndarray:
    A = np.asarray(A)
    M, K = A.shape
    nzmask = A != 0
    nnz = int(nzmask.sum())
    row = nzmask.sum(axis=1).astype(np.int64)
    P = (M + m_r - 1) // m_r
    panel_nnz = np.array([row[p * m_r:(p + 1) * m_r].sum() for p in range(P)], dtype=np.int64)
    panel_cols = np.array([int(nzmask[p * m_r:(p + 1) * m_r].any(axis=0).sum())
                           for p in range(P)], dtype=np.int64)
    f = np.zeros(N_FEATURES, dtype=np.float64)
    f[0], f[1], f[2] = np.log2(M), np.log2(K), np.log2(N)
    f[3] = nnz / (M * K)
    f[4] = np.log2(1 + nnz)
    mean_row = row.mean()
    f[5] = np.log2(1 + mean_row)
    f[6] = _cv(row)
    f[7] = np.log2(1 + row.max()) - np.log2(1 + mean_row)
    f[8] = np.mean(100 * row < K)
    f[9] = np.mean((20 * row < K) & (K <= 100 * row))
    f[10] = np.mean((5 * row < K) & (K <= 20 * row))
    f[11] = np.mean(K <= 5 * row)
    f[12] = np.mean(panel_cols / K)
    f[13] = _cv(panel_nnz)
    tc = panel_cols.sum()
    f[14] = np.log2(1 + (nnz / tc if tc else 0.0))
    f[15] = np.mean(panel_nnz == 0)
    return f
