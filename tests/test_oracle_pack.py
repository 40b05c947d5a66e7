"""Pins for the oracle's Alg. 1 packer (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle.pack import pack_tile, pack_panels, unpack_panels

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_hand_example_alg1():
    g = _golden("hand_example.json")
    A = np.array(g["A"], dtype=np.float32)
    A_p, loc_m, col_ind, nnz = pack_tile(A)
    assert A_p.tolist() == g["A_p"]
    assert loc_m.tolist() == g["loc_m"]
    assert col_ind.tolist() == g["col_ind"]
    assert nnz.tolist() == g["nnz"]
    assert not set(g["untouched_B_rows"]) & set(col_ind.tolist())


def test_fig4_skipped_rows():
    g = _golden("fig4_column.json")
    A = np.array(g["column"], dtype=np.float32)[:, None]
    A_p, loc_m, col_ind, nnz = pack_tile(A)
    assert loc_m.tolist() == g["loc_m"]
    assert not set(g["skipped_rows"]) & set(loc_m.tolist())
    assert nnz.tolist() == [len(g["loc_m"])] and col_ind.tolist() == [0]


def test_fig5_shape_column_major_order():
    # Fig. 5: a 6 x 16 tile with 22 nonzeros packs into one buffer of 22
    # values laid out column after column.
    rng = np.random.default_rng(5)
    A = np.zeros((6, 16), dtype=np.float32)
    pos = rng.choice(96, size=22, replace=False)
    A.ravel()[pos] = np.arange(1, 23, dtype=np.float32)
    A_p, loc_m, col_ind, nnz = pack_tile(A)
    assert A_p.size == 22 and nnz.sum() == 22
    # independent statement of column-major order: the transpose's row-major nonzeros
    assert np.array_equal(A_p, A.T[A.T != 0])
    assert np.array_equal(col_ind, np.flatnonzero((A != 0).any(axis=0)))


@pytest.mark.parametrize("M,K,m_r,s", [(1, 1, 8, 0.0), (7, 5, 4, 0.5), (33, 17, 8, 0.9),
                                       (64, 40, 32, 0.99), (70, 9, 16, 0.0), (5, 12, 32, 1.0)])
def test_round_trip_and_invariants(M, K, m_r, s):
    rng = np.random.default_rng(M * 1000 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    A[rng.random((M, K)) < s] = 0
    pk = pack_panels(A, m_r)
    assert np.array_equal(unpack_panels(pk), A)
    assert pk.A_p.size == np.count_nonzero(A) == pk.nnz.sum()
    assert pk.n_panels == (M + m_r - 1) // m_r
    for p in range(pk.n_panels):
        cols = pk.col_ind[pk.panel_cols[p]:pk.panel_cols[p + 1]]
        assert np.all(np.diff(cols) > 0), "col_ind strictly ascending"
        rows = min(m_r, M - p * m_r)
        pos = pk.panel_nnz[p]
        for c in range(pk.panel_cols[p], pk.panel_cols[p + 1]):
            assert pk.nnz[c] >= 1
            lm = pk.loc_m[pos:pos + pk.nnz[c]]
            assert np.all(np.diff(lm) > 0), "loc_m ascending within a column"
            assert lm.min() >= 0 and lm.max() < rows
            pos += pk.nnz[c]
        assert pos == pk.panel_nnz[p + 1]
        # every non-empty column of the panel appears, empty ones do not
        blk = A[p * m_r:p * m_r + rows]
        assert np.array_equal(cols, np.flatnonzero((blk != 0).any(axis=0)))


def test_ieee_zero_test():
    # -0.0 is skipped (it compares equal to 0); NaN and Inf are kept
    A = np.array([[-0.0, np.nan, np.inf, 1.0]], dtype=np.float32)
    A_p, loc_m, col_ind, nnz = pack_tile(A)
    assert col_ind.tolist() == [1, 2, 3]
    assert np.isnan(A_p[0]) and A_p[1] == np.inf and A_p[2] == 1.0


def test_int8_dtype_kept():
    A = np.array([[0, -3], [7, 0]], dtype=np.int8)
    A_p, loc_m, col_ind, nnz = pack_tile(A)
    assert A_p.dtype == np.int8 and A_p.tolist() == [7, -3]
    assert loc_m.tolist() == [1, 0]
