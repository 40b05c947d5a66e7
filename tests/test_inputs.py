"""Seeded generators: exact counts, reproducibility, pattern structure."""
import numpy as np
import pytest

from paper_2307_03930_gb300 import inputs as gen


def test_exact_nnz_values():
    assert gen.exact_nnz(1024, 1024, 0.9) == 104858
    assert [gen.exact_nnz(512, 4608, s) for s in (0.5, 0.7, 0.9, 0.95, 0.99, 0.998)] == \
        [1179648, 707789, 235930, 117965, 23593, 4719]
    assert gen.exact_nnz(11008, 4096, 0.9) == 4508877
    assert gen.exact_nnz(3, 3, 1.0) == 0 and gen.exact_nnz(3, 3, 0.0) == 9


@pytest.mark.parametrize("pattern", ["uniform", "magnitude"])
def test_exact_count_and_reproducible(pattern):
    a = gen.sparse_weight(64, 96, 0.9, gen.rng_for(1, 2), pattern)
    b = gen.sparse_weight(64, 96, 0.9, gen.rng_for(1, 2), pattern)
    assert np.array_equal(a, b)
    assert np.count_nonzero(a) == gen.exact_nnz(64, 96, 0.9)
    c = gen.sparse_weight(64, 96, 0.9, gen.rng_for(1, 3), pattern)
    assert not np.array_equal(a, c)


def test_magnitude_prune_keeps_largest():
    W = gen.normal((40, 50), gen.rng_for(0))
    P = gen.magnitude_prune(W, 0.7)
    kept = np.abs(W[P != 0])
    dropped = np.abs(W[P == 0])
    assert kept.min() >= dropped.max()


def test_block4x1_structure():
    m = gen.block4x1_mask(37, 50, 0.9, gen.rng_for(4))
    full = np.zeros((40, 50), bool)
    full[:37] = m
    blocks = full.reshape(10, 4, 50)
    s = blocks.sum(axis=1)
    # each aligned 4-row block is all-or-nothing (except the ragged tail)
    assert np.all((s[:-1] == 0) | (s[:-1] == 4))
    assert abs(int(m.sum()) - gen.exact_nnz(37, 50, 0.9)) <= 4


def test_powerlaw_rows_exact_and_skewed():
    m = gen.powerlaw_rows_mask(500, 300, 0.95, gen.rng_for(4, 1))
    assert int(m.sum()) == gen.exact_nnz(500, 300, 0.95)
    r = m.sum(axis=1)
    assert r.max() > 5 * r.mean()
    assert r.max() <= 300


def test_relu_b_half_zeros():
    B = gen.relu_normal((400, 500), gen.rng_for(1, 9))
    assert B.min() == 0 and abs((B == 0).mean() - 0.5) < 0.01


def test_c4_shapes_ranges():
    sh = gen.c4_shapes(3)
    assert len(sh) == 64
    for M, K, N, s in sh:
        assert 64 <= M <= 4096 and 64 <= K <= 4096 and 196 <= N <= 12544 and 0.7 <= s <= 0.99
    assert sh == gen.c4_shapes(3)
