"""Pins for the oracle's precision handling and selector features."""
import math

import numpy as np
import pytest
import torch

from oracle.quant import bf16_round, bf16_bits, quantize_rows_int8, quantize_cols_int8
from oracle.features import features, N_FEATURES


def test_bf16_hand_cases():
    one = np.float32(1.0)
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                       # tie -> even (mantissa 0)
        1.0 + 2.0 ** -7 + 2.0 ** -8: 1.0 + 2.0 ** -6,  # tie -> even (rounds up)
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,  # above the tie
        -2.5: -2.5,
        float("inf"): float("inf"),
    }
    for x, want in cases.items():
        assert bf16_round(np.array([x], np.float32))[0] == np.float32(want), x
    assert np.isnan(bf16_round(np.array([np.nan], np.float32))[0])
    big = np.array([np.finfo(np.float32).max], np.float32)
    assert bf16_round(big)[0] == np.inf                 # RNE overflows to Inf
    assert one.dtype == np.float32


def test_bf16_matches_library_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32),
        (rng.standard_normal(2000) * 1e-38).astype(np.float32),   # subnormals
        np.frombuffer(rng.integers(0, 2 ** 32, 5000, dtype=np.uint64).astype(np.uint32).tobytes(),
                      dtype=np.float32),
    ])
    x = x[np.isfinite(x)]
    lib = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(bf16_bits(x), lib)


def test_int8_rows_hand_case_and_bounds():
    A = np.array([[0.5, -1.0, 0.25, 0.0], [0, 0, 0, 0], [3.0, 0, -0.1, 2.9]], np.float32)
    q, s = quantize_rows_int8(A)
    assert s[0] == np.float32(1.0) / np.float32(127.0)
    assert q[0].tolist() == [64, -127, 32, 0]          # rint(63.5) = 64 (half to even)
    assert s[1] == 1.0 and q[1].tolist() == [0, 0, 0, 0]
    assert q[2, 0] == 127
    rng = np.random.default_rng(2)
    A = rng.standard_normal((50, 80)).astype(np.float32)
    q, s = quantize_rows_int8(A)
    assert np.all(np.abs(q.astype(np.int32)).max(axis=1) == 127)
    err = np.abs(q.astype(np.float64) * s[:, None].astype(np.float64) - A)
    assert np.all(err <= 0.5 * s[:, None] * (1 + 1e-6) + 1e-12)
    qc, sc = quantize_cols_int8(A)
    qt, st = quantize_rows_int8(A.T.copy())
    assert np.array_equal(qc, qt.T) and np.array_equal(sc, st)


def test_features_hand_case():
    # 4 x 10 matrix, panels of 2 rows, N = 16
    A = np.zeros((4, 10), np.float32)
    A[0, [0, 3]] = 1
    A[1, 3] = 1
    A[3, :] = 1
    f = features(A, 2, 16)
    assert f.shape == (N_FEATURES,)
    row = np.array([2, 1, 0, 10])
    assert f[0] == 2 and f[1] == math.log2(10) and f[2] == 4
    assert f[3] == 13 / 40 and f[4] == math.log2(14)
    assert f[5] == math.log2(1 + 13 / 4)
    m = 13 / 4
    assert abs(f[6] - math.sqrt(np.mean((row - m) ** 2)) / m) < 1e-15
    assert abs(f[7] - (math.log2(11) - math.log2(1 + m))) < 1e-15
    # bins: r=2 -> 5r=10>=K -> bin 11?  100r<K? no; 20r<K? no; 5r<K? no; K<=5r yes
    # r=1: 5*1=5<10 and 10<=20 -> bin 10; r=0: 0<10 -> bin 8; r=10 -> bin 11
    assert f[8:12].tolist() == [0.25, 0.0, 0.25, 0.5]
    # panel 0 rows 0-1: columns {0,3} -> 2/10; panel 1 rows 2-3: 10/10
    assert f[12] == (0.2 + 1.0) / 2
    pn = np.array([3, 10])
    assert abs(f[13] - np.sqrt(np.mean((pn - 6.5) ** 2)) / 6.5) < 1e-15
    assert f[14] == math.log2(1 + 13 / 12)
    assert f[15] == 0.0
