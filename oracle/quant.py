"""Oracle: reduced-precision storage of A's nonzeros and of B.  Test infrastructure.

The paper computes in FP32 only (Sec. 5).  The reduced-precision forms store
values as BF16 (round to nearest, ties to even, from FP32) or as symmetric
INT8 with one FP32 scale per row of A and per column of B:

    s_i = max_k |a_ik| / 127 (FP32 division), 1 for an all-zero row
    q_ik = clamp(rint(a_ik / s_i), -127, 127)   (FP32 division, ties to even)

The quotient that decides each integer code is an FP32 operation on both sides,
so the codes agree exactly.  The sparsity mask is that of the codes (q != 0).
"""
from __future__ import annotations

import numpy as np

__all__ = ["bf16_round", "bf16_bits", "quantize_rows_int8", "quantize_cols_int8"]


def bf16_bits(x) -> np.ndarray:
    """Upper 16 bits of the FP32 value rounded to nearest-even BF16 (uint16).
    NaN inputs become a quiet NaN with their sign."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    rounded = ((u + 0x7FFF + lsb) >> 16) & 0xFFFF
    nan = np.isnan(x)
    rounded = np.where(nan, ((u >> 16) | 0x0040) & 0xFFFF, rounded)
    return rounded.astype(np.uint16)


def bf16_round(x) -> np.ndarray:
    """FP32 array holding the BF16-rounded values of x."""
    b = bf16_bits(x).astype(np.uint32) << 16
    return b.view(np.float32)


def _sym_int8(X, axis):
    X = np.asarray(X, dtype=np.float32)
    amax = np.max(np.abs(X), axis=axis, keepdims=True) if X.size else np.zeros(0, np.float32)
    scale = (amax / np.float32(127.0)).astype(np.float32)
    scale = np.where(amax == 0, np.float32(1.0), scale).astype(np.float32)
    q = np.rint(X / scale)                 # FP32 quotient, round half to even
    q = np.clip(q, -127, 127).astype(np.int8)
    return q, np.squeeze(scale, axis=axis).astype(np.float32)


def quantize_rows_int8(A):
    """Per-row symmetric INT8 codes of A (M x K) and the M row scales."""
    return _sym_int8(A, axis=1)


def quantize_cols_int8(B):
    """Per-column symmetric INT8 codes of B (K x N) and the N column scales."""
    return _sym_int8(B, axis=0)
