"""Seeded synthetic input generators shared by the tests, the bench and the smoke run.

This module only draws random matrices and masks.  It holds none of the method's
arithmetic (no packing, no products, no rounding to BF16/INT8): those live
separately in the CUDA library and, independently, in the oracle.

Workload shapes follow the synthetic stand-ins for the paper's experiments
(synthetic uniform sparsity, Sec. 5.2; magnitude-pruned weights, Sec. 5.3/5.4):

* sparsity ``s`` fixes the exact nonzero count
  ``nnz = M*K - round_half_up(s*M*K)`` (uniform-density assumption of Sec. 4.2),
* uniform masks pick exactly ``nnz`` positions without replacement,
* magnitude pruning draws N(0,1) and zeroes the smallest ``|x|`` (ties broken
  by flat index, a stable order),
* post-ReLU activations are ``max(0, z)`` with ``z ~ N(0,1)``,
* 4x1 blocks cover 4 consecutive rows (aligned to 4) of one column,
* power-law rows give row i a weight ``U_i^(-1/alpha)`` (Pareto, alpha = 1.5).

Every function takes a ``numpy.random.Generator`` or a seed; nothing reads
global state.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng_for", "exact_nnz", "normal", "relu_normal", "uniform_mask",
    "magnitude_prune", "block4x1_mask", "powerlaw_rows_mask", "sparse_weight",
    "c4_shapes", "loguniform_int",
]


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    """Independent generator for (seed, stream...) so that separate tensors of
    one workload never share a random stream."""
    return np.random.default_rng([int(seed), *[int(x) for x in stream]])


def exact_nnz(M: int, K: int, s: float) -> int:
    """Number of nonzeros for sparsity s: M*K minus round-half-up(s*M*K)."""
    total = int(M) * int(K)
    zeros = int(math.floor(float(s) * total + 0.5))
    zeros = min(max(zeros, 0), total)
    return total - zeros


def normal(shape, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal(shape, dtype=np.float32)


def relu_normal(shape, rng: np.random.Generator) -> np.ndarray:
    """Post-ReLU activations: half-normal with (in expectation) 50% zeros."""
    z = rng.standard_normal(shape, dtype=np.float32)
    return np.maximum(z, np.float32(0.0))


def uniform_mask(M: int, K: int, s: float, rng: np.random.Generator) -> np.ndarray:
    """Boolean M x K mask with exactly exact_nnz(M, K, s) True entries placed
    uniformly at random (without replacement)."""
    nnz = exact_nnz(M, K, s)
    mask = np.zeros(M * K, dtype=bool)
    if nnz:
        pos = rng.choice(M * K, size=nnz, replace=False)
        mask[pos] = True
    return mask.reshape(M, K)


def magnitude_prune(W: np.ndarray, s: float) -> np.ndarray:
    """Zero the round_half_up(s*size) entries of smallest |x|; ties broken by
    flat index (stable sort).  Returns a new array."""
    M, K = W.shape
    zeros = M * K - exact_nnz(M, K, s)
    out = np.array(W, copy=True)
    if zeros:
        order = np.argsort(np.abs(out).ravel(), kind="stable")
        out.ravel()[order[:zeros]] = 0
    return out


def block4x1_mask(M: int, K: int, s: float, rng: np.random.Generator) -> np.ndarray:
    """Mask made of 4x1 blocks (4 consecutive rows aligned to 4, one column;
    the last row block may be shorter when M % 4 != 0).  Blocks are taken in
    a uniformly random order until the nnz target is met, so the count
    exceeds exact_nnz by at most 3."""
    nnz = exact_nnz(M, K, s)
    mb = (M + 3) // 4
    mask = np.zeros((mb * 4, K), dtype=bool)
    if nnz:
        order = rng.permutation(mb * K)
        bi, kj = np.divmod(order, K)
        size = np.where(bi == mb - 1, M - 4 * (mb - 1), 4)
        take = int(np.searchsorted(np.cumsum(size), nnz)) + 1
        bi, kj = bi[:take], kj[:take]
        for r in range(4):
            mask[bi * 4 + r, kj] = True
    return mask[:M]


def powerlaw_rows_mask(M: int, K: int, s: float, rng: np.random.Generator,
                       alpha: float = 1.5) -> np.ndarray:
    """Mask whose row nonzero counts follow a power law: row i gets weight
    U_i^(-1/alpha), counts are scaled to the exact nnz target (largest
    remainder), capped at K with the excess moved to uncapped rows; columns
    are uniform without replacement within each row."""
    nnz = exact_nnz(M, K, s)
    u = rng.random(M)
    u = np.maximum(u, 1e-12)
    w = u ** (-1.0 / alpha)
    counts = np.zeros(M, dtype=np.int64)
    remaining = nnz
    free = np.ones(M, dtype=bool)
    while remaining > 0 and free.any():
        ww = np.where(free, w, 0.0)
        share = ww / ww.sum() * remaining
        add = np.floor(share).astype(np.int64)
        rem = remaining - int(add.sum())
        if rem > 0:
            frac = np.where(free, share - add, -1.0)
            top = np.argsort(-frac, kind="stable")[:rem]
            add[top] += 1
        counts += add
        over = counts > K
        excess = int((counts[over] - K).sum())
        counts[over] = K
        free &= counts < K
        remaining = excess
    mask = np.zeros((M, K), dtype=bool)
    for i in range(M):
        c = int(counts[i])
        if c:
            mask[i, rng.choice(K, size=c, replace=False)] = True
    return mask


def sparse_weight(M: int, K: int, s: float, rng: np.random.Generator,
                  pattern: str = "uniform") -> np.ndarray:
    """FP32 weight matrix with N(0,1) nonzeros and the requested pattern:
    'uniform' (uniform random mask), 'magnitude' (magnitude pruning of a dense
    N(0,1) draw), 'block4x1' or 'powerlaw'."""
    if pattern == "magnitude":
        return magnitude_prune(normal((M, K), rng), s)
    if pattern == "uniform":
        mask = uniform_mask(M, K, s, rng)
    elif pattern == "block4x1":
        mask = block4x1_mask(M, K, s, rng)
    elif pattern == "powerlaw":
        mask = powerlaw_rows_mask(M, K, s, rng)
    else:
        raise ValueError(f"unknown sparsity pattern {pattern!r}")
    vals = normal((M, K), rng)
    # a drawn exact zero would silently drop a mask entry; nudge it
    vals[vals == 0] = np.float32(1.0)
    return np.where(mask, vals, np.float32(0.0)).astype(np.float32)


def loguniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def c4_shapes(seed: int, count: int = 64, smin: float = 0.70, smax: float = 0.99):
    """Uneven per-layer problems: M, K log-uniform in [64, 4096], N log-uniform
    in [196, 12544], sparsity uniform in [smin, smax].  Draw order per
    problem: M, K, N, s."""
    rng = rng_for(seed, 0)
    out = []
    for _ in range(count):
        M = loguniform_int(rng, 64, 4096)
        K = loguniform_int(rng, 64, 4096)
        N = loguniform_int(rng, 196, 12544)
        s = float(rng.uniform(smin, smax))
        out.append((M, K, N, s))
    return out
