"""Oracle: the sparsity-aware tiling model of Sec. 4.2 as plain formulas.
Test infrastructure.

Quantities are in elements (the paper's caches hold elements of one type):
d density, p cores, m_c = k_c the core-level tile, m_r x n_r the register tile.

  Eq. 1   3 d p m_c k_c + p m_c k_c + p^2 m_c^2 <= L3   (A with index arrays,
          B block, p m_c x p m_c partial C tile)
  Eq. 2   BW = IO / T = (3 d + 1) / (d m_c) * peak
  Eq. 3   3 d m_r k_c + k_c n_r + m_r n_r <= L1
"""
from __future__ import annotations

import math

__all__ = ["eq1_lhs", "eq1_max_mc", "eq2_bw", "eq3_lhs", "outer_product_intensity"]


def eq1_lhs(d, p, m_c, k_c):
    return 3 * d * p * m_c * k_c + p * m_c * k_c + p * p * m_c * m_c


def eq1_max_mc(d, p, L3):
    """Largest integer m_c (= k_c) with Eq. 1 satisfied."""
    coef = 3 * d * p + p + p * p
    m = int(math.floor(math.sqrt(L3 / coef)))
    while m > 0 and eq1_lhs(d, p, m, m) > L3:
        m -= 1
    while eq1_lhs(d, p, m + 1, m + 1) <= L3:
        m += 1
    return m


def eq2_bw(d, m_c, peak):
    return (3 * d + 1) / (d * m_c) * peak


def eq3_lhs(d, m_r, k_c, n_r):
    return 3 * d * m_r * k_c + k_c * n_r + m_r * n_r


def outer_product_intensity(m, n, d=1.0):
    """MACs per streamed element of a (packed) outer-product tile, Sec. 2.1 and
    Sec. 4.2: d m n / (d m + n); d = 1 gives the dense m n / (m + n)."""
    return d * m * n / (d * m + n)
