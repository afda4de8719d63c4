"""Closed forms printed in the paper, restated plainly -- TEST INFRASTRUCTURE ONLY.

Each function follows one equation or worked example and is used by the tests to check
the library's host-side helpers (cost model, threshold, skew, tile-shape rules) and the
oracle's own bookkeeping.
"""
from __future__ import annotations

import math


def cost_vector(nnz: float, p_vec: float) -> float:
    """Eq. 1, vector engine: time proportional to the nonzeros it touches."""
    return nnz / p_vec


def cost_matrix(rows: float, cols: float, p_mat: float) -> float:
    """Eq. 1, matrix engine: time proportional to the full tile volume M*K."""
    return rows * cols / p_mat


def alpha(p_vec: float, p_mat: float, r: float) -> float:
    """Eq. 3: density threshold alpha = r * P_vec / P_mat (the minimiser of Eq. 2)."""
    return r * p_vec / p_mat


def nnz_star(rows: int, cols: int, p_vec: float, p_mat: float, r: float) -> float:
    """Eq. 2 solved in closed form: NNZ* / P_vec = r * M * K / P_mat."""
    return r * p_vec * rows * cols / p_mat


def len_threshold(a: float, dim: int) -> float:
    """Eq. 5: Thres = alpha * K for a vector of dimension K."""
    return a * dim


def tau_tile(a: float, tm: int, tk: int) -> int:
    """Integer tile threshold: a tile of tm*tk slots is dense iff nnz >= ceil(alpha*tm*tk)."""
    return int(math.ceil(a * tm * tk))


def skew(dt_mat: float, dt_vec: float) -> float:
    """Eq. 6: Skew = max(dt) / min(dt) >= 1."""
    return max(dt_mat, dt_vec) / min(dt_mat, dt_vec)


def needs_migration(dt_mat: float, dt_vec: float, eps: float = 0.05) -> bool:
    """Section 5.3: migrate only when Skew > 1 + eps."""
    return skew(dt_mat, dt_vec) > 1.0 + eps


def migration_direction(dt_mat: float, dt_vec: float) -> str:
    """Section 5.3: the slower engine gives work away ('to_vector' when the matrix side lags)."""
    if dt_mat > dt_vec:
        return "to_vector"
    if dt_vec > dt_mat:
        return "to_matrix"
    return "none"


def l0_limits(cap_a: int, cap_b: int, cap_c: int, a_bytes: int = 2, c_bytes: int = 4):
    """Eq. 8: with double buffering each tile may use half of each buffer.

    Returns the bounds on M*K, N*K and M*N (elements).
    """
    return cap_a // 2 // a_bytes, cap_b // 2 // a_bytes, cap_c // 2 // c_bytes


def tile_fits(M: int, N: int, K: int, cap_a: int, cap_b: int, cap_c: int) -> bool:
    mk, nk, mn = l0_limits(cap_a, cap_b, cap_c)
    return (M * K <= mk and N * K <= nk and M * N <= mn
            and M % 16 == 0 and N % 16 == 0 and K % 16 == 0)


def tile_input_bytes(M: int, N: int, K: int, elem_bytes: int = 2) -> int:
    """Section 6.2.2: per-tile input traffic = A-tile + B-tile footprint = 2(MK + NK) for fp16."""
    return elem_bytes * (M * K + N * K)


def density_improvement(rho_after: float, rho_before: float) -> float:
    """Section 8.3: multiplicative increase of the tile nonzero ratio."""
    return rho_after / rho_before


def redundant_zero_fraction(dense_pattern, t: int) -> float:
    """Section 3.2 / Table 1 metric: fraction of zeros inside t x t tiles that hold a nonzero."""
    import numpy as np
    a = np.asarray(dense_pattern) != 0
    m, n = a.shape
    zeros = 0
    slots = 0
    for bi in range(0, m, t):
        for bj in range(0, n, t):
            blk = a[bi:bi + t, bj:bj + t]
            c = int(blk.sum())
            if c:
                zeros += t * t - c
                slots += t * t
    return zeros / slots if slots else 0.0


def spmm_flops(nnz: int, K: int) -> int:
    """Useful flops of one SpMM: one multiply and one add per nonzero and output column."""
    return 2 * nnz * K


def algorithmic_bytes(m: int, nnz: int, K: int, n_touched: int, b_bytes: int) -> int:
    """CSR-input byte model: row pointers, (col, val) pairs, each touched B row once, C once."""
    return 4 * (m + 1) + 8 * nnz + b_bytes * K * n_touched + 4 * m * K
