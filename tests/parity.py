"""Result checks against the FP64 oracle (test infrastructure).

Every element of C is compared with the definition C[i,:] = sum_p vals[p] * B[col[p], :] in
float64.  Beside the matrix-wide relative Frobenius error (the stated tolerance: 1e-5 for the
FP32 path, 2e-2 when B and the dense tiles are BF16), each element must meet the forward error
bound of a floating-point dot product,

    |C_ik - C*_ik| <= gamma_i * (|A| |B|)_ik,    gamma_i = (len_i + 16) * 2^-22 [+ 2^-8 for BF16 tiles]

where len_i is the row's nonzero count: any summation order of len_i FP32 products (plus the
partial-row sums of a split row) stays within len_i * 2^-24 of |A||B| when rounding to nearest;
the bound allows twice that plus slack for the three-term TF32 products and for tensor-core
accumulation.  Rounding the dense-tile values of A to BF16 adds at most 2^-9 |a| per product.
A row of the reference that is exactly zero (an empty row) must be exactly zero.
"""
from __future__ import annotations

import numpy as np

import oracle


def abs_csr(A: dict) -> dict:
    out = dict(A)
    out["vals"] = np.abs(np.asarray(A["vals"], dtype=np.float32))
    return out


def abs_b(B: np.ndarray, b_bf16: bool) -> np.ndarray:
    return (B & np.uint16(0x7FFF)) if b_bf16 else np.abs(B)


def check_result(C: np.ndarray, A: dict, B: np.ndarray, *, b_bf16: bool = False,
                 bf16_tiles: bool = False, tol: float = 1e-5, rows: np.ndarray | None = None,
                 threads: int = 8, block: int = 1 << 17) -> dict:
    """Compare C (all rows, or the rows in `rows`) with the oracle; assert the tolerance, the
    element-wise bound and exact zeros.  Returns the error figures.  Rows are taken in blocks so
    the float64 temporaries stay small at full size."""
    m = int(A["m"])
    rows = np.arange(m, dtype=np.int32) if rows is None else np.asarray(rows, dtype=np.int32)
    lens_all = np.diff(np.asarray(A["rowptr"], dtype=np.int64))
    absA, absB = abs_csr(A), abs_b(B, b_bf16)
    d2 = r2 = 0.0
    max_row_rel = max_ratio = 0.0
    worst = None
    for r0 in range(0, len(rows), block):
        rb = rows[r0:r0 + block]
        ref = oracle.spmm(A, B, rows=rb, b_bf16=b_bf16, threads=threads)
        mag = oracle.spmm(absA, absB, rows=rb, b_bf16=b_bf16, threads=threads)
        Cs = np.asarray(C[rb], dtype=np.float64)
        assert np.isfinite(Cs).all(), "non-finite output"
        diff = np.abs(Cs - ref)
        gamma = (lens_all[rb] + 16).astype(np.float64) * 2.0 ** -22 + (2.0 ** -8 if bf16_tiles else 0.0)
        bound = gamma[:, None] * mag
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(bound > 0, diff / bound, np.where(diff > 0, np.inf, 0.0))
        if ratio.size and ratio.max() > max_ratio:
            max_ratio = float(ratio.max())
            k = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
            worst = (int(rb[k[0]]), int(k[1]), float(diff[k]), float(bound[k]))
        rn = np.linalg.norm(ref, axis=1)
        dn = np.linalg.norm(diff, axis=1)
        zero = rn == 0
        assert np.all(dn[zero] == 0), "a row that must be zero is not"
        if (~zero).any():
            max_row_rel = max(max_row_rel, float((dn[~zero] / rn[~zero]).max()))
        d2 += float((dn ** 2).sum())
        r2 += float((rn ** 2).sum())
    fro = (d2 ** 0.5 / r2 ** 0.5) if r2 > 0 else (0.0 if d2 == 0 else float("inf"))
    out = {"rel_frobenius": fro, "max_row_rel_err": max_row_rel, "max_bound_ratio": max_ratio,
           "rows": int(len(rows))}
    assert fro <= tol, f"relative Frobenius error {fro} above {tol}"
    assert max_ratio <= 1.0, f"element (row, col, |diff|, bound) {worst} breaks the dot-product bound"
    return out
