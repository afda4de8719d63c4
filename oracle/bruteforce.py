"""Pure-Python brute-force partition for tiny matrices -- TEST INFRASTRUCTURE ONLY.

An independent restatement of the reference partition (row/column extraction with the
Len rule of Eq. 4-5, Section 6.1 local reordering, row windows and column compaction, density
binning with the integer tile threshold, and the residual of Section 5.2.2), written with
Python sets, dicts and a dense pattern instead of the C oracle's sorted arrays.  It pins
:func:`oracle.plan`: both must produce identical arrays on every tiny input.  O(m*n) memory;
keep m, n <= a few hundred.
"""
from __future__ import annotations

import math
from fractions import Fraction
from collections import Counter

import numpy as np

from . import DEFAULT_TUNE, TAU_INF


def _bf16_library(x: np.ndarray) -> np.ndarray:
    """BF16 bit patterns via PyTorch's cast (round to nearest even), independent of the C oracle."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()


def jaccard(a: set, b: set) -> Fraction:
    union = len(a | b)
    return Fraction(len(a & b), union) if union else Fraction(0)


def local_reorder(rows: list, row: list, keep_col: set, TM: int, cluster: int) -> list:
    """Section 6.1 local stage: in each cluster of consecutive rows, the first unassigned row
    anchors a new window and takes the TM - 1 unassigned rows with the largest Jaccard
    similarity of kept-column sets (earlier rows first on ties)."""
    out = []
    for c0 in range(0, len(rows), cluster):
        cl = rows[c0:c0 + cluster]
        cols = [set(row[i]) & keep_col for i in cl]
        free = list(range(len(cl)))
        while free:
            a = free.pop(0)
            out.append(cl[a])
            ranked = sorted(free, key=lambda b: (-jaccard(cols[a], cols[b]), b))
            take = ranked[:TM - 1]
            out.extend(cl[b] for b in take)
            free = [b for b in free if b not in take]
    return out


def plan(A: dict, K: int, *, b_bf16: bool = False, **tune) -> dict:
    t = dict(DEFAULT_TUNE)
    t.update(tune)
    TM, TK, tau = t["TM"], t["TK"], t["tau_tile"]
    m, n = int(A["m"]), int(A["n"])
    rp, ci, v = A["rowptr"], A["colidx"], A["vals"]
    row = [dict((int(ci[p]), np.float32(v[p])) for p in range(rp[i], rp[i + 1])) for i in range(m)]

    windows_on = tau != TAU_INF
    aic = [i for i in range(m) if windows_on and len(row[i]) > t["tau_row"]]
    keep_col = set(range(n))
    if windows_on and t["tau_col"] > 0:
        cc = Counter(j for i in aic for j in row[i])
        keep_col = {j for j in range(n) if cc.get(j, 0) > t["tau_col"]}

    if windows_on and t.get("reorder", 0) > 0:
        aic = local_reorder(aic, row, keep_col, TM, t["reorder"] * TM)
    n_win = math.ceil(len(aic) / TM)
    windows = [[aic[w * TM + r] if w * TM + r < len(aic) else -1 for r in range(TM)]
               for w in range(n_win)]

    in_dense_tile = set()          # (i, j) covered by a dense tile
    tiles = []                     # (window, [cols], {(r, c)}) in order
    win_dptr = [0]
    for w, wr in enumerate(windows):
        counts = Counter(j for i in wr if i >= 0 for j in row[i] if j in keep_col)
        if t["col_order"] == 0:
            order = sorted(counts, key=lambda j: (-counts[j], j))
        else:
            order = sorted(counts)
        for s in range(0, len(order), TK):
            cols = order[s:s + TK]
            if sum(counts[j] for j in cols) >= tau:
                cells = {(r, c) for r, i in enumerate(wr) if i >= 0
                         for c, j in enumerate(cols) if j in row[i]}
                tiles.append((w, cols, cells))
                for r, c in cells:
                    in_dense_tile.add((wr[r], cols[c]))
        win_dptr.append(len(tiles))

    BW = TM * TK // 32
    dtile_cols, dtile_bits, voff, dvals = [], [], [0], []
    for w, cols, cells in tiles:
        dtile_cols += cols + [-1] * (TK - len(cols))
        words = [0] * BW
        for r, c in cells:
            b = r * TK + c
            words[b // 32] |= 1 << (b % 32)
        dtile_bits += words
        seq = [row[windows[w][r]][cols[c]] for r in range(TM) for c in range(TK) if (r, c) in cells]
        pad = (-len(seq)) % 8
        dvals += seq + [np.float32(0)] * pad
        voff.append(voff[-1] + len(seq) + pad)

    res = [[(j, row[i][j]) for j in sorted(row[i]) if (i, j) not in in_dense_tile] for i in range(m)]
    res_rowptr = [0]
    for i in range(m):
        res_rowptr.append(res_rowptr[-1] + len(res[i]))

    if b_bf16:
        dvals_arr = _bf16_library(np.asarray(dvals, dtype=np.float32)) if dvals else np.zeros(0, np.uint16)
    else:
        dvals_arr = np.asarray(dvals, dtype=np.float32)
    i32 = lambda x: np.asarray(x, dtype=np.int32)
    return dict(
        m=m, n=n, m_aic=len(aic), n_win=n_win, n_dtiles=len(tiles),
        n_dwin=sum(1 for w in range(n_win) if win_dptr[w + 1] > win_dptr[w]),
        n_dvals=voff[-1], n_res=res_rowptr[-1],
        aic_rows=i32(aic), win_rows=i32([i for wr in windows for i in wr]),
        win_dptr=i32(win_dptr),
        dtile_cols=i32(dtile_cols), dtile_bits=np.asarray(dtile_bits, dtype=np.uint32),
        dtile_voff=i32(voff), dtile_vals=dvals_arr,
        res_rowptr=i32(res_rowptr), res_col=i32([j for r in res for j, _ in r]),
        res_val=np.asarray([x for r in res for _, x in r], dtype=np.float32),
    )
