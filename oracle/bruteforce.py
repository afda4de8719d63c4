"""Pure-Python brute-force partition for tiny matrices -- TEST INFRASTRUCTURE ONLY.

An independent restatement of the reference partition (row/column extraction with the
Len rule of Eq. 4-5, row windows and column compaction of Section 6.1, density binning
with the integer tile threshold, the residual and its balanced chunks, Section 7), written
with Python sets, dicts and a dense pattern instead of the C oracle's sorted arrays.  It pins
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

    owner = {}          # row -> (dense item index, absorbs)
    dwin, dwin_absorb, dcost = [], [], []
    for w, wr in enumerate(windows):
        ntd = win_dptr[w + 1] - win_dptr[w]
        if ntd == 0:
            continue
        rows_w = [i for i in wr if i >= 0]
        res_w = sum(len(res[i]) for i in rows_w)
        absorb = res_w <= t["absorb_cap"]
        for i in rows_w:
            owner[i] = (len(dwin), absorb)
        dwin.append(w)
        dwin_absorb.append(1 if absorb else 0)
        dcost.append(ntd * TM * TK * t["cost_tc"] + ((res_w if absorb else 0) + len(rows_w)) * t["cost_res"])

    rl = [i for i in range(m) if i not in owner or (not owner[i][1] and len(res[i]) > 0)]
    starts = [0]
    for i in rl:
        starts.append(starts[-1] + len(res[i]) + 1)
    T = starts[-1]
    W = t["chunk_nnz"]
    nc = -(-T // W) if T else 0
    # merge item x belongs to RL row k when starts[k] <= x < starts[k+1]
    item_row = []
    for k, i in enumerate(rl):
        item_row += [k] * (len(res[i]) + 1)
    bounds = [0]
    for c in range(1, nc):
        k = item_row[c * W]
        bounds.append(starts[k] if 2 * (len(res[rl[k]]) + 1) <= W else c * W)
    if nc:
        bounds.append(T)
    chunk_of_item = []
    for c in range(nc):
        chunk_of_item += [c] * (bounds[c + 1] - bounds[c])
    chunk_k0 = [item_row[bounds[c]] for c in range(nc)]

    pieces = {i: 1 for i in owner}
    first_chunk = {}
    for k, i in enumerate(rl):
        chunks = set(chunk_of_item[starts[k]:starts[k + 1]])
        pieces[i] = pieces.get(i, 0) + len(chunks)
        first_chunk[i] = min(chunks)
    split = [i for i in range(m) if pieces.get(i, 0) >= 2]
    row_split = [-1] * m
    split_np, split_slot, split_base = [], [], []
    slot = 0
    for s, i in enumerate(split):
        row_split[i] = s
        split_np.append(pieces[i])
        split_slot.append(slot)
        split_base.append(first_chunk[i] - (1 if i in owner else 0))
        slot += pieces[i]

    G = t["group"]
    nq = -(-nc // G) if nc else 0
    costs = list(dcost) + [(bounds[min(q * G + G, nc)] - bounds[q * G]) * t["cost_res"]
                           for q in range(nq)]
    bucket = [c.bit_length() - 1 if c >= 1 else 0 for c in costs]
    queue = sorted(range(len(costs)), key=lambda it: (-bucket[it], it))

    if b_bf16:
        dvals_arr = _bf16_library(np.asarray(dvals, dtype=np.float32)) if dvals else np.zeros(0, np.uint16)
    else:
        dvals_arr = np.asarray(dvals, dtype=np.float32)
    i32 = lambda x: np.asarray(x, dtype=np.int32)
    return dict(
        m=m, n=n, m_aic=len(aic), n_win=n_win, n_dtiles=len(tiles), n_dwin=len(dwin),
        n_dvals=voff[-1], n_res=res_rowptr[-1], n_rl=len(rl), T=T, n_chunks=nc,
        n_split=len(split), n_slots=slot, n_items=len(costs),
        aic_rows=i32(aic), win_rows=i32([i for wr in windows for i in wr]),
        win_dptr=i32(win_dptr), dwin=i32(dwin), dwin_absorb=i32(dwin_absorb),
        dtile_cols=i32(dtile_cols), dtile_bits=np.asarray(dtile_bits, dtype=np.uint32),
        dtile_voff=i32(voff), dtile_vals=dvals_arr,
        res_rowptr=i32(res_rowptr), res_col=i32([j for r in res for j, _ in r]),
        res_val=np.asarray([x for r in res for _, x in r], dtype=np.float32),
        rl_rows=i32(rl), rl_start=i32(starts), chunk_b=i32(bounds if nc else [0]),
        chunk_k0=i32(chunk_k0), row_split=i32(row_split), split_row=i32(split),
        split_np=i32(split_np), split_slot=i32(split_slot), split_base=i32(split_base),
        queue=i32(queue), item_cost=np.asarray(costs, dtype=np.int64),
    )
