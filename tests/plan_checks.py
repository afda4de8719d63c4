"""Checks of a device plan against the CPU reference partition (test infrastructure).

`compare_plan` splits a device plan in two:

* the paper's partition (Sections 5.2.2 and 6.1: kept rows, windows, compacted dense tiles with
  their bitmaps and packed values, the residual CSR) must equal the oracle's bit for bit;
* the execute kernel's bookkeeping (which rows the residual chunks cover, the merge-path chunk
  boundaries, split rows and their partial-row slots, the work-list order) is not the paper's
  partition, so it is not compared with a restatement of the planner.  `check_bookkeeping`
  checks instead what the kernel needs for every output row to be written exactly once from all
  of its pieces, plus the balance and ordering properties the planner promises.  The product
  (every GPU test compares C with the FP64 definition) checks the rest.

Everything is vectorised with numpy so the checks run on the full-size workloads too.
"""
from __future__ import annotations

import numpy as np

import oracle

BOOKKEEPING = ("dwin", "dwin_absorb", "rl_rows", "rl_start", "chunk_b", "chunk_k0", "row_split",
               "split_row", "split_np", "split_slot", "split_base", "queue", "item_cost")


def oracle_tune(t) -> dict:
    """The partition parameters of a Tune (the oracle takes no execution-only field)."""
    d = t.as_dict()
    return {k: d[k] for k in oracle.DEFAULT_TUNE}


def exports(plan) -> dict:
    return {name: plan.export(name) for name in BOOKKEEPING}


def compare_partition(st: dict, arrays: dict, ref: dict) -> None:
    """Scalars and arrays of the partition bit-exact against the oracle's."""
    for k in oracle.PLAN_SCALARS:
        assert st[k] == ref[k], f"scalar {k}: device {st[k]} vs reference {ref[k]}"
    for name in oracle.PLAN_ARRAYS:
        if name == "win_dptr" and ref["n_win"] == 0:
            continue
        got, exp = arrays[name], np.asarray(ref[name])
        assert got.dtype == exp.dtype, (name, got.dtype, exp.dtype)
        assert got.shape == exp.shape, (name, got.shape, exp.shape)
        if not np.array_equal(got.view(np.uint8), exp.view(np.uint8)):
            bad = np.nonzero(got != exp)[0][:10]
            raise AssertionError(f"plan array {name} differs at {bad}: {got[bad]} vs {exp[bad]}")


def _cost_class(c: np.ndarray) -> np.ndarray:
    """floor(log2(c)) for c >= 1, 0 otherwise (exact on int64)."""
    c = np.asarray(c, dtype=np.int64)
    out = np.zeros(c.shape, dtype=np.int64)
    pos = c >= 1
    v = c[pos].copy()
    cls = np.zeros(v.shape, dtype=np.int64)
    for sh in (32, 16, 8, 4, 2, 1):
        big = v >= (np.int64(1) << sh)
        cls[big] += sh
        v[big] >>= sh
    out[pos] = cls
    return out


def check_bookkeeping(A: dict, part: dict, st: dict, ex: dict, tune: dict) -> None:
    """Invariants of the execute bookkeeping of a device plan.

    `part` is the (already verified) partition, `st` the plan's counts, `ex` its exported
    bookkeeping arrays, `tune` the full tune as a dict.
    """
    m = int(A["m"])
    TM, W, G = int(part["TM"]), int(tune["chunk_nnz"]), int(tune["group"])
    res_len = np.diff(part["res_rowptr"].astype(np.int64))
    win_rows = part["win_rows"].reshape(-1, TM) if part["n_win"] else np.zeros((0, TM), np.int32)
    ntiles = np.diff(part["win_dptr"].astype(np.int64)) if part["n_win"] else np.zeros(0, np.int64)

    # ---- dense work items: the windows that hold a dense tile, in window order ----
    dwin = ex["dwin"].astype(np.int64)
    assert np.array_equal(dwin, np.nonzero(ntiles > 0)[0]), "dwin is not the list of dense windows"
    absorb = ex["dwin_absorb"]
    assert absorb.shape == dwin.shape and np.all((absorb == 0) | (absorb == 1))
    owned = np.zeros(m, np.int8)          # 1: a dense window computes the row's residual too
    cost_dense = np.zeros(len(dwin), np.int64)
    for d, w in enumerate(dwin):
        rows = win_rows[w][win_rows[w] >= 0]
        res_w = int(res_len[rows].sum())
        # a window keeps its rows' residual iff it is small (the absorb rule)
        assert absorb[d] == (1 if res_w <= tune["absorb_cap"] else 0), f"absorb flag of window {w}"
        owned[rows] = 1 if absorb[d] else 2
        cost_dense[d] = (int(ntiles[w]) * TM * int(part["TK"]) * tune["cost_tc"]
                         + ((res_w if absorb[d] else 0) + len(rows)) * tune["cost_res"])

    # ---- the residual list: every row no dense window finishes by itself, in row order ----
    need = (owned == 0) | ((owned == 2) & (res_len > 0))
    rl = ex["rl_rows"].astype(np.int64)
    assert np.array_equal(rl, np.nonzero(need)[0]), "residual row list"
    assert st["n_rl"] == len(rl)
    rs = ex["rl_start"].astype(np.int64)
    assert rs[0] == 0 and np.array_equal(np.diff(rs), res_len[rl] + 1), "merge starts"
    T = int(rs[-1])
    assert st["T"] == T

    # ---- merge-path chunks: cover [0, T), balanced, short rows never cut ----
    b = ex["chunk_b"].astype(np.int64)
    nc = int(st["n_chunks"])
    assert nc == (-(-T // W) if T else 0) and len(b) == nc + 1
    if nc:
        assert b[0] == 0 and b[-1] == T and np.all(np.diff(b) > 0), "chunk boundaries"
        sz = np.diff(b)
        assert np.all(2 * sz <= 3 * W), "a chunk exceeds 3W/2 merge items"
        assert np.all(2 * sz[:-1] >= W - 1), "a chunk below W/2 merge items"
        k0 = np.searchsorted(rs, b[:-1], side="right") - 1
        assert np.array_equal(ex["chunk_k0"].astype(np.int64), k0), "first row of a chunk"
    fc = np.searchsorted(b, rs[:-1], side="right") - 1 if len(rl) else np.zeros(0, np.int64)
    lc = np.searchsorted(b, rs[1:] - 1, side="right") - 1 if len(rl) else np.zeros(0, np.int64)
    short = 2 * (res_len[rl] + 1) <= W
    assert np.all(fc[short] == lc[short]), "a short residual row is cut by a chunk boundary"

    # ---- pieces: each output row is written by exactly its pieces, each piece to its slot ----
    npieces = (owned > 0).astype(np.int64)
    npieces[rl] += lc - fc + 1
    assert np.all(npieces >= 1), "a row no item writes"
    split = npieces >= 2
    rsp = ex["row_split"].astype(np.int64)
    n_split = int(split.sum())
    assert st["n_split"] == n_split
    assert np.array_equal(rsp, np.where(split, np.cumsum(split) - 1, -1)), "row -> split id"
    srow = ex["split_row"].astype(np.int64)
    assert np.array_equal(srow, np.nonzero(split)[0])
    snp = ex["split_np"].astype(np.int64)
    assert np.array_equal(snp, npieces[split]), "pieces per split row"
    slot = ex["split_slot"].astype(np.int64)
    assert np.array_equal(slot, np.concatenate([[0], np.cumsum(snp)[:-1]]) if n_split else slot)
    assert st["n_slots"] == int(snp.sum())
    # chunk c delivers piece c - split_base of its row; a dense window delivers piece 0.  The
    # pieces of a row must be exactly 0 .. np - 1, so its first chunk delivers piece `owned`.
    if n_split:
        fc_row = np.full(m, -1, np.int64)
        fc_row[rl] = fc
        first = fc_row[srow]
        own = (owned[srow] > 0).astype(np.int64)
        has_chunk = first >= 0
        assert np.array_equal(ex["split_base"].astype(np.int64)[has_chunk], (first - own)[has_chunk]), \
            "piece numbering of split rows"

    # ---- the work list: every item once, heaviest cost class (Eq. 1) first, then item id ----
    nq = -(-nc // G) if nc else 0
    n_items = len(dwin) + nq
    assert st["n_items"] == n_items
    q = ex["queue"].astype(np.int64)
    assert np.array_equal(np.sort(q), np.arange(n_items)), "work list is not a permutation"
    cost = ex["item_cost"].astype(np.int64)
    assert np.array_equal(cost[:len(dwin)], cost_dense), "dense item costs"
    if nq:
        ends = b[np.minimum((np.arange(nq) + 1) * G, nc)]
        assert np.array_equal(cost[len(dwin):], (ends - b[np.arange(nq) * G]) * tune["cost_res"])
    cls = _cost_class(cost[q]) if n_items else np.zeros(0, np.int64)
    assert np.all(np.diff(cls) <= 0), "work list not ordered by cost class"
    same = np.diff(cls) == 0
    assert np.all(np.diff(q)[same] > 0), "ties not in item order"


def tile_x_offsets(TM: int, TK: int) -> np.ndarray:
    """Element offset of (row r, column c) of a TM x TK tile in the expanded tile layout: 8 x 8
    blocks of 64 consecutive elements (8 rows of 8 columns), blocks of a row group side by side
    along the columns, row groups one after another."""
    r = np.arange(TM)[:, None]
    c = np.arange(TK)[None, :]
    return ((r // 8) * (TK // 8) * 64 + (c // 8) * 64 + (r % 8) * 8 + (c % 8)).reshape(-1)


def check_expanded_tiles(part: dict, x: np.ndarray) -> None:
    """BF16 plans: every dense tile expanded (zeros where the bitmap is clear) equals dtile_x."""
    nd, TM, TK = int(part["n_dtiles"]), int(part["TM"]), int(part["TK"])
    assert x.dtype == np.uint16 and x.size == nd * TM * TK, "expanded tiles: size"
    if nd == 0:
        return
    bits = np.unpackbits(part["dtile_bits"].reshape(nd, -1).view(np.uint8), axis=1, bitorder="little")
    bits = bits[:, :TM * TK].astype(bool)                      # bit r * TK + c
    rank = np.cumsum(bits, axis=1) - 1                         # value index inside the tile
    voff = part["dtile_voff"].astype(np.int64)[:-1]
    vals = part["dtile_vals"]
    dense = np.zeros((nd, TM * TK), np.uint16)
    dense[bits] = vals[(voff[:, None] + rank)[bits]]
    expect = np.zeros((nd, TM * TK), np.uint16)
    expect[:, tile_x_offsets(TM, TK)] = dense
    assert np.array_equal(x.reshape(nd, -1), expect), "expanded tiles differ from bitmap + values"


def compare_plan(plan, ref: dict, A: dict, tune) -> None:
    """The device plan's partition bit-exact with the oracle's, and its bookkeeping valid."""
    st = plan.stats()
    arrays = {name: plan.export(name) for name in oracle.PLAN_ARRAYS}
    compare_partition(st, arrays, ref)
    check_bookkeeping(A, ref, st, exports(plan), tune.as_dict())
    if st["b_bf16"]:
        check_expanded_tiles(ref, plan.export("dtile_x"))
