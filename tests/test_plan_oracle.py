"""Pins of the CPU reference partition (CPU only).

* the C planner equals the pure-Python brute-force planner on tiny inputs, for many tunes;
* partition invariants hold (every nonzero exactly once, reconstruction, thresholds, window
  coverage, the row extraction rule);
* the product evaluated from the plan equals the SpMM definition;
* the paper's closed forms (Eq. 1-3, 6, 8 and the tile-shape worked numbers).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import bruteforce, formulas

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.TAU_INF


def _cmp_plans(a, b):
    for k in oracle.PLAN_SCALARS:
        if k in b:
            assert a[k] == b[k], k
    for k in oracle.PLAN_ARRAYS:
        if k in b:
            x, y = np.asarray(a[k]), np.asarray(b[k])
            assert x.shape == y.shape, (k, x.shape, y.shape)
            assert np.array_equal(x.view(np.uint8) if x.dtype == np.float32 else x,
                                  y.view(np.uint8) if y.dtype == np.float32 else y), k


TINY_TUNES = [
    dict(tau_tile=INF),
    dict(tau_tile=1),
    dict(tau_tile=3, TM=16, TK=16),
    dict(tau_tile=6, TM=32, TK=16, col_order=1),
    dict(tau_tile=2, TM=16, TK=32, tau_row=2),
    dict(tau_tile=2, TM=16, TK=16, tau_col=1),
    dict(tau_tile=4, TM=64, TK=16),
    dict(tau_tile=5, TM=16, TK=16),
    dict(tau_tile=6, TM=16, TK=16, tau_row=3),
    dict(tau_tile=12, TM=16, TK=16, tau_row=1, col_order=1),
    dict(tau_tile=3, TM=16, TK=16, reorder=1),
    dict(tau_tile=2, TM=16, TK=16, reorder=3, tau_col=1),
    dict(tau_tile=5, TM=32, TK=16, reorder=2, tau_row=1),
    dict(tau_tile=9, TM=32, TK=32, tau_col=2, col_order=1),
]


@pytest.mark.parametrize("ti", range(len(TINY_TUNES)))
@pytest.mark.parametrize("case", ["random", "hubs", "empty", "dense", "band"])
def test_c_planner_equals_bruteforce(case, ti):
    tune = TINY_TUNES[ti]
    if case == "random":
        A = synth.random_csr(70, 90, 0.08, seed=ti)
    elif case == "hubs":
        A = synth.random_csr(100, 60, 0.03, seed=ti, hub_rows=3, empty_rows=0.2)
    elif case == "empty":
        A = synth.random_csr(33, 20, 0.0, seed=ti)
    elif case == "dense":
        A = synth.random_csr(40, 24, 0.9, seed=ti)
    else:
        A = synth.block_sparse_csr(256, seed=ti, block=16, band=2, p_random=0.05)
    for b_bf16 in (False, True):
        c = oracle.plan(A, 8, b_bf16=b_bf16, **tune)
        p = bruteforce.plan(A, 8, b_bf16=b_bf16, **tune)
        _cmp_plans(c, p)


def _check_invariants(A, P):
    m, n = A["m"], A["n"]
    t = P["tune"]
    TM, TK, tau = P["TM"], P["TK"], t["tau_tile"]
    rp, ci, v = A["rowptr"], A["colidx"], A["vals"].astype(np.float32)
    BW = TM * TK // 32
    # windows cover the kept rows exactly once, in order
    wr = P["win_rows"]
    valid = wr[wr >= 0]
    assert np.array_equal(valid, P["aic_rows"])
    if P["n_win"]:
        assert np.all(wr[: P["m_aic"]] >= 0) and np.all(wr[P["m_aic"]:] == -1)
    # every element appears exactly once across dense tiles and residual; values preserved
    seen = {}
    bits = P["dtile_bits"].reshape(-1, BW) if P["n_dtiles"] else np.zeros((0, BW), np.uint32)
    cols = P["dtile_cols"].reshape(-1, TK) if P["n_dtiles"] else np.zeros((0, TK), np.int32)
    win_of_tile = np.repeat(np.arange(P["n_win"]), np.diff(P["win_dptr"]))
    dv = P["dtile_vals"]
    for d in range(P["n_dtiles"]):
        w = win_of_tile[d]
        k = P["dtile_voff"][d]
        cnt = 0
        for bit in range(TM * TK):
            if (bits[d, bit // 32] >> (bit % 32)) & 1:
                i = wr[w * TM + bit // TK]
                j = cols[d, bit % TK]
                assert i >= 0 and j >= 0
                assert (i, j) not in seen
                seen[(i, j)] = dv[k]
                k += 1
                cnt += 1
        assert cnt >= tau                                      # dense tile rule
        assert P["dtile_voff"][d + 1] - P["dtile_voff"][d] == -(-cnt // 8) * 8
        assert np.all(dv[k:P["dtile_voff"][d + 1]] == 0)       # zero padding
    rrp = P["res_rowptr"]
    for i in range(m):
        for z in range(rrp[i], rrp[i + 1]):
            key = (i, int(P["res_col"][z]))
            assert key not in seen
            seen[key] = P["res_val"][z]
        assert np.all(np.diff(P["res_col"][rrp[i]:rrp[i + 1]]) > 0)
    assert len(seen) == A.nnz
    for i in range(m):
        for p in range(rp[i], rp[i + 1]):
            got = seen[(i, int(ci[p]))]
            if isinstance(got, np.uint16):
                assert got == oracle.bf16_rne(np.array([v[p]]))[0]
            else:
                assert np.float32(got).view(np.uint32) == v[p].view(np.uint32)
    # the row-window list: windows with at least one dense tile
    assert P["n_dwin"] == int(np.count_nonzero(np.diff(P["win_dptr"]))) if P["n_win"] else P["n_dwin"] == 0
    # rows extracted by the row stage are exactly the rows with Len <= tau_row (Eq. 5)
    if tau != INF:
        lens = np.diff(rp)
        assert np.array_equal(np.sort(P["aic_rows"]), np.nonzero(lens > t["tau_row"])[0])
    else:
        assert P["m_aic"] == 0 and P["n_res"] == A.nnz


def _plan_product(A, P, B, b_bf16=False):
    """C from the plan: dense tiles (values as stored) plus the residual, float64."""
    m, K = A["m"], B.shape[1]
    Bd = ((B.astype(np.uint32) << 16).view(np.float32) if b_bf16 else B).astype(np.float64)
    C = np.zeros((m, K))
    TM, TK = P["TM"], P["TK"]
    BW = TM * TK // 32
    win_of_tile = np.repeat(np.arange(P["n_win"]), np.diff(P["win_dptr"]))
    dv = P["dtile_vals"]
    if b_bf16:
        dv = (dv.astype(np.uint32) << 16).view(np.float32)
    for d in range(P["n_dtiles"]):
        w = win_of_tile[d]
        k = P["dtile_voff"][d]
        bits = P["dtile_bits"][d * BW:(d + 1) * BW]
        for bit in range(TM * TK):
            if (bits[bit // 32] >> (bit % 32)) & 1:
                i = P["win_rows"][w * TM + bit // TK]
                j = P["dtile_cols"][d * TK + bit % TK]
                C[i] += float(dv[k]) * Bd[j]
                k += 1
    rrp = P["res_rowptr"]
    for i in range(m):
        for z in range(rrp[i], rrp[i + 1]):
            C[i] += float(P["res_val"][z]) * Bd[P["res_col"][z]]
    return C


MED_TUNES = [dict(tau_tile=INF), dict(tau_tile=1), dict(tau_tile=24, TM=16, TK=16),
             dict(tau_tile=200, TM=32, TK=16, tau_row=4),
             dict(tau_tile=64, TM=64, TK=32, tau_col=1, col_order=1),
             dict(tau_tile=24, TM=16, TK=16, reorder=4)]


@pytest.mark.parametrize("ti", range(len(MED_TUNES)))
def test_invariants_and_product_medium(ti):
    tune = MED_TUNES[ti]
    mats = [synth.uniform_csr(300, 300, 16, seed=1),
            synth.block_sparse_csr(512, seed=2),
            synth.rmat_csr(9, 4000, seed=3)]
    for A in mats:
        for b_bf16 in (False, True):
            P = oracle.plan(A, 16, b_bf16=b_bf16, **tune)
            _check_invariants(A, P)
            B = synth.dense_b(A["n"], 16, seed=4)
            Bx = synth.bf16_bits(B) if b_bf16 else B
            got = _plan_product(A, P, Bx, b_bf16)
            if b_bf16:
                # dense-tile values are RNE(A); compare with the definition on that matrix
                A2 = synth.Csr(A)
                vals = A["vals"].copy()
                A2["vals"] = vals
                dense_mask = np.ones(A.nnz, bool)
                rrp = P["res_rowptr"]
                for i in range(A["m"]):
                    cols_res = set(P["res_col"][rrp[i]:rrp[i + 1]].tolist())
                    for p in range(A["rowptr"][i], A["rowptr"][i + 1]):
                        if int(A["colidx"][p]) in cols_res:
                            dense_mask[p] = False
                vals[dense_mask] = (oracle.bf16_rne(vals[dense_mask]).astype(np.uint32) << 16).view(np.float32)
                ref = oracle.spmm(A2, Bx, b_bf16=True)
            else:
                ref = oracle.spmm(A, Bx)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_tau_extremes():
    A = synth.block_sparse_csr(512, seed=5)
    P = oracle.plan(A, 8, tau_tile=INF)
    assert P["n_dtiles"] == 0 and P["n_win"] == 0
    assert np.array_equal(P["res_rowptr"], A["rowptr"]) and np.array_equal(P["res_col"], A["colidx"])
    P = oracle.plan(A, 8, tau_tile=1)
    assert P["n_res"] == 0                       # no extraction: everything lands in tiles
    P = oracle.plan(A, 8, tau_tile=1, tau_row=10 ** 6)
    assert P["n_dtiles"] == 0 and P["n_res"] == A.nnz   # every row extracted


def test_attention_windows_are_full_tiles():
    # a 64-row block row with 16-row windows: every band/random block column has count 16,
    # so COUNT_DESC puts them first and the scattered singletons last
    A = synth.block_sparse_csr(2048, seed=1)
    P = oracle.plan(A, 8, tau_tile=128, TM=16, TK=16)
    nb = np.diff(P["dtile_voff"])
    assert np.all(nb == 256)                          # only full 16x16 tiles are dense
    assert P["n_res"] == A["m"]                       # one scattered nonzero per row remains
    assert np.array_equal(np.diff(P["res_rowptr"]), np.ones(A["m"], np.int32))
    assert P["n_dwin"] == P["n_win"] == A["m"] // 16  # every window holds dense tiles


def test_invalid_csr_rejected():
    A = synth.random_csr(10, 10, 0.5, seed=0)
    bad = synth.Csr(A)
    bad["colidx"] = A["colidx"].copy()
    i = int(np.argmax(np.diff(A["rowptr"]) >= 2))
    p = A["rowptr"][i]
    bad["colidx"][p], bad["colidx"][p + 1] = A["colidx"][p + 1], A["colidx"][p]
    with pytest.raises(oracle.PlanError):
        oracle.plan(bad, 4)
    dup = synth.Csr(A)
    dup["colidx"] = A["colidx"].copy()
    dup["colidx"][p + 1] = dup["colidx"][p]
    with pytest.raises(oracle.PlanError):
        oracle.plan(dup, 4)
    oor = synth.Csr(A)
    oor["colidx"] = A["colidx"].copy()
    oor["colidx"][-1] = 10
    with pytest.raises(oracle.PlanError):
        oracle.plan(oor, 4)
    nm = synth.Csr(A)
    nm["rowptr"] = A["rowptr"].copy()
    nm["rowptr"][3] = nm["rowptr"][4] + 1
    with pytest.raises(oracle.PlanError):
        oracle.plan(nm, 4)
    with pytest.raises(oracle.PlanError):
        oracle.plan(A, 4, TM=24)


# ---------------------------------------------------------------------------------------
# the paper's closed forms
# ---------------------------------------------------------------------------------------

def test_tile_shape_worked_numbers():
    g = json.load(open(os.path.join(GOLD, "paper_tile_shape.json")))
    buf = g["buffers_bytes"]
    mk, nk, mn = formulas.l0_limits(buf["L0A"], buf["L0B"], buf["L0C"])
    assert (mk, nk, mn) == (g["limits"]["MK"], g["limits"]["NK"], g["limits"]["MN"])
    for key, val in g["input_traffic_bytes"].items():
        M, N, K = map(int, key.split(","))
        assert formulas.tile_input_bytes(M, N, K) == val
    M, N, K = g["final_tile_MNK"]
    assert formulas.tile_fits(M, N, K, buf["L0A"], buf["L0B"], buf["L0C"])
    assert M * N * K == 128 * 128 * 128                       # same MNK as (128,128,128)
    assert not formulas.tile_fits(128, g["max_N_at_M128"] + 16, 64, buf["L0A"], buf["L0B"], buf["L0C"])
    best = max((M2 * N2 * K2, (M2, N2, K2)) for (M2, N2, K2) in g["alternatives_MNK"] + [g["final_tile_MNK"]]
               if formulas.tile_fits(M2, N2, K2, buf["L0A"], buf["L0B"], buf["L0C"]))
    assert best[0] == 128 ** 3


def test_cost_model_and_threshold():
    g = json.load(open(os.path.join(GOLD, "paper_coordination.json")))
    r = g["r_ascend"]
    p_vec, p_mat = 3.0e9, 6.0e12
    a = formulas.alpha(p_vec, p_mat, r)
    assert a == pytest.approx(2 * 3.0e9 / 6.0e12)
    # Eq. 2: the minimiser balances Cost_vec(NNZ*) = r * Cost_mat
    M, K = 128, 64
    ns = formulas.nnz_star(M, K, p_vec, p_mat, r)
    assert formulas.cost_vector(ns, p_vec) == pytest.approx(r * formulas.cost_matrix(M, K, p_mat))
    assert ns / (M * K) == pytest.approx(a)
    # brute-force minimisation of Eq. 2 over integer NNZ agrees with the closed form
    cands = np.arange(0, M * K + 1)
    obj = (cands / p_vec / (M * K / p_mat) - r) ** 2
    assert abs(int(np.argmin(obj)) - ns) <= 1
    assert formulas.len_threshold(g["alpha_default"], 1000) == pytest.approx(2.0)
    assert formulas.tau_tile(g["alpha_default"], 16, 16) == 1
    assert formulas.tau_tile(0.1, 16, 16) == 26


def test_skew_rule():
    eps = json.load(open(os.path.join(GOLD, "paper_coordination.json")))["epsilon"]
    assert formulas.skew(2.0, 1.0) == formulas.skew(1.0, 2.0) == 2.0
    assert formulas.skew(1.0, 1.0) == 1.0
    assert not formulas.needs_migration(1.04, 1.0, eps)
    assert formulas.needs_migration(1.06, 1.0, eps)
    assert formulas.migration_direction(2.0, 1.0) == "to_vector"
    assert formulas.migration_direction(1.0, 2.0) == "to_matrix"


def test_redundancy_metric_small_cases():
    a = np.zeros((8, 8))
    a[0, 0] = 1
    assert formulas.redundant_zero_fraction(a, 4) == 15 / 16
    assert formulas.redundant_zero_fraction(np.ones((8, 8)), 4) == 0.0
    a[7, 7] = 1
    assert formulas.redundant_zero_fraction(a, 8) == 62 / 64


def test_algorithmic_bytes_and_flops():
    assert formulas.spmm_flops(10, 4) == 80
    assert formulas.algorithmic_bytes(2, 3, 4, 2, 4) == 4 * 3 + 8 * 3 + 4 * 4 * 2 + 4 * 2 * 4


def _two_patterns(m=64, width=16):
    """Rows alternate between columns [0, width) and [width, 2 width), all values 1."""
    rows = [list(range(0, width)) if i % 2 == 0 else list(range(width, 2 * width)) for i in range(m)]
    rowptr = np.zeros(m + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.array([c for r in rows for c in r], dtype=np.int32)
    return dict(m=m, n=2 * width, rowptr=rowptr, colidx=colidx, vals=np.ones(len(colidx), np.float32))


def test_local_reorder_groups_alike_rows():
    # Section 6.1 local stage: interleaved patterns give half-full tiles in row order; the
    # Jaccard rebuild puts each pattern's rows in windows of their own, so every tile is full
    A = _two_patterns()
    plain = oracle.plan(A, 16, tau_tile=200, TM=16, TK=16)
    re = oracle.plan(A, 16, tau_tile=200, TM=16, TK=16, reorder=4)
    assert plain["n_dtiles"] == 0
    assert re["n_dtiles"] == 4
    w = re["win_rows"].reshape(-1, 16)
    assert all(len(set(int(i) % 2 for i in win)) == 1 for win in w)   # one pattern per window
    # the anchor leads each window, then the equal-similarity rows in their current order
    assert list(w[0]) == list(range(0, 32, 2))
    assert sorted(re["aic_rows"].tolist()) == sorted(plain["aic_rows"].tolist())


@pytest.mark.parametrize("seed", range(4))
def test_local_reorder_permutes_within_clusters(seed):
    A = synth.random_csr(300, 120, 0.05, seed=seed)
    for TM, R in ((16, 1), (16, 3), (32, 2)):
        plain = oracle.plan(A, 16, tau_tile=8, TM=TM, TK=16)["aic_rows"]
        re = oracle.plan(A, 16, tau_tile=8, TM=TM, TK=16, reorder=R)["aic_rows"]
        cl = R * TM
        for c0 in range(0, len(plain), cl):
            assert sorted(re[c0:c0 + cl].tolist()) == sorted(plain[c0:c0 + cl].tolist())
            assert re[c0] == plain[c0]          # the first window keeps its anchor
