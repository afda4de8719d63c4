"""The result checker itself (CPU only): a correct FP32 product in another summation order passes;
an error above the dot-product bound, a non-zero empty row and BF16-rounded tiles checked as
FP32 are all caught."""
import numpy as np
import pytest

import synth
from parity import check_result


def _fp32_product(A, B, reverse=True, vals=None):
    """C = A B accumulated in float32, nonzeros of a row taken in reverse order."""
    rp, ci = A["rowptr"], A["colidx"]
    v = A["vals"] if vals is None else vals
    C = np.zeros((A["m"], B.shape[1]), np.float32)
    for i in range(A["m"]):
        ps = range(rp[i + 1] - 1, rp[i] - 1, -1) if reverse else range(rp[i], rp[i + 1])
        acc = np.zeros(B.shape[1], np.float32)
        for p in ps:
            acc = (acc + np.float32(v[p]) * B[ci[p]]).astype(np.float32)
        C[i] = acc
    return C


@pytest.fixture(scope="module")
def case():
    A = synth.random_csr(120, 90, 0.2, seed=3, hub_rows=2, empty_rows=0.1)
    B = synth.dense_b(90, 16, seed=4)
    return A, B


def test_fp32_other_order_passes(case):
    A, B = case
    rep = check_result(_fp32_product(A, B), A, B, tol=1e-5, threads=1, block=37)
    assert rep["rows"] == A["m"] and rep["max_bound_ratio"] <= 1.0 and rep["rel_frobenius"] < 1e-6


def test_error_above_bound_caught(case):
    A, B = case
    C = _fp32_product(A, B)
    i = int(np.argmax(np.diff(A["rowptr"])))
    C[i, 3] += 1e-3 * max(abs(C[i, 3]), 1.0)
    with pytest.raises(AssertionError, match="bound"):
        check_result(C, A, B, tol=1.0, threads=1)


def test_nonzero_empty_row_caught(case):
    A, B = case
    C = _fp32_product(A, B)
    i = int(np.nonzero(np.diff(A["rowptr"]) == 0)[0][0])
    C[i, 0] = 1e-30
    with pytest.raises(AssertionError, match="zero"):
        check_result(C, A, B, tol=1.0, threads=1)


def test_bf16_tiles_need_their_allowance(case):
    A, B = case
    import oracle
    vb = (oracle.bf16_rne(A["vals"]).astype(np.uint32) << 16).view(np.float32)
    C = _fp32_product(A, B, vals=vb)            # every value rounded, as in a BF16 dense tile
    check_result(C, A, B, bf16_tiles=True, tol=2e-2, threads=1)
    with pytest.raises(AssertionError):
        check_result(C, A, B, bf16_tiles=False, tol=2e-2, threads=1)


def test_expanded_tile_check_on_the_oracle_partition():
    # the expanded-tile layout check, on an expansion written here element by element
    import oracle
    from plan_checks import check_expanded_tiles
    A = synth.block_sparse_csr(256, seed=4, block=16, band=2, p_random=0.1)
    for TM, TK in ((16, 16), (32, 16), (16, 32), (64, 32)):
        P = oracle.plan(A, 16, b_bf16=True, tau_tile=40, TM=TM, TK=TK)
        nd, BW = P["n_dtiles"], TM * TK // 32
        assert nd > 0
        x = np.zeros(nd * TM * TK, np.uint16)
        for d in range(nd):
            k = P["dtile_voff"][d]
            for r in range(TM):
                for c in range(TK):
                    bit = r * TK + c
                    if (P["dtile_bits"][d * BW + bit // 32] >> (bit % 32)) & 1:
                        off = (r // 8) * (TK // 8) * 64 + (c // 8) * 64 + (r % 8) * 8 + c % 8
                        x[d * TM * TK + off] = P["dtile_vals"][k]
                        k += 1
        check_expanded_tiles(P, x)
        x[7] ^= 1
        with pytest.raises(AssertionError):
            check_expanded_tiles(P, x)
