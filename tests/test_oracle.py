"""Pins of the FP64 oracle against mathematics and the paper (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong index,
a transposed operand, a wrong widening of BF16) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _dense(A):
    return A.to_dense()


@pytest.mark.parametrize("density", [0.0, 0.05, 0.3, 1.0])
@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (40, 33), (64, 64)])
def test_spmm_matches_dense_matmul(shape, density):
    m, n = shape
    A = synth.random_csr(m, n, density, seed=m * 100 + n + int(density * 10))
    B = synth.dense_b(n, 5, seed=3)
    ref = _dense(A) @ B.astype(np.float64)
    got = oracle.spmm(A, B)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_spmm_identity_exact():
    A = synth.identity_csr(50)
    B = synth.dense_b(50, 8, seed=1)
    assert np.array_equal(oracle.spmm(A, B), B.astype(np.float64))


def test_spmm_permutation_exact():
    A, perm = synth.permutation_csr(97, seed=5)
    B = synth.dense_b(97, 16, seed=2)
    assert np.array_equal(oracle.spmm(A, B), B[perm].astype(np.float64))


def test_spmm_transposed_operand_would_fail():
    # a non-square, non-symmetric case: A^T B has another shape, A B^T another value
    A = synth.random_csr(9, 4, 0.6, seed=11, values="int")
    B = synth.dense_b(4, 3, seed=7)
    ref = _dense(A) @ B.astype(np.float64)
    assert oracle.spmm(A, B).shape == (9, 3)
    np.testing.assert_allclose(oracle.spmm(A, B), ref, rtol=0, atol=1e-12)


def test_row_sums_with_ones():
    A = synth.random_csr(60, 45, 0.2, seed=4)
    ones = np.ones((45, 3), dtype=np.float32)
    got = oracle.spmm(A, ones)
    for i in range(60):
        s = math.fsum(float(x) for x in A["vals"][A["rowptr"][i]:A["rowptr"][i + 1]])
        assert abs(got[i, 0] - s) <= 1e-12 * max(1.0, abs(s))
        assert got[i, 0] == got[i, 1] == got[i, 2]


def test_row_normalised_attention_rows_sum_to_one():
    A = synth.block_sparse_csr(1024, seed=0)
    ones = np.ones((1024, 1), dtype=np.float32)
    got = oracle.spmm(A, ones)[:, 0]
    lens = np.diff(A["rowptr"].astype(np.int64))
    # values were rounded to float32 after normalisation: |sum - 1| <= len * 2^-24 (+ fp64 sum)
    assert np.all(np.abs(got - 1.0) <= lens * 2.0 ** -24 + 1e-12)


def test_reorder_invariance():
    rng = np.random.default_rng(0)
    A = synth.random_csr(30, 20, 0.25, seed=8)
    B = synth.dense_b(20, 4, seed=9)
    p = rng.permutation(30)
    q = rng.permutation(20)
    D = _dense(A)
    PAQt = D[p][:, q]
    r, c = np.nonzero(PAQt)
    A2 = synth.csr_from_coo(30, 20, r, c, PAQt[r, c].astype(np.float32))
    QB = B[q]
    lhs = oracle.spmm(A2, QB)
    rhs = oracle.spmm(A, B)[p]
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_bf16_widening_is_exact():
    A = synth.random_csr(20, 30, 0.3, seed=1)
    B = synth.dense_b(30, 6, seed=2)
    Bb = synth.bf16_bits(B)
    Bf = (Bb.astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(oracle.spmm(A, Bb, b_bf16=True), oracle.spmm(A, Bf))


def test_bf16_rne_matches_library_cast():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(4096).astype(np.float32),
        rng.uniform(-1, 1, 4096).astype(np.float32) * 1e-30,
        # exact ties: low half 0x8000 with even and odd kept bit
        (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x00008000, 0x7F7F8000], dtype=np.uint32)).view(np.float32),
        np.array([0.0, -0.0, 1.0, 65504.0, 3.4e38], dtype=np.float32),
    ])
    assert np.array_equal(oracle.bf16_rne(x), synth.bf16_bits(x))


def test_threaded_spmm_identical():
    A = synth.uniform_csr(500, 300, 12, seed=2)
    B = synth.dense_b(300, 16, seed=1)
    assert np.array_equal(oracle.spmm(A, B), oracle.spmm(A, B, threads=4))
    rows = np.array([499, 0, 17, 17], dtype=np.int32)
    assert np.array_equal(oracle.spmm(A, B, rows=rows), oracle.spmm(A, B)[rows])


def test_spmm_empty_matrix_and_empty_rows():
    A = synth.random_csr(10, 10, 0.0, seed=0)
    B = synth.dense_b(10, 4, seed=0)
    assert np.count_nonzero(oracle.spmm(A, B)) == 0
    A = synth.random_csr(50, 40, 0.3, seed=1, empty_rows=0.5)
    B = synth.dense_b(40, 4, seed=0)
    got = oracle.spmm(A, B)
    lens = np.diff(A["rowptr"])
    assert np.all(got[lens == 0] == 0.0)
    assert (lens == 0).sum() > 5


def test_rel_frobenius():
    ref = np.array([[3.0, 4.0]])
    assert oracle.rel_frobenius(ref, ref) == 0.0
    assert abs(oracle.rel_frobenius(np.array([[3.0, 4.5]]), ref) - 0.1) < 1e-15
    assert oracle.rel_frobenius(np.zeros((1, 2)), np.zeros((1, 2))) == 0.0
    assert oracle.rel_frobenius(np.ones((1, 2)), np.zeros((1, 2))) == float("inf")
