"""Hybrid path (dense tiles on the tensor cores + residual on the CUDA cores) against the FP64
oracle (GPU): plans with windows bit-exact with the CPU reference partition; FP32 (3xTF32)
within 1e-5 and BF16 within 2e-2 relative Frobenius error."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from nsutil import compare_plan, oracle_tune, to_dev, tune_from  # noqa: E402
from test_gpu_residual import run  # noqa: E402

F32, BF16 = ns.NS_F32, ns.NS_BF16
TOL = {F32: 1e-5, BF16: 2e-2}

CASES = [
    dict(tau_tile=1),
    dict(tau_tile=24),
    dict(tau_tile=128, TM=16, TK=16),
    dict(tau_tile=100, TM=32, TK=16, col_order=1),
    dict(tau_tile=200, TM=64, TK=16),
    dict(tau_tile=64, TM=16, TK=32, tau_row=4),
    dict(tau_tile=30, TM=16, TK=16, tau_col=1),
    dict(tau_tile=40, TM=16, TK=16, absorb_cap=0, chunk_nnz=16),   # split rows dense + residual
    dict(tau_tile=24, TM=16, TK=16, reorder=4),                     # Section 6.1 local reordering
    dict(tau_tile=100, TM=32, TK=16, reorder=2, tau_col=1),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("dtype", [F32, BF16])
def test_attention_like(ci, dtype):
    A = synth.block_sparse_csr(2048, seed=ci)
    B = synth.dense_b(2048, 64, seed=ci + 1)
    c, ref = run(A, B, dtype, tune=tune_from(ns, **CASES[ci]))
    assert oracle.rel_frobenius(c, ref) <= TOL[dtype]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_powerlaw_like(ci):
    A = synth.rmat_csr(12, 60000, seed=ci)
    B = synth.dense_b(A["n"], 32, seed=ci)
    c, ref = run(A, B, F32, tune=tune_from(ns, **CASES[ci]))
    assert oracle.rel_frobenius(c, ref) <= TOL[F32]


@pytest.mark.parametrize("K", [8, 16, 24, 64, 128, 256])
@pytest.mark.parametrize("dtype", [F32, BF16])
def test_widths_dense(K, dtype):
    A = synth.block_sparse_csr(1024, seed=K, band=2)
    B = synth.dense_b(1024, K, seed=3)
    TM = 64 if K <= 256 else 16
    c, ref = run(A, B, dtype, tune=tune_from(ns, tau_tile=16, TM=TM if K * TM <= 16384 else 16))
    assert oracle.rel_frobenius(c, ref) <= TOL[dtype]


def test_identity_exact_on_tensor_cores():
    # a tile of the identity holds one 1 per row: with BF16 B the products are exact
    A = synth.identity_csr(512)
    B = synth.dense_b(512, 64, seed=1)
    Bb = synth.bf16_bits(B)
    c, ref = run(A, Bb, BF16, tune=tune_from(ns, tau_tile=1))
    assert np.array_equal(c, ref.astype(np.float32))


def test_dense_only_and_residual_only_agree():
    A = synth.block_sparse_csr(1024, seed=3)
    B = synth.dense_b(1024, 128, seed=4)
    c_dense, ref = run(A, B, F32, tune=tune_from(ns, tau_tile=1))
    c_res, _ = run(A, B, F32, tune=tune_from(ns, tau_tile=ns.NS_TAU_INF), check_plan=False)
    assert oracle.rel_frobenius(c_dense, ref) <= 1e-5
    assert oracle.rel_frobenius(c_res, ref) <= 1e-6


def test_tm_k_limit():
    A = synth.block_sparse_csr(512, seed=0)
    with pytest.raises(ns.NsError) as e:
        ns.spmm_plan(to_dev(A, torch.device("cuda", 0)), 512, F32, tune_from(ns, tau_tile=8, TM=64))
    assert e.value.code == 2
