"""Epoch-level re-balance on the GPU (Section 5.3): the loop ends within 10 epochs, the per-class
spans come from the execute kernel's clocks, and C is the product A @ B."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from nsutil import to_dev, tune_from  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("which,dtype", [("attention", ns.NS_BF16), ("attention", ns.NS_F32), ("powerlaw", ns.NS_F32)])
def test_rebalance_loop(which, dtype):
    if which == "attention":
        A = synth.block_sparse_csr(4096, seed=3)
    else:
        A = synth.rmat_csr(14, 250000, seed=4)
    K = 64
    B = synth.dense_b(A["n"], K, seed=5)
    if dtype == ns.NS_BF16:
        Bh = synth.bf16_bits(B)
        Bt = torch.from_numpy(Bh.view(np.int16)).to(DEV).view(torch.bfloat16)
    else:
        Bh = B
        Bt = torch.from_numpy(B).to(DEV)
    C = torch.full((A["m"], K), float("nan"), device=DEV)
    start = tune_from(ns, TM=16, TK=16)
    t, rep = ns.rebalance(to_dev(A, DEV), K, dtype, Bt, C, start=start, eps=0.05, max_iter=10)
    torch.cuda.synchronize()
    assert 1 <= rep["iterations"] <= 10
    assert 1 <= t.tau_tile <= 16 * 16
    assert t.tau_tile in rep["tau"]
    # every epoch timed something: the residual class always has work or the dense class does
    for tc, res in zip(rep["dt_tc_ms"], rep["dt_res_ms"]):
        assert tc >= 0 and res >= 0 and max(tc, res) > 0
    # bisection: the visited taus never repeat
    assert len(set(rep["tau"])) == len(rep["tau"])
    # the loop keeps the threshold of the epoch that finished first (span = the later class's end)
    spans = [max(a, b) for a, b in zip(rep["dt_tc_ms"], rep["dt_res_ms"])]
    assert t.tau_tile == rep["tau"][int(np.argmin(spans))]
    # Eq. 6: converged exactly when some epoch's two classes ended within 1 + eps of each other
    # (a class with no work gives an unbounded skew); a small margin absorbs the eps rounding
    ratios = [max(a, b) / min(a, b) if min(a, b) > 0 else float("inf")
              for a, b in zip(rep["dt_tc_ms"], rep["dt_res_ms"])]
    if rep["converged"]:
        assert min(ratios) <= 1.05 + 1e-6
    else:
        assert min(ratios) > 1.05 - 1e-6
    tol = 2e-2 if dtype == ns.NS_BF16 else 1e-5
    ref = oracle.spmm(A, Bh, b_bf16=dtype == ns.NS_BF16)
    assert oracle.rel_frobenius(C.cpu().numpy(), ref) <= tol
