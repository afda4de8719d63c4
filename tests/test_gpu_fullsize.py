"""Full-size workloads in the benchmark's launch configuration (GPU): the plan's partition
bit-exact with the CPU reference partition and its bookkeeping valid; EVERY row of C compared
with the FP64 oracle (relative Frobenius error, element-wise dot-product error bound, exact
zeros), with the per-row maximum relative error reported."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from nsutil import compare_plan, oracle_tune, to_dev, tune_from  # noqa: E402
from parity import check_result  # noqa: E402

DEV = torch.device("cuda", 0)
THREADS = max(1, min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 8))


def _report(name, rep):
    print(f"\n[parity] {name}: " + json.dumps(rep))


def check(A, B, dtype, tune, tol, plan_check=True, name=""):
    At = to_dev(A, DEV)
    K = B.shape[1]
    bf16 = dtype == ns.NS_BF16
    if bf16:
        Bh = synth.bf16_bits(B)
        Bt = torch.from_numpy(Bh.view(np.int16)).to(DEV).view(torch.bfloat16)
    else:
        Bh = B
        Bt = torch.from_numpy(B).to(DEV)
    C = torch.full((A["m"], K), float("nan"), device=DEV)
    with ns.spmm_plan(At, K, dtype, tune) as p:
        if plan_check:
            compare_plan(p, oracle.plan(A, K, b_bf16=bf16, **oracle_tune(tune)), A, tune)
        dense = p.stats()["n_dtiles"] > 0
        p.execute(Bt, C)
        torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    assert not np.isnan(Ch).any(), "rows left unwritten"
    rep = check_result(Ch, A, Bh, b_bf16=bf16, bf16_tiles=bf16 and dense, tol=tol, threads=THREADS)
    _report(name, rep)
    return Ch, rep


@pytest.fixture(scope="module")
def powerlaw():
    return synth.config_powerlaw(0)


def test_powerlaw_residual_full(powerlaw):
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=ns.NS_TAU_INF), 1e-5, name="powerlaw residual")


def test_powerlaw_bench_chunk_full(powerlaw):
    # the benchmark's autotuned chunk size on this graph (W = 512)
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=ns.NS_TAU_INF, chunk_nnz=512, absorb_cap=512), 1e-5,
          name="powerlaw residual W512")


def test_powerlaw_hot_rows_l2_full(powerlaw):
    # Section 6.2.1 hot-B staging: only the most gathered B rows keep the evict-last policy
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=ns.NS_TAU_INF, l2_hints=2), 1e-5, name="powerlaw hot-B")


def test_powerlaw_hybrid_full(powerlaw):
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=48, tau_row=32, TM=16), 1e-5, name="powerlaw hybrid")


def test_destroy_right_after_async_execute(powerlaw):
    # the benchmark's pattern: plan, execute, destroy with no synchronisation in between
    A, B = powerlaw
    At = to_dev(A, DEV)
    Bt = torch.from_numpy(B).to(DEV)
    C = torch.full((A["m"], 128), float("nan"), device=DEV)
    for _ in range(4):
        p = ns.spmm_plan(At, 128, ns.NS_F32)
        p.execute(Bt, C)
        p.close()
    torch.cuda.synchronize()
    check_result(C.cpu().numpy(), A, B, tol=1e-5, threads=THREADS)


@pytest.mark.parametrize("dtype,tol", [(ns.NS_F32, 1e-5), (ns.NS_BF16, 2e-2)])
def test_attention_full(dtype, tol):
    A, B = synth.config_attention(0)
    check(A, B, dtype, tune_from(ns, tau_tile=128, TM=16, TK=16), tol, name=f"attention hybrid {dtype}")


@pytest.mark.parametrize("dtype,tol", [(ns.NS_F32, 1e-5), (ns.NS_BF16, 2e-2)])
def test_attention_residual_full(dtype, tol):
    # all of A on the CUDA cores; B (16 MiB) fits in L2, so the FP32 form gathers through the
    # register ring rather than the shared-memory ring the power-law B (512 MiB) takes
    A, B = synth.config_attention(0)
    check(A, B, dtype, tune_from(ns, tau_tile=ns.NS_TAU_INF), tol, name=f"attention residual {dtype}")


def test_small_config_full():
    A, B = synth.config_small(0)
    C, rep = check(A, B, ns.NS_F32, ns.tune_default(), 1e-5, name="small")
    assert rep["rel_frobenius"] <= 1e-6
