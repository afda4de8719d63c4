"""Full-size workloads in the benchmark's launch configuration (GPU): plans bit-exact with the
CPU reference partition; outputs checked on sampled rows (uniform sample plus the longest rows)
against the FP64 oracle, which computes those rows one by one."""
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

DEV = torch.device("cuda", 0)


def sample_rows(A, k=3000, seed=0):
    rng = np.random.default_rng(seed)
    lens = np.diff(A["rowptr"].astype(np.int64))
    top = np.argsort(-lens)[:64]
    rows = np.unique(np.concatenate([rng.choice(A["m"], size=k, replace=False), top,
                                     np.nonzero(lens == 0)[0][:32], [0, A["m"] - 1]]))
    return rows.astype(np.int32)


def check(A, B, dtype, tune, tol, plan_check=True):
    At = to_dev(A, DEV)
    K = B.shape[1]
    if dtype == ns.NS_BF16:
        Bh = synth.bf16_bits(B)
        Bt = torch.from_numpy(Bh.view(np.int16)).to(DEV).view(torch.bfloat16)
    else:
        Bh = B
        Bt = torch.from_numpy(B).to(DEV)
    C = torch.full((A["m"], K), float("nan"), device=DEV)
    with ns.spmm_plan(At, K, dtype, tune) as p:
        if plan_check:
            compare_plan(p, oracle.plan(A, K, b_bf16=dtype == ns.NS_BF16, **oracle_tune(tune)))
        p.execute(Bt, C)
        torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    assert not np.isnan(Ch).any()
    rows = sample_rows(A)
    ref = oracle.spmm(A, Bh, rows=rows, b_bf16=dtype == ns.NS_BF16, threads=8)
    err = oracle.rel_frobenius(Ch[rows], ref)
    assert err <= tol, err
    return Ch


@pytest.fixture(scope="module")
def powerlaw():
    return synth.config_powerlaw(0)


def test_powerlaw_residual_full(powerlaw):
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=ns.NS_TAU_INF), 1e-5)


def test_powerlaw_hybrid_full(powerlaw):
    A, B = powerlaw
    check(A, B, ns.NS_F32, tune_from(ns, tau_tile=48, tau_row=32, TM=16), 1e-5)


def test_destroy_right_after_async_execute(powerlaw):
    # the benchmark's pattern: plan, execute, destroy with no synchronisation in between
    A, B = powerlaw
    At = to_dev(A, DEV)
    Bt = torch.from_numpy(B).to(DEV)
    C = torch.empty((A["m"], 128), device=DEV)
    for _ in range(4):
        p = ns.spmm_plan(At, 128, ns.NS_F32)
        p.execute(Bt, C)
        p.close()
    torch.cuda.synchronize()
    rows = sample_rows(A, 500, seed=2)
    err = oracle.rel_frobenius(C.cpu().numpy()[rows], oracle.spmm(A, B, rows=rows, threads=8))
    assert err <= 1e-5


@pytest.mark.parametrize("dtype,tol", [(ns.NS_F32, 1e-5), (ns.NS_BF16, 2e-2)])
def test_attention_full(dtype, tol):
    A, B = synth.config_attention(0)
    check(A, B, dtype, tune_from(ns, tau_tile=128, TM=16, TK=16), tol)


@pytest.mark.parametrize("dtype,tol", [(ns.NS_F32, 1e-5), (ns.NS_BF16, 2e-2)])
def test_attention_residual_full(dtype, tol):
    # all of A on the CUDA cores; B (16 MiB) fits in L2, so the FP32 form gathers through the
    # register ring rather than the shared-memory ring the power-law B (512 MiB) takes
    A, B = synth.config_attention(0)
    check(A, B, dtype, tune_from(ns, tau_tile=ns.NS_TAU_INF), tol)


def test_small_config_full():
    A, B = synth.config_small(0)
    C = check(A, B, ns.NS_F32, ns.tune_default(), 1e-5)
    assert oracle.rel_frobenius(C, oracle.spmm(A, B)) <= 1e-6
