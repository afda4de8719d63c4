"""Batched form (one persistent launch from a CUDA graph over many uneven graphs) and the
autotuner, against the FP64 oracle (GPU)."""
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


@pytest.mark.parametrize("tau", [ns.NS_TAU_INF, 24])
def test_batch_matches_oracle_and_replays(tau):
    graphs = synth.batch_graphs(24, seed=5, n_lo=200, n_hi=6000)
    K = 64
    rng = np.random.default_rng(1)
    Bs = [rng.standard_normal((g["n"], K), dtype=np.float32) for g in graphs]
    Ad = [to_dev(g, DEV) for g in graphs]
    Bd = [torch.from_numpy(b).to(DEV) for b in Bs]
    Cd = [torch.full((g["m"], K), float("nan"), device=DEV) for g in graphs]
    bt = ns.Batch(Ad, [K] * len(graphs), ns.NS_F32, tune_from(ns, tau_tile=tau))
    assert bt.stats()["n_graphs"] == len(graphs)
    launches = ns.launch_count()
    bt.execute(Bd, Cd)
    torch.cuda.synchronize()
    assert ns.launch_count() - launches == 1          # one persistent launch for all graphs
    first = [c.cpu().numpy() for c in Cd]
    for g, b, c in zip(graphs, Bs, first):
        assert oracle.rel_frobenius(c, oracle.spmm(g, b)) <= 1e-5
    bt.execute(Bd, Cd)                                 # graph replay
    torch.cuda.synchronize()
    for c0, c in zip(first, Cd):
        assert np.array_equal(c0, c.cpu().numpy())
    Cd2 = [torch.zeros_like(c) for c in Cd]           # new output pointers refresh the table
    bt.execute(Bd, Cd2)
    torch.cuda.synchronize()
    for c0, c in zip(first, Cd2):
        assert np.array_equal(c0, c.cpu().numpy())
    bt.close()


def test_batch_autotune_picks_a_chunk_size():
    graphs = synth.batch_graphs(12, seed=9, n_lo=300, n_hi=5000)
    K = 64
    rng = np.random.default_rng(3)
    Bs = [rng.standard_normal((g["n"], K), dtype=np.float32) for g in graphs]
    Ad = [to_dev(g, DEV) for g in graphs]
    Bd = [torch.from_numpy(b).to(DEV) for b in Bs]
    Cd = [torch.empty((g["m"], K), device=DEV) for g in graphs]
    start = tune_from(ns, TM=32)
    t, ms = ns.batch_autotune(Ad, [K] * len(graphs), ns.NS_F32, Bd, Cd, start=start)
    assert t.chunk_nnz in (128, 256, 512, 1024) and t.absorb_cap == t.chunk_nnz
    assert t.TM == 32 and ms > 0                       # the rest of the start tune is kept
    bt = ns.Batch(Ad, [K] * len(graphs), ns.NS_F32, t)
    bt.execute(Bd, Cd)
    torch.cuda.synchronize()
    for g, b, c in zip(graphs, Bs, Cd):
        assert oracle.rel_frobenius(c.cpu().numpy(), oracle.spmm(g, b)) <= 1e-5
    bt.close()


def test_batch_mixed_K():
    graphs = synth.batch_graphs(6, seed=7, n_lo=300, n_hi=3000)
    Ks = [32, 64, 32, 128, 64, 32]
    rng = np.random.default_rng(2)
    Bs = [rng.standard_normal((g["n"], k), dtype=np.float32) for g, k in zip(graphs, Ks)]
    bt = ns.Batch([to_dev(g, DEV) for g in graphs], Ks, ns.NS_F32)
    Cd = [torch.empty((g["m"], k), device=DEV) for g, k in zip(graphs, Ks)]
    bt.execute([torch.from_numpy(b).to(DEV) for b in Bs], Cd)
    torch.cuda.synchronize()
    for g, b, c in zip(graphs, Bs, Cd):
        assert oracle.rel_frobenius(c.cpu().numpy(), oracle.spmm(g, b)) <= 1e-5


@pytest.mark.parametrize("which", ["attention", "powerlaw"])
def test_autotune_gives_valid_fast_tune(which):
    if which == "attention":
        A = synth.block_sparse_csr(4096, seed=1)
    else:
        A = synth.rmat_csr(14, 250000, seed=2)
    K = 64
    B = synth.dense_b(A["n"], K, seed=3)
    At = to_dev(A, DEV)
    t, rep = ns.autotune(At, K, ns.NS_F32, report=True)
    assert rep["trials"] >= 3 and rep["p_res"] > 0
    C = torch.empty((A["m"], K), device=DEV)
    with ns.spmm_plan(At, K, ns.NS_F32, t) as p:
        p.execute(torch.from_numpy(B).to(DEV), C)
        torch.cuda.synchronize()
    assert oracle.rel_frobenius(C.cpu().numpy(), oracle.spmm(A, B)) <= 1e-5


@pytest.mark.slow
def test_batched_config_at_size():
    # the batched workload at its full size: 512 uneven graphs (node counts log-uniform in
    # [1e3, 5e4], mean degree 8-32, about 128 M nonzeros), K = 64, one persistent launch replayed
    # from a CUDA graph; every graph compared in full with the FP64 oracle
    import os
    from parity import check_result
    threads = max(1, min(16, len(os.sched_getaffinity(0))))
    graphs, Bs = synth.config_batched(0)
    K = 64
    assert len(graphs) == 512
    Ad = [to_dev(g, DEV) for g in graphs]
    Bd = [torch.from_numpy(b).to(DEV) for b in Bs]
    Cd = [torch.full((g["m"], K), float("nan"), device=DEV) for g in graphs]
    bt = ns.Batch(Ad, [K] * len(graphs), ns.NS_F32, tune_from(ns, chunk_nnz=512, absorb_cap=512))
    launches = ns.launch_count()
    for _ in range(2):                                  # capture, then one replay
        bt.execute(Bd, Cd)
    torch.cuda.synchronize()
    assert ns.launch_count() - launches == 2
    worst = 0.0
    for g, b, c in zip(graphs, Bs, Cd):
        rep = check_result(c.cpu().numpy(), g, b, tol=1e-5, threads=threads)
        worst = max(worst, rep["rel_frobenius"])
    print(f"\n[parity] batched 512 graphs, {sum(g.nnz for g in graphs)} nnz: max rel. Frobenius {worst:.3e}")
    bt.close()
