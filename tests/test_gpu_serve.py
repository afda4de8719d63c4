"""Serving: continuous batching of SpMM requests (GPU).  Every result matches the oracle, and
each request's C is the same alone and in the mix (bit for bit: a row is summed in a fixed order
given its plan, whatever else shares the launch)."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from nsutil import to_dev  # noqa: E402


def pinned(shape, dtype):
    t = torch.empty(shape, dtype=dtype).pin_memory()
    return t.numpy()


def wait_all(sv, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            done, st = sv.poll(t)
            if done:
                out[t] = st
                pending.discard(t)
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.0005)
    return out


def make_requests(graphs, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        g = int(rng.integers(0, len(graphs)))
        K = int(rng.choice([32, 64, 128]))
        bf16 = bool(rng.integers(0, 2))
        B = rng.standard_normal((graphs[g]["n"], K), dtype=np.float32)
        reqs.append((g, K, bf16, synth.bf16_bits(B) if bf16 else B))
    return reqs


def serve(graphs, reqs, **cfg):
    sv = ns.Server(**cfg)
    gids = [sv.register(g) for g in graphs]
    outs, tickets = [], []
    for g, K, bf16, B in reqs:
        Bp = pinned(B.shape, torch.int16 if bf16 else torch.float32)
        Bp[...] = B.view(np.int16) if bf16 else B
        Bp = Bp.view(np.uint16) if bf16 else Bp
        C = pinned((graphs[g]["m"], K), torch.float32)
        C[...] = np.nan
        tickets.append(sv.submit(gids[g], Bp, C, ns.NS_BF16 if bf16 else ns.NS_F32))
        outs.append(C)
    stats = wait_all(sv, tickets)
    sv.close()
    return outs, [stats[t] for t in tickets]


def test_mix_matches_oracle_and_alone():
    graphs = [synth.serve_graph(n, seed=i) for i, n in enumerate([700, 3000, 12000, 40000])]
    reqs = make_requests(graphs, 40, seed=1)
    mixed, stats = serve(graphs, reqs, max_inflight=16)
    for (g, K, bf16, B), C, st in zip(reqs, mixed, stats):
        assert st["status"] == 0
        assert st["t_done"] >= st["t_start"] >= st["t_admit"] > 0
        ref = oracle.spmm(graphs[g], B, b_bf16=bf16)
        assert oracle.rel_frobenius(C, ref) <= 1e-5
    # the default tune keeps every nonzero on the CUDA cores: one plan per graph serves every K
    # and dtype, built for the first request on the graph
    firsts = {}
    for k, (g, K, bf16, B) in enumerate(reqs):
        firsts.setdefault(g, k)
    assert [k for k, st in enumerate(stats) if st["plan_built"]] == sorted(firsts.values())
    for k in firsts.values():
        assert stats[k]["t_planned"] > 0 and stats[k]["t_admit"] >= stats[k]["t_planned"]
    # the same requests one at a time
    for i in (0, 7, 13, 29):
        alone, _ = serve(graphs, [reqs[i]], max_inflight=1)
        assert np.array_equal(alone[0], mixed[i])


def test_admission_errors():
    g = synth.serve_graph(5000, seed=3)
    sv = ns.Server(hbm_budget_bytes=1 << 20, max_inflight=4)
    gid = sv.register(g)
    B = np.zeros((g["n"], 128), dtype=np.float32)
    C = np.zeros((g["m"], 128), dtype=np.float32)
    with pytest.raises(ns.NsError) as e:
        sv.submit(gid, B, C)
    assert e.value.code == 7                                   # footprint over the budget
    with pytest.raises(ns.NsError) as e:
        sv.submit(gid + 5, B, C)
    assert e.value.code == 8                                   # unknown graph
    with pytest.raises(ns.NsError) as e:
        sv.submit(gid, B[:, :12], C[:, :12])
    assert e.value.code == 2                                   # K % 8 != 0
    sv.close()


def test_small_budget_still_serves_everything():
    # budget fits about one request at a time: admission waits for memory, nothing is lost
    graphs = [synth.serve_graph(20000, seed=5)]
    reqs = [(0, 64, False, synth.dense_b(20000, 64, seed=s)) for s in range(6)]
    need = 20000 * 64 * 4 * 2 + 20000 * 24 + graphs[0].nnz * 8
    outs, stats = serve(graphs, reqs, hbm_budget_bytes=int(need * 2.5), max_inflight=8)
    for (g, K, bf16, B), C in zip(reqs, outs):
        assert oracle.rel_frobenius(C, oracle.spmm(graphs[0], B)) <= 1e-5


def test_hybrid_tune_plans_per_key():
    # with dense tiles the plan depends on K and dtype: one plan per (graph, K, dtype)
    graphs = [synth.block_sparse_csr(2048, seed=4, block=16, band=2, p_random=0.05),
              synth.serve_graph(3000, seed=2)]
    reqs = make_requests(graphs, 24, seed=5)
    tune = ns.tune_default()
    tune.tau_tile, tune.TM = 48, 16
    outs, stats = serve(graphs, reqs, max_inflight=8, tune=tune)
    keys = {}
    for k, (g, K, bf16, B) in enumerate(reqs):
        keys.setdefault((g, K, bf16), k)
    assert [k for k, st in enumerate(stats) if st["plan_built"]] == sorted(keys.values())
    for (g, K, bf16, B), C, st in zip(reqs, outs, stats):
        assert st["status"] == 0
        ref = oracle.spmm(graphs[g], B, b_bf16=bf16)
        assert oracle.rel_frobenius(C, ref) <= (2e-2 if bf16 else 1e-5)


def _al256(b):
    return (b + 255) // 256 * 256


def test_admission_by_built_plan_size():
    # a budget that the submit-time estimate fits but the built plan plus the request's slots do
    # not: the request is refused at admission with NS_ERR_TOO_LARGE (7), and the server goes on
    g = synth.serve_graph(30000, seed=9)
    K = 128
    At = to_dev(g, torch.device("cuda", 0))
    with ns.spmm_plan(At, K, ns.NS_F32) as p:
        st = p.stats()
    est = g["m"] * 24 + g.nnz * 8 + 4096
    io = _al256(g["n"] * K * 4) + _al256(g["m"] * K * 4)
    submit_need = io + _al256(4) + est                        # no slots, one counter word
    admit_need = io + _al256(st["n_slots"] * K * 4) + _al256(max(st["n_split"], 1) * 4) + st["device_bytes"]
    if admit_need <= submit_need:
        pytest.skip("the estimate covers this plan")
    B = pinned((g["n"], K), torch.float32)
    B[...] = synth.dense_b(g["n"], K, seed=1)
    C = pinned((g["m"], K), torch.float32)
    sv = ns.Server(hbm_budget_bytes=submit_need, max_inflight=2)
    gid = sv.register(g)
    t = sv.submit(gid, B, C)
    t0 = time.time()
    while True:
        try:
            done, _ = sv.poll(t)
        except ns.NsError as e:
            assert e.code == 7
            break
        assert not done, "admitted over the budget"
        assert time.time() - t0 < 30
        time.sleep(0.001)
    # a budget with room for the built plan serves the same request
    sv.close()
    outs, stats = serve([g], [(0, K, False, np.asarray(B))], hbm_budget_bytes=admit_need, max_inflight=2)
    assert stats[0]["status"] == 0
    assert oracle.rel_frobenius(outs[0], oracle.spmm(g, np.asarray(B))) <= 1e-5
