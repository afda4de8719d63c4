"""Error paths driven from the host (GPU): an allocation that fails part-way through planning,
batching or serving returns NS_ERR_OOM and leaves the library usable; a status bit in a plan's
device word (as a kernel guard or a bounded wait would set it) is reported by a later execute.
Nothing here faults, traps or hangs the GPU."""
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
from nsutil import to_dev, tune_from  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.fixture(autouse=True)
def _injection_off():
    yield
    ns.inject_alloc_failure(-1)


def _case():
    A = synth.block_sparse_csr(512, seed=2, block=16, band=2, p_random=0.05)
    B = synth.dense_b(A["n"], 32, seed=3)
    return A, B


@pytest.mark.parametrize("tune_kw", [dict(tau_tile=ns.NS_TAU_INF), dict(tau_tile=40, TM=16)])
def test_plan_survives_a_failed_allocation_at_every_stage(tune_kw):
    A, B = _case()
    At, Bt = to_dev(A, DEV), torch.from_numpy(B).to(DEV)
    tune = tune_from(ns, **tune_kw)
    ref = oracle.spmm(A, B)
    failed = 0
    for after in range(0, 16):
        ns.inject_alloc_failure(after)
        try:
            p = ns.spmm_plan(At, 32, ns.NS_F32, tune)
        except ns.NsError as e:
            assert e.code == 3, e                     # NS_ERR_OOM
            failed += 1
            continue
        finally:
            ns.inject_alloc_failure(-1)
        p.close()
        # a plan made with fewer allocations than `after`: every later one fails no more
        break
    assert failed >= 2                                # planning allocates more than once
    with ns.spmm_plan(At, 32, ns.NS_F32, tune) as p:  # the library is still usable
        C = torch.full((A["m"], 32), float("nan"), device=DEV)
        p.execute(Bt, C)
        torch.cuda.synchronize()
        assert oracle.rel_frobenius(C.cpu().numpy(), ref) <= 1e-5


def test_batch_plan_failed_allocation():
    graphs = [synth.serve_graph(n, seed=i) for i, n in enumerate([300, 900, 2000])]
    for after in (0, 3, 9):
        ns.inject_alloc_failure(after)
        with pytest.raises(ns.NsError) as e:
            ns.Batch([to_dev(g, DEV) for g in graphs], [16] * 3, ns.NS_F32)
        assert e.value.code == 3
    ns.inject_alloc_failure(-1)
    b = ns.Batch([to_dev(g, DEV) for g in graphs], [16] * 3, ns.NS_F32)
    b.close()


def test_serve_request_fails_then_server_goes_on():
    g = synth.serve_graph(3000, seed=4)
    B = synth.dense_b(g["n"], 32, seed=1)
    Bp = torch.from_numpy(B).pin_memory().numpy()
    sv = ns.Server(max_inflight=4)
    gid = sv.register(g)
    ns.inject_alloc_failure(0)                        # the plan or the request's block fails
    C1 = np.full((g["m"], 32), np.nan, np.float32)
    t1 = sv.submit(gid, Bp, C1)
    t0 = time.time()
    with pytest.raises(ns.NsError) as e:
        while not sv.poll(t1)[0]:
            assert time.time() - t0 < 30
            time.sleep(0.001)
    assert e.value.code == 3
    C2 = np.full((g["m"], 32), np.nan, np.float32)
    t2 = sv.submit(gid, Bp, C2)
    while True:
        done, st = sv.poll(t2)
        if done:
            break
        assert time.time() - t0 < 30
        time.sleep(0.001)
    sv.close()
    assert st["status"] == 0
    assert oracle.rel_frobenius(C2, oracle.spmm(g, B)) <= 1e-5


@pytest.mark.parametrize("bits,code", [(4, 4), (2, 5)])
def test_status_word_reported_by_a_later_execute(bits, code):
    A, B = _case()
    Bt = torch.from_numpy(B).to(DEV)
    C = torch.empty((A["m"], 32), device=DEV)
    with ns.spmm_plan(to_dev(A, DEV), 32, ns.NS_F32) as p:
        p.execute(Bt, C)
        torch.cuda.synchronize()
        p.execute(Bt, C)                              # its status copy still reads 0
        torch.cuda.synchronize()
        p.inject_status(bits)
        p.execute(Bt, C)                              # copies the word back
        torch.cuda.synchronize()
        with pytest.raises(ns.NsError) as e:
            p.execute(Bt, C)
        assert e.value.code == code
    with pytest.raises(ns.NsError) as e:              # bits outside the status set are refused
        with ns.spmm_plan(to_dev(A, DEV), 32, ns.NS_F32) as p:
            p.inject_status(1)
    assert e.value.code == 1
