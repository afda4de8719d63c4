"""GCN forward on the hybrid SpMM (GPU): two layers, H' = relu(A_hat (H W)), against an FP64
reference that uses the oracle's SpMM and numpy products."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from paper_2606_22482_gb300.gcn import GCN  # noqa: E402
from nsutil import to_dev, tune_from  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("K,tau", [(64, ns.NS_TAU_INF), (128, ns.NS_TAU_INF), (64, 24)])
def test_gcn_two_layers(K, tau):
    A = synth.rmat_csr(12, 60000, seed=K)
    X = synth.dense_b(A["n"], K, seed=5)
    rng = np.random.default_rng(9)
    Ws = [(rng.standard_normal((K, K)) / np.sqrt(K)).astype(np.float32) for _ in range(2)]
    with ns.spmm_plan(to_dev(A, DEV), K, ns.NS_F32, tune_from(ns, tau_tile=tau)) as p:
        net = GCN(p, [torch.from_numpy(W).to(DEV) for W in Ws])
        out = net.forward(torch.from_numpy(X).to(DEV))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        again = net.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()  # plan reused
    H = X.astype(np.float64)
    for li, W in enumerate(Ws):
        H = oracle.spmm(A, (H @ W.astype(np.float64)).astype(np.float32))
        if li + 1 < len(Ws):
            H = np.maximum(H, 0.0)
    assert oracle.rel_frobenius(got, H) <= 1e-5
    assert np.array_equal(got, again)
