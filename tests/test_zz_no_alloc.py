"""The allocation-free entry point, for callers that cannot call cudaMalloc (their device memory
belongs to another allocator, or they cannot afford the implicit synchronisation of
cudaMalloc/cudaFree).  It must give the same C as the planned path, call after call, although
every call reuses one static scratch array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from parity import check_result

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2606_22482_gb300 as ns  # noqa: E402
from paper_2606_22482_gb300 import _abi  # noqa: E402

DEV = torch.device("cuda", 0)


def _csr(At, A):
    return _abi.Csr(int(A["m"]), int(A["n"]), int(A.nnz), ctypes.c_void_p(At["rowptr"].data_ptr()),
                    ctypes.c_void_p(At["colidx"].data_ptr()), ctypes.c_void_p(At["vals"].data_ptr()), 1)


def _static(At, A, Bt, C, K, dtype):
    c = _csr(At, A)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ns.lib.ns_spmm_csr_static(ctypes.byref(c), ctypes.c_void_p(Bt.data_ptr()), K,
                                     ctypes.c_void_p(C.data_ptr()), K, K, dtype, s)


def _dev(A):
    return {k: (torch.from_numpy(v).to(DEV) if isinstance(v, np.ndarray) else v) for k, v in A.items()}


def _b(B, dtype):
    if dtype == ns.NS_BF16:
        Bh = synth.bf16_bits(B)
        return Bh, torch.from_numpy(Bh.view(np.int16)).to(DEV).view(torch.bfloat16)
    return B, torch.from_numpy(B).to(DEV)


@pytest.mark.parametrize("K,dtype", [(8, ns.NS_F32), (64, ns.NS_F32), (128, ns.NS_F32), (512, ns.NS_F32),
                                     (1024, ns.NS_F32), (8, ns.NS_BF16), (32, ns.NS_BF16)])
def test_static_matches_planned_path(K, dtype):
    A = synth.rmat_csr(13, 120000, seed=K)       # power-law rows: long rows are cut into pieces
    B = synth.dense_b(A["n"], K, seed=1)
    At = _dev(A)
    Bh, Bt = _b(B, dtype)
    C_ref = torch.empty((A["m"], K), device=DEV)
    with ns.spmm_plan(At, K, dtype) as p:
        p.execute(Bt, C_ref)
    torch.cuda.synchronize()
    ref = C_ref.cpu().numpy()
    for _ in range(2):                            # two calls in a row share the scratch array
        C = torch.full((A["m"], K), float("nan"), device=DEV)
        rc = _static(At, A, Bt, C, K, dtype)
        assert rc == 0, ns.lib.ns_last_error()
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        assert not np.isnan(got).any()
        assert oracle.rel_frobenius(got, ref) <= 1e-5
    check_result(got, A, Bh, b_bf16=dtype == ns.NS_BF16, tol=1e-5)


def test_static_large_then_small():
    # a small call right after a large one must not see the counters the large one left behind
    big = synth.rmat_csr(15, 600000, seed=3)
    small = synth.random_csr(300, 200, 0.05, seed=4, hub_rows=3, empty_rows=0.3)
    for A in (big, small, big, small):
        B = synth.dense_b(A["n"], 64, seed=5)
        At, Bt = _dev(A), torch.from_numpy(B).to(DEV)
        C = torch.full((A["m"], 64), float("nan"), device=DEV)
        assert _static(At, A, Bt, C, 64, ns.NS_F32) == 0, ns.lib.ns_last_error()
        torch.cuda.synchronize()
        check_result(C.cpu().numpy(), A, B, tol=1e-5)


@pytest.mark.parametrize("kind", ["no_nonzeros", "empty_rows", "no_rows"])
def test_static_degenerate(kind):
    if kind == "no_nonzeros":
        A = synth.random_csr(100, 50, 0.0, seed=1)
    elif kind == "empty_rows":
        A = synth.random_csr(500, 80, 0.02, seed=2, empty_rows=0.7)
    else:
        A = synth.random_csr(0, 50, 0.0, seed=3)
    B = synth.dense_b(A["n"], 16, seed=6)
    At, Bt = _dev(A), torch.from_numpy(B).to(DEV)
    C = torch.full((max(A["m"], 1), 16), float("nan"), device=DEV)
    assert _static(At, A, Bt, C, 16, ns.NS_F32) == 0, ns.lib.ns_last_error()
    torch.cuda.synchronize()
    got = C.cpu().numpy()[:A["m"]]
    if A["m"]:
        check_result(got, A, B, tol=1e-5)
    if A.nnz == 0:
        assert np.all(got == 0)


def test_static_rejects_oversized():
    # documented limit: 2 * ceil((m + nnz) / 256) partial rows of K floats must fit in 32 MiB
    A = synth.uniform_csr(65536, 4096, 18, seed=2)
    K = 1024
    nc = -(-(A["m"] + A.nnz) // 256)
    assert 2 * nc * K * 4 > 32 << 20
    At = {k: (torch.from_numpy(v).to(DEV) if isinstance(v, np.ndarray) else v) for k, v in A.items()}
    Bt = torch.zeros((A["n"], K), device=DEV)
    C = torch.zeros((A["m"], K), device=DEV)
    rc = _static(At, A, Bt, C, K, ns.NS_F32)
    assert rc == 7, rc
    assert b"static scratch" in ns.lib.ns_last_error()
