"""Parity of the CUDA path against the FP64 oracle (GPU): the plan's partition bit-exact with the
CPU reference partition and its execute bookkeeping valid, results within the FP32 / BF16
tolerances, exact cases exact."""
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

DEV = torch.device("cuda", 0)
TOL = {ns.NS_F32: 1e-5, ns.NS_BF16: 2e-2}


def run(A, B, dtype=ns.NS_F32, tune=None, check_plan=True, C=None):
    K = B.shape[1]
    At = to_dev(A, DEV)
    if dtype == ns.NS_BF16:
        Bb = synth.bf16_bits(B) if B.dtype == np.float32 else B
        Bt = torch.from_numpy(Bb.view(np.int16)).to(DEV).view(torch.bfloat16)
        ref = oracle.spmm(A, Bb, b_bf16=True)
    else:
        Bt = torch.from_numpy(B).to(DEV)
        ref = oracle.spmm(A, B)
    tune = tune or ns.tune_default()
    Ct = torch.full((A["m"], K), float("nan"), device=DEV) if C is None else C
    with ns.spmm_plan(At, K, dtype, tune) as p:
        if check_plan:
            compare_plan(p, oracle.plan(A, K, b_bf16=dtype == ns.NS_BF16, **oracle_tune(tune)), A, tune)
        p.execute(Bt, Ct)
        torch.cuda.synchronize()
        c1 = Ct.cpu().numpy()
        p.execute(Bt, Ct)   # a second launch: ticket and split counters were reset
        torch.cuda.synchronize()
        c2 = Ct.cpu().numpy()
    assert np.array_equal(c1, c2), "second launch differs"
    assert not np.isnan(c1).any(), "rows left unwritten"
    return c1, ref


@pytest.mark.parametrize("dtype", [ns.NS_F32, ns.NS_BF16])
def test_small_uniform(dtype):
    A, B = synth.config_small(0)
    c, ref = run(A, B, dtype)
    assert oracle.rel_frobenius(c, ref) <= 1e-6


@pytest.mark.parametrize("K", [8, 16, 24, 32, 64, 96, 128, 136, 256, 512])
def test_widths(K):
    A = synth.rmat_csr(12, 40000, seed=K, values="uniform")
    B = synth.dense_b(A["n"], K, seed=1)
    c, ref = run(A, B)
    assert oracle.rel_frobenius(c, ref) <= 1e-6


@pytest.mark.parametrize("W", [2, 3, 16, 64, 256, 1024])
def test_chunk_sizes_split_rows(W):
    # hub rows longer than W/2 are cut into pieces assembled through the slots
    A = synth.random_csr(300, 500, 0.02, seed=W, hub_rows=4, empty_rows=0.3)
    B = synth.dense_b(500, 32, seed=2)
    t = tune_from(ns, chunk_nnz=W)
    c, ref = run(A, B, tune=t)
    assert oracle.rel_frobenius(c, ref) <= 1e-6


@pytest.mark.parametrize("K", [72, 96, 128])
@pytest.mark.parametrize("W", [16, 512])
def test_bf16_paired_widths(K, W):
    # BF16 with 64 < K <= 128: each lane gathers 8 adjacent columns and the warp takes two
    # nonzeros per step; W = 16 cuts the hub rows into pieces assembled through the slots
    A = synth.random_csr(300, 500, 0.05, seed=K + W, hub_rows=4, empty_rows=0.2)
    B = synth.dense_b(500, K, seed=3)
    c, ref = run(A, B, ns.NS_BF16, tune=tune_from(ns, chunk_nnz=W, absorb_cap=W))
    assert oracle.rel_frobenius(c, ref) <= 1e-6


def test_identity_and_permutation_exact():
    A = synth.identity_csr(3000)
    B = synth.dense_b(3000, 64, seed=3)
    c, _ = run(A, B)
    assert np.array_equal(c, B)
    P, perm = synth.permutation_csr(3000, seed=4)
    c, _ = run(P, B)
    assert np.array_equal(c, B[perm])


def test_empty_and_degenerate():
    B = synth.dense_b(50, 16, seed=0)
    A = synth.random_csr(40, 50, 0.0, seed=0)            # no nonzeros: C must be exactly 0
    c, _ = run(A, B)
    assert np.count_nonzero(c) == 0
    A = synth.random_csr(1, 50, 1.0, seed=0)             # one dense row
    c, ref = run(A, B, tune=tune_from(ns, chunk_nnz=8))
    assert oracle.rel_frobenius(c, ref) <= 1e-6
    A = synth.random_csr(0, 50, 0.0, seed=0)             # zero rows
    At = to_dev(A, DEV)
    with ns.spmm_plan(At, 16, ns.NS_F32) as p:
        p.execute(torch.from_numpy(B).to(DEV), torch.empty((0, 16), device=DEV))
        torch.cuda.synchronize()


def test_l2_hints_off_same_result():
    A = synth.rmat_csr(12, 30000, seed=5)
    B = synth.dense_b(A["n"], 64, seed=6)
    c1, ref = run(A, B, tune=tune_from(ns, l2_hints=1))
    c0, _ = run(A, B, tune=tune_from(ns, l2_hints=0), check_plan=False)
    assert np.array_equal(c0, c1)


def test_invalid_csr_rejected():
    A = synth.random_csr(20, 20, 0.4, seed=1)
    bad = dict(A)
    bad["colidx"] = A["colidx"].copy()
    i = int(np.argmax(np.diff(A["rowptr"]) >= 2))
    p = A["rowptr"][i]
    bad["colidx"][p] = bad["colidx"][p + 1]               # duplicate inside a row
    with pytest.raises(ns.NsError) as e:
        ns.spmm_plan(to_dev(bad, DEV), 8, ns.NS_F32)
    assert e.value.code == 1
    oob = dict(A)
    oob["colidx"] = A["colidx"].copy()
    oob["colidx"][0] = 20
    with pytest.raises(ns.NsError) as e:
        ns.spmm_plan(to_dev(oob, DEV), 8, ns.NS_F32)
    assert e.value.code == 1
    with pytest.raises(ns.NsError) as e:                  # host CSR path validates too
        ns.spmm_plan(bad, 8, ns.NS_F32, device=False)
    assert e.value.code == 1


def test_unsupported_shapes_and_alignment():
    A = synth.random_csr(20, 20, 0.4, seed=1)
    At = to_dev(A, DEV)
    with pytest.raises(ns.NsError) as e:
        ns.spmm_plan(At, 12, ns.NS_F32)
    assert e.value.code == 2
    with ns.spmm_plan(At, 16, ns.NS_F32) as p:
        Bbig = torch.zeros(20 * 16 + 1, device=DEV)
        B = Bbig[1:].view(20, 16)                          # 4-byte offset: not 16-byte aligned
        with pytest.raises(ns.NsError) as e:
            p.execute(B, torch.zeros(20, 16, device=DEV))
        assert e.value.code == 2


def test_host_csr_plan_equals_device_plan():
    A = synth.rmat_csr(11, 20000, seed=9)
    t = tune_from(ns, chunk_nnz=32)
    with ns.spmm_plan(A, 32, ns.NS_F32, t, device=False) as ph:
        compare_plan(ph, oracle.plan(A, 32, **oracle_tune(t)), A, t)


def test_spmm_host_entry():
    A = synth.rmat_csr(12, 50000, seed=11)
    B = synth.dense_b(A["n"], 64, seed=12)
    C = np.full((A["m"], 64), np.nan, dtype=np.float32)
    ns.spmm_host(A, B, C)
    assert oracle.rel_frobenius(C, oracle.spmm(A, B)) <= 1e-6


def test_kernels_really_launch():
    before = ns.launch_count()
    A, B = synth.config_small(1)
    run(A, B, check_plan=False)
    assert ns.launch_count() > before


@pytest.mark.parametrize("K,TN", [(128, 64), (128, 32), (256, 64), (96, 32), (64, 16)])
def test_column_slices(K, TN):
    # Column slices of B and C give the same product.  A narrower slice may take several
    # nonzeros per warp step (lane groups summed at the row's end), so the summation order, and
    # with it the last bits, can differ from the full width; each form is deterministic.
    A = synth.rmat_csr(12, 50000, seed=K + TN)
    B = synth.dense_b(A["n"], K, seed=4)
    c_full, ref = run(A, B, tune=tune_from(ns, TN=0), check_plan=False)
    c_sl, _ = run(A, B, tune=tune_from(ns, TN=TN), check_plan=False)
    c_sl2, _ = run(A, B, tune=tune_from(ns, TN=TN), check_plan=False)
    assert np.array_equal(c_sl, c_sl2)
    assert oracle.rel_frobenius(c_sl, ref) <= 1e-6
    assert oracle.rel_frobenius(c_full, ref) <= 1e-6


@pytest.mark.parametrize("tau", [ns.NS_TAU_INF, 8])
@pytest.mark.parametrize("dtype", [ns.NS_F32, ns.NS_BF16])
def test_hot_rows_l2_policy(tau, dtype):
    # Section 6.2.1 hot-B staging (l2_hints = 2): the planner marks the most gathered B rows and
    # the gathers pick their L2 policy from that map; the product must not change
    A = synth.rmat_csr(13, 120000, seed=17)
    B = synth.dense_b(A["n"], 64, seed=18)
    c, ref = run(A, B, dtype, tune=tune_from(ns, tau_tile=tau, TM=16, l2_hints=2))
    assert oracle.rel_frobenius(c, ref) <= TOL[dtype]
    c1, _ = run(A, B, dtype, tune=tune_from(ns, tau_tile=tau, TM=16, l2_hints=1), check_plan=False)
    assert oracle.rel_frobenius(c1, ref) <= TOL[dtype]


def test_bookkeeping_checker_bites():
    # the invariant checker of the execute bookkeeping accepts the device plan and rejects
    # planted mistakes in each of its arrays
    from plan_checks import check_bookkeeping, exports
    A = synth.random_csr(400, 500, 0.03, seed=5, hub_rows=4, empty_rows=0.2)
    # long rows kept for windows (tau_row), tiles dense only where columns repeat (tau 40), no
    # absorption: the kept rows are assembled from a dense piece and residual chunk pieces
    t = tune_from(ns, tau_tile=40, TM=16, TK=16, tau_row=20, chunk_nnz=16, absorb_cap=0)
    part = oracle.plan(A, 32, **oracle_tune(t))
    with ns.spmm_plan(to_dev(A, DEV), 32, ns.NS_F32, t) as p:
        st, ex = p.stats(), exports(p)
    td = t.as_dict()
    check_bookkeeping(A, part, st, ex, td)
    assert st["n_split"] > 0 and st["n_dwin"] > 0 and st["n_chunks"] > 2

    def bump(name, k, d=1):
        def f(e):
            e[name] = e[name].copy()
            e[name][k] += d
        return f

    def swap_queue(e):
        e["queue"] = e["queue"].copy()
        e["queue"][[0, -1]] = e["queue"][[-1, 0]]

    def drop_rl(e):
        e["rl_rows"] = e["rl_rows"][:-1].copy()

    def empty_chunk(e):
        e["chunk_b"] = e["chunk_b"].copy()
        e["chunk_b"][1] = e["chunk_b"][0]

    # (moving a boundary by one inside a long row is not a mistake: the pieces stay consistent)
    mutations = [empty_chunk, bump("chunk_b", -1, -1), bump("chunk_k0", 1), bump("split_base", 0),
                 bump("split_slot", 0),
                 bump("split_np", 0), bump("row_split", int(np.argmax(ex["row_split"] < 0)), 1),
                 bump("dwin_absorb", 0), bump("rl_start", 2), bump("item_cost", 0, 1 << 20),
                 swap_queue, drop_rl]
    for mutate in mutations:
        bad = {k: v for k, v in ex.items()}
        mutate(bad)
        with pytest.raises(AssertionError):
            check_bookkeeping(A, part, st, bad, td)
