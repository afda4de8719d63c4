"""The seeded workload generators against the input recipe they stand for (CPU only).

The generators replace the paper's datasets (Section 8.1), so the shapes, skews and structure
the benchmarks rely on are checked here: fixed-degree uniform rows, RMAT quadrant statistics and
GCN values, the block-sparse attention mask, the batched graphs' size and degree ranges, and the
serving pool's lognormal sizes.
"""
import numpy as np

import synth


def _rows_sorted_unique(A):
    rp, ci = A["rowptr"].astype(np.int64), A["colidx"].astype(np.int64)
    d = np.diff(ci)
    starts = np.zeros(len(ci), dtype=bool)
    starts[rp[:-1][rp[:-1] < rp[1:]]] = True
    # inside a row the next column is strictly larger; across a row start anything goes
    return bool(np.all((d > 0) | starts[1:])) and bool(np.all((ci >= 0) & (ci < A["n"])))


def test_small_config_shape():
    A, B = synth.config_small()
    assert A["m"] == A["n"] == 4096 and A.nnz == 4096 * 16
    assert np.all(np.diff(A["rowptr"]) == 16)
    assert _rows_sorted_unique(A)
    assert A["vals"].dtype == np.float32 and np.all(np.abs(A["vals"]) <= 1.0)
    assert B.shape == (4096, 32) and B.dtype == np.float32
    assert abs(float(B.mean())) < 0.02 and abs(float(B.std()) - 1.0) < 0.02


def test_rmat_quadrant_statistics_and_gcn_values():
    # without the relabelling the top bit of a row (column) id is 1 with probability c + d (b + d)
    scale, nnz = 12, 40000
    A = synth.rmat_csr(scale, nnz, seed=3, relabel=False)
    assert A.nnz == nnz and _rows_sorted_unique(A)
    half = 1 << (scale - 1)
    rows = np.repeat(np.arange(A["m"]), np.diff(A["rowptr"]))
    cols = A["colidx"]
    assert abs(float(np.mean(rows >= half)) - 0.24) < 0.03
    assert abs(float(np.mean(cols >= half)) - 0.24) < 0.03
    # the a quadrant (both bits 0) dominates at every level: column 0's in-degree is the largest
    cnt = np.bincount(cols, minlength=A["n"])
    assert int(np.argmax(cnt)) == 0 and cnt[0] > 20 * cnt.mean()
    deg = np.diff(A["rowptr"]).astype(np.int64)
    assert np.array_equal(A["vals"], (1.0 / deg[rows]).astype(np.float32))


def test_rmat_relabel_and_community_order_keep_the_graph():
    scale, nnz = 11, 15000
    A0 = synth.rmat_csr(scale, nnz, seed=4, relabel=False)
    A1 = synth.rmat_csr(scale, nnz, seed=4)
    A2 = synth.rmat_csr(scale, nnz, seed=4, community=True)
    for A in (A1, A2):
        assert A.nnz == nnz and _rows_sorted_unique(A)
    # relabelling permutes vertex ids: the degree multisets are those of the unlabelled graph
    assert np.array_equal(np.sort(np.diff(A0["rowptr"])), np.sort(np.diff(A1["rowptr"])))
    assert np.array_equal(np.sort(np.bincount(A0["colidx"], minlength=A0["n"])),
                          np.sort(np.bincount(A1["colidx"], minlength=A1["n"])))
    # the community variant reorders rows only: the same set of column lists
    def row_sets(A):
        rp, ci = A["rowptr"], A["colidx"]
        return sorted(tuple(ci[rp[i]:rp[i + 1]]) for i in range(A["m"]))
    assert row_sets(A1) == row_sets(A2)


def test_block_sparse_attention_mask():
    n, blk = 2048, 64
    A = synth.block_sparse_csr(n, seed=5)
    assert A["m"] == A["n"] == n and _rows_sorted_unique(A)
    rp, ci, v = A["rowptr"], A["colidx"], A["vals"]
    assert np.all(v > 0)
    sums = np.add.reduceat(v.astype(np.float64), rp[:-1])
    assert np.max(np.abs(sums - 1.0)) < 1e-5
    for i in range(n):
        bi = i // blk
        c = ci[rp[i]:rp[i + 1]]
        cb = c // blk
        for bj in range(max(0, bi - 3), bi + 1):  # the causal band of four blocks, complete
            assert np.sum(cb == bj) == blk
        ub, counts = np.unique(cb, return_counts=True)
        full = ub[counts >= blk]
        # exactly one nonzero outside the row's active (complete) blocks
        assert np.sum(~np.isin(cb, full)) == 1
        if i % blk == 0:
            first_full = full
        else:
            assert np.array_equal(full, first_full)  # one active-block set per block row


def test_block_sparse_random_block_rate():
    n, blk = 8192, 64
    nb = n // blk
    A = synth.block_sparse_csr(n, seed=6)
    rp, ci = A["rowptr"], A["colidx"]
    off_band = 0
    for bi in range(nb):
        i = bi * blk
        cb = ci[rp[i]:rp[i + 1]] // blk
        ub, counts = np.unique(cb, return_counts=True)
        full = ub[counts == blk]
        off_band += int(np.sum((full < bi - 3) | (full > bi)))
    cand = sum(nb - len(range(max(0, bi - 3), bi + 1)) for bi in range(nb))
    assert abs(off_band / cand - 0.03) < 0.006


def test_batched_graph_ranges():
    graphs = synth.batch_graphs(6, seed=0)
    for g in graphs:
        assert 1000 <= g["n"] <= 50000 and g["m"] == g["n"]
        assert _rows_sorted_unique(g)
        d = g.nnz / g["n"]
        assert 4.0 <= d <= 32.0  # mean degree U(8, 32) before duplicates are dropped
        assert np.all(np.abs(g["vals"]) <= 1.0)


def test_serving_pool_sizes():
    s = synth.serve_pool_sizes(8192, seed=0)
    assert s.min() >= 64 and s.max() <= 2_000_000
    assert abs(float(np.median(s)) / 20000.0 - 1.0) < 0.05
    z = np.log(s.astype(np.float64) / 20000.0)
    assert abs(float(np.std(z)) - 1.2) < 0.05


def test_serve_graph_degree():
    g = synth.serve_graph(5000, seed=2)
    assert g["m"] == g["n"] == 5000 and g.nnz == 5000 * 16
    assert _rows_sorted_unique(g)
