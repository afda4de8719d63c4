"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *draws* inputs.  It holds none of the SpMM method's arithmetic:
no products, no partitioning, no tiling.  Both the FP64 oracle (``oracle/``) and
the CUDA path consume what it returns; neither imports the other.

The paper evaluates on SuiteSparse matrices and GNN graphs (Table "Datasets",
Section 8.1) that are not available here; the generators below stand in for
them with the shapes and skews of those workloads:

* ``uniform_csr``      -- fixed row degree, uniform distinct columns
* ``rmat_csr``         -- power-law graph (RMAT), GCN-normalised values
* ``block_sparse_csr`` -- sparse-attention mask: causal band of 64x64 blocks,
                          random blocks and one scattered nonzero per row
* ``batch_graphs``     -- many uneven graphs (Erdos-Renyi + RMAT mix)
* ``serve_graph``      -- one graph of the serving pool

Every generator takes an explicit seed and uses numpy's PCG64 stream
(``numpy.random.default_rng``), so both sides see identical arrays.
A CSR matrix is a dict with int32 ``rowptr`` (m+1), int32 ``colidx`` (nnz,
sorted and unique inside each row), float32 ``vals`` and the shape ``m``, ``n``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Csr", "csr_from_coo", "uniform_csr", "rmat_csr", "block_sparse_csr",
    "batch_graphs", "serve_graph", "serve_pool_sizes", "dense_b", "bf16_bits",
    "random_csr", "identity_csr", "permutation_csr", "config_small",
    "config_powerlaw", "config_attention", "config_batched",
]


class Csr(dict):
    """A CSR matrix: keys m, n, rowptr (int32), colidx (int32), vals (float32)."""

    @property
    def nnz(self) -> int:
        return int(self["rowptr"][-1])

    def to_dense(self) -> np.ndarray:
        """Dense float64 copy (tiny inputs only)."""
        m, n = self["m"], self["n"]
        out = np.zeros((m, n), dtype=np.float64)
        rp, ci, v = self["rowptr"], self["colidx"], self["vals"]
        for i in range(m):
            for p in range(rp[i], rp[i + 1]):
                out[i, ci[p]] = v[p]
        return out


def csr_from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray,
                 vals: np.ndarray | None = None) -> Csr:
    """Build a CSR from unique (row, col) pairs; columns end up sorted per row."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(max(n, 1)) + cols
    if vals is None:
        order = None
        ks = np.sort(key)
        rows_s, cols_s = ks // np.int64(max(n, 1)), ks % np.int64(max(n, 1))
    else:
        order = np.argsort(key, kind="stable")
        rows_s = rows[order]
        cols_s = cols[order]
    counts = np.bincount(rows_s, minlength=m).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if vals is None:
        v = np.ones(len(cols_s), dtype=np.float32)
    else:
        v = np.asarray(vals, dtype=np.float32)[order]
    return Csr(m=int(m), n=int(n), rowptr=rowptr.astype(np.int32),
               colidx=cols_s.astype(np.int32), vals=v)


def dense_b(rows: int, K: int, seed: int) -> np.ndarray:
    """B ~ N(0, 1), float32, row-major rows x K."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((rows, K), dtype=np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """BF16 copy of a float32 array as uint16 bit patterns (PyTorch's round-to-nearest-even cast).

    This prepares the BF16 *input* B of the precision form; it is a library cast, not part of
    the method.
    """
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()


# ----------------------------------------------------------------------------------------
# small / test matrices
# ----------------------------------------------------------------------------------------

def uniform_csr(m: int, n: int, deg: int, seed: int) -> Csr:
    """``deg`` distinct uniform columns per row (sorted), values U(-1, 1) float32."""
    rng = np.random.default_rng(seed)
    deg = min(deg, n)
    cols = np.empty((m, deg), dtype=np.int64)
    block = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, m, block):
        r1 = min(m, r0 + block)
        keys = rng.random((r1 - r0, n), dtype=np.float32)
        part = np.argpartition(keys, deg - 1, axis=1)[:, :deg] if deg < n else \
            np.tile(np.arange(n), (r1 - r0, 1))
        cols[r0:r1] = np.sort(part, axis=1)
    vals = rng.uniform(-1.0, 1.0, size=m * deg).astype(np.float32)
    rowptr = (np.arange(m + 1, dtype=np.int64) * deg).astype(np.int32)
    return Csr(m=m, n=n, rowptr=rowptr, colidx=cols.reshape(-1).astype(np.int32), vals=vals)


def random_csr(m: int, n: int, density: float, seed: int, *, empty_rows: float = 0.0,
               hub_rows: int = 0, values: str = "uniform") -> Csr:
    """Bernoulli(density) pattern with optional empty rows and dense hub rows (tests)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    if empty_rows > 0:
        mask[rng.random(m) < empty_rows] = False
    for h in range(min(hub_rows, m)):
        mask[rng.integers(0, m)] = rng.random(n) < 0.9
    rows, cols = np.nonzero(mask)
    if values == "ones":
        vals = np.ones(len(rows), dtype=np.float32)
    elif values == "int":
        vals = rng.integers(-4, 5, size=len(rows)).astype(np.float32)
    else:
        vals = rng.uniform(-1.0, 1.0, size=len(rows)).astype(np.float32)
    return csr_from_coo(m, n, rows, cols, vals)


def identity_csr(n: int) -> Csr:
    idx = np.arange(n)
    return csr_from_coo(n, n, idx, idx, np.ones(n, dtype=np.float32))


def permutation_csr(n: int, seed: int) -> tuple[Csr, np.ndarray]:
    """Permutation matrix P with P[i, perm[i]] = 1, so (P B)[i] = B[perm[i]]."""
    perm = np.random.default_rng(seed).permutation(n)
    return csr_from_coo(n, n, np.arange(n), perm, np.ones(n, dtype=np.float32)), perm


# ----------------------------------------------------------------------------------------
# RMAT power-law graphs
# ----------------------------------------------------------------------------------------

def _rmat_pairs(rng: np.random.Generator, count: int, scale: int,
                a: float, b: float, c: float) -> tuple[np.ndarray, np.ndarray]:
    """Draw ``count`` RMAT (row, col) pairs: per level, quadrant a/b/c/d picks one bit of each.

    The quadrant is chosen from a 16-bit uniform draw (probabilities quantised to 1/65536).
    """
    dt = np.uint32 if scale <= 31 else np.uint64
    i = np.zeros(count, dtype=dt)
    j = np.zeros(count, dtype=dt)
    ta = np.uint16(min(65535, round(a * 65536)))
    tab = np.uint16(min(65535, round((a + b) * 65536)))
    tabc = np.uint16(min(65535, round((a + b + c) * 65536)))
    for _ in range(scale):
        u = rng.integers(0, 1 << 16, size=count, dtype=np.uint16)
        bi = u >= tab                          # quadrants c, d -> row bit 1
        bj = ((u >= ta) & ~bi) | (u >= tabc)   # quadrants b, d -> col bit 1
        i <<= dt(1)
        j <<= dt(1)
        i |= bi
        j |= bj
    return i.astype(np.int64), j.astype(np.int64)


def _rmat_unique(rng: np.random.Generator, scale: int, target: int,
                 abcd=(0.57, 0.19, 0.19, 0.05), limit: int | None = None) -> np.ndarray:
    """Keys (row << scale | col) of the first ``target`` distinct RMAT edges in draw order.

    Pairs with an id >= ``limit`` are rejected (used for graphs whose size is not a power of two).
    """
    a, b, c, _ = abcd
    keys = np.empty(0, dtype=np.int64)
    chunk = max(1 << 16, int(target * 1.3))
    while True:
        i, j = _rmat_pairs(rng, chunk, scale, a, b, c)
        if limit is not None:
            ok = (i < limit) & (j < limit)
            i, j = i[ok], j[ok]
        keys = np.concatenate([keys, (i << scale) | j])
        order = np.argsort(keys)
        ks = keys[order]
        new = np.empty(len(ks), dtype=bool)
        if len(ks):
            new[0] = True
            np.not_equal(ks[1:], ks[:-1], out=new[1:])
        starts = np.flatnonzero(new)
        if len(starts) >= target:
            first = np.minimum.reduceat(order, starts) if len(starts) else starts
            return keys[np.sort(first)[:target]]
        chunk = max(1 << 16, int((target - len(starts)) * 1.5))


def rmat_csr(scale: int, nnz: int, seed: int, *, abcd=(0.57, 0.19, 0.19, 0.05),
             relabel: bool = True, community: bool = False, values: str = "gcn") -> Csr:
    """RMAT graph with 2**scale vertices and ``nnz`` distinct edges (self loops kept).

    Vertex ids are relabelled by a seeded random permutation.  ``community=True`` then sorts
    the rows (only) by their pre-relabel id >> 10, ties broken by a seeded key, which groups
    rows of one RMAT sub-quadrant together.  ``values="gcn"`` gives 1/deg(row).
    """
    rng = np.random.default_rng(seed)
    n = 1 << scale
    keys = _rmat_unique(rng, scale, nnz, abcd)
    i = keys >> scale
    j = keys & (n - 1)
    if relabel:
        perm = rng.permutation(n)
        ri, cj = perm[i], perm[j]
        if community:
            tie = rng.permutation(n)
            inv = np.empty(n, dtype=np.int64)
            inv[perm] = np.arange(n)            # relabelled id -> original id
            order = np.lexsort((tie, inv >> 10))  # relabelled ids in community order
            rank = np.empty(n, dtype=np.int64)
            rank[order] = np.arange(n)
            ri = rank[ri]
        i, j = ri, cj
    csr = csr_from_coo(n, n, i, j, None)
    deg = np.diff(csr["rowptr"].astype(np.int64))
    if values == "gcn":
        rows = np.repeat(np.arange(n), deg)
        csr["vals"] = (1.0 / deg[rows]).astype(np.float32)
    else:
        csr["vals"] = rng.uniform(-1.0, 1.0, size=csr.nnz).astype(np.float32)
    return csr


# ----------------------------------------------------------------------------------------
# block-sparse attention mask
# ----------------------------------------------------------------------------------------

def block_sparse_csr(n: int, seed: int, *, block: int = 64, band: int = 4,
                     p_random: float = 0.03, extra_per_row: int = 1) -> Csr:
    """Sparse-attention pattern on n x n.

    Block (bi, bj) of a ``block`` x ``block`` grid is active if bj lies in the causal band
    [bi - band + 1, bi] or, independently, with probability ``p_random``.  Each row then gets
    ``extra_per_row`` nonzeros at columns drawn uniformly outside its active blocks.  Values
    are U(0, 1) divided by the row sum (softmax-like), stored as float32.
    """
    rng = np.random.default_rng(seed)
    nb = n // block
    active = rng.random((nb, nb)) < p_random
    for bi in range(nb):
        active[bi, max(0, bi - band + 1):bi + 1] = True
    col_parts = []
    row_lens = []
    ar = np.arange(block, dtype=np.int64)
    for bi in range(nb):
        blocks = np.nonzero(active[bi])[0]
        base = (blocks[:, None] * block + ar[None, :]).reshape(-1)
        inactive = np.ones(nb, dtype=bool)
        inactive[blocks] = False
        free_cols = (np.nonzero(inactive)[0][:, None] * block + ar[None, :]).reshape(-1)
        rows = np.empty((block, len(base) + extra_per_row), dtype=np.int64)
        rows[:, :len(base)] = base[None, :]
        for e in range(extra_per_row):
            if len(free_cols) == 0:
                raise ValueError("no free column for the scattered nonzero")
            pick = rng.integers(0, len(free_cols), size=block)
            rows[:, len(base) + e] = free_cols[pick]
        rows.sort(axis=1)
        if extra_per_row > 1:
            rows = [np.unique(r) for r in rows]
            for r in rows:
                col_parts.append(r)
                row_lens.append(len(r))
        else:
            col_parts.append(rows.reshape(-1))
            row_lens.extend([rows.shape[1]] * block)
    colidx = np.concatenate(col_parts).astype(np.int32)
    lens = np.asarray(row_lens, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    raw = rng.random(len(colidx))
    sums = np.add.reduceat(raw, rowptr[:-1]) if len(raw) else raw
    vals = (raw / np.repeat(sums, lens)).astype(np.float32)
    return Csr(m=n, n=n, rowptr=rowptr.astype(np.int32), colidx=colidx, vals=vals)


# ----------------------------------------------------------------------------------------
# batched and served graphs
# ----------------------------------------------------------------------------------------

def batch_graphs(count: int, seed: int, *, n_lo: int = 1000, n_hi: int = 50000,
                 deg_lo: float = 8.0, deg_hi: float = 32.0) -> list[Csr]:
    """``count`` graphs, n log-uniform in [n_lo, n_hi], mean degree U(deg_lo, deg_hi).

    Half of each graph's draws are Erdos-Renyi uniform (i, j), half RMAT at scale
    ceil(log2 n) with ids >= n rejected; duplicates are removed.  Values U(-1, 1).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ng = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        dg = rng.uniform(deg_lo, deg_hi)
        edges = int(round(ng * dg))
        half = edges // 2
        ei = rng.integers(0, ng, size=half)
        ej = rng.integers(0, ng, size=half)
        scale = max(1, math.ceil(math.log2(ng)))
        rk = _rmat_unique(rng, scale, edges - half, limit=ng)
        ri, rj = rk >> scale, rk & ((1 << scale) - 1)
        key = np.unique(np.concatenate([ei * ng + ej, ri * ng + rj]))
        rows, cols = key // ng, key % ng
        vals = rng.uniform(-1.0, 1.0, size=len(key)).astype(np.float32)
        out.append(csr_from_coo(ng, ng, rows, cols, vals))
    return out


def serve_pool_sizes(count: int, seed: int, *, median: float = 20000.0, sigma: float = 1.2,
                     n_min: int = 64, n_max: int = 2_000_000) -> np.ndarray:
    """Node counts of the serving pool: lognormal(median, sigma), clipped to [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(count)
    return np.clip(np.round(median * np.exp(sigma * z)), n_min, n_max).astype(np.int64)


def serve_graph(n: int, seed: int, *, avg_degree: int = 16) -> Csr:
    """One RMAT graph of the serving pool (n nodes, about avg_degree * n edges)."""
    rng = np.random.default_rng(seed)
    scale = max(1, math.ceil(math.log2(n)))
    target = min(int(n) * avg_degree, int(n) * int(n))
    keys = _rmat_unique(rng, scale, target, limit=n)
    i, j = keys >> scale, keys & ((1 << scale) - 1)
    perm = rng.permutation(n)
    vals = rng.uniform(-1.0, 1.0, size=len(keys)).astype(np.float32)
    return csr_from_coo(n, n, perm[i], perm[j], vals)


# ----------------------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------------------

def config_small(seed: int = 0):
    """Plain SpMM, small: 4096 x 4096, 16 nnz/row uniform, B 4096 x 32 N(0,1)."""
    a = uniform_csr(4096, 4096, 16, seed)
    b = dense_b(4096, 32, seed + 1)
    return a, b


def config_powerlaw(seed: int = 0, *, scale: int = 20, nnz: int = 1 << 24, K: int = 128,
                    community: bool = False):
    """Plain hybrid SpMM on an RMAT(.57,.19,.19,.05) graph, GCN values, B n x K N(0,1)."""
    a = rmat_csr(scale, nnz, seed, community=community)
    b = dense_b(a["n"], K, seed + 1)
    return a, b


def config_attention(seed: int = 0, *, n: int = 32768, K: int = 128):
    """Sparse-attention shape: 64x64 block mask (band 4, 3% random) + 1 scattered nnz/row."""
    a = block_sparse_csr(n, seed)
    b = dense_b(n, K, seed + 1)
    return a, b


def config_batched(seed: int = 0, *, count: int = 512, K: int = 64):
    """Batched form: ``count`` uneven graphs, K = 64 features each."""
    graphs = batch_graphs(count, seed)
    rng = np.random.default_rng(seed + 1)
    bs = [rng.standard_normal((g["n"], K), dtype=np.float32) for g in graphs]
    return graphs, bs
