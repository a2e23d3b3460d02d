"""Seeded synthetic inputs for FastPI: sparse power-law feature matrices and
binary multi-label targets.

This module only draws random inputs.  It holds none of FastPI's arithmetic,
so both the CPU oracle (``oracle/``) and the CUDA library's tests and bench
can use it without sharing any part of the method.

Shape profile (Table 3 and Section 4.1 of the paper): the feature matrix A is
m x n with m > n, very sparse, and its bipartite graph (Definition 1) has
heavy-tailed instance and feature degrees; the label matrix Y is m x L binary
with a few positives per row (Application 1).  The paper's datasets (Amazon,
RCV, Eurlex, Bibtex) are not available here, so Chung-Lu sampling with
power-law weights stands in for them.

Recipe (all with ``numpy.random.default_rng(seed)``):
  * row weight w_i = (i+1)^(-1/(gamma-1)), column weight likewise;
  * draw (row, col) pairs independently from the two weight distributions in
    batches, keep the first occurrence of each pair, stop once the number of
    distinct pairs reaches ``nnz``, cut to exactly ``nnz``;
  * apply a uniformly random row permutation and column permutation so that
    hubs are not pre-sorted;
  * values: uniform(0, 1] as ``1 - rng.random()``, or all ones (binary);
  * Y: ``p`` distinct labels per row drawn with ``rng.choice(L, p,
    replace=False)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Workload", "CONFIGS", "chung_lu_csr", "labels_dense", "labels_csr",
           "make", "make_tiny_random"]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    nnz: int
    gamma: float
    L: int
    p: int            # positives per label row
    k: float          # hub selection ratio (Algorithm 2)
    r: int            # target rank
    binary: bool = False
    sparse_y: bool = False


# The five workload shapes.  "small" finishes in the oracle in seconds; "medium"
# is the FP64-vs-mixed comparison workload timed by bench.py.
CONFIGS = {
    "small": Workload("small 2000x500 nnz20k r100", 2000, 500, 20_000, 2.1, 50, 3, 0.01, 100),
    "medium": Workload("medium 20000x5000 nnz500k r500", 20_000, 5_000, 500_000, 2.1, 400, 5, 0.01, 500),
    "large": Workload("large 200000x50000 nnz5M r1000", 200_000, 50_000, 5_000_000, 2.0, 1000, 5, 0.01, 1000),
    "xlarge": Workload("xlarge 1000000x200000 nnz20M r2000 binary", 1_000_000, 200_000, 20_000_000, 2.0,
                       3000, 4, 0.005, 2000, binary=True, sparse_y=True),
}


def _power_law_cdf(count: int, gamma: float) -> np.ndarray:
    w = np.arange(1, count + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    c = np.cumsum(w)
    return c / c[-1]


def chung_lu_csr(m: int, n: int, nnz: int, gamma: float, rng: np.random.Generator,
                 binary: bool = False):
    """Return (rowptr int64[m+1], col int32[nnz], val float64[nnz]) in CSR with
    sorted, duplicate-free column indices per row."""
    if nnz > m * n:
        raise ValueError("nnz exceeds m*n")
    cdf_r = _power_law_cdf(m, gamma)
    cdf_c = _power_law_cdf(n, gamma)
    keys = np.empty(0, dtype=np.int64)
    seen_count = 0
    while seen_count < nnz:
        batch = max(1024, int(1.3 * (nnz - seen_count)) + 1024)
        rows = np.searchsorted(cdf_r, rng.random(batch), side="right")
        cols = np.searchsorted(cdf_c, rng.random(batch), side="right")
        rows = np.minimum(rows, m - 1)
        cols = np.minimum(cols, n - 1)
        new = rows.astype(np.int64) * n + cols
        allk = np.concatenate([keys, new])
        # keep first occurrence, in draw order
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first]
        seen_count = keys.size
    keys = keys[:nnz]
    prow = rng.permutation(m)
    pcol = rng.permutation(n)
    rows = prow[keys // n]
    cols = pcol[keys % n]
    if binary:
        vals = np.ones(nnz, dtype=np.float64)
    else:
        vals = 1.0 - rng.random(nnz)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals


def labels_dense(m: int, L: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """Binary m x L label matrix (C order, float64) with p distinct positives per row."""
    Y = np.zeros((m, L), dtype=np.float64)
    for i in range(m):
        Y[i, rng.choice(L, p, replace=False)] = 1.0
    return Y


def labels_csr(m: int, L: int, p: int, rng: np.random.Generator):
    """The same label draw as :func:`labels_dense`, returned as CSR."""
    cols = np.empty((m, p), dtype=np.int32)
    for i in range(m):
        cols[i] = np.sort(rng.choice(L, p, replace=False))
    rowptr = np.arange(0, m * p + 1, p, dtype=np.int64)
    return rowptr, cols.reshape(-1), np.ones(m * p, dtype=np.float64)


def make(name: str, seed: int = 0, with_y: bool = True):
    """Build one named workload.  Returns a dict with CSR A, Y and the config."""
    cfg = CONFIGS[name]
    rng = np.random.default_rng(seed)
    rowptr, col, val = chung_lu_csr(cfg.m, cfg.n, cfg.nnz, cfg.gamma, rng, cfg.binary)
    out = {"cfg": cfg, "m": cfg.m, "n": cfg.n, "rowptr": rowptr, "col": col, "val": val}
    if with_y:
        if cfg.sparse_y:
            out["Y_csr"] = labels_csr(cfg.m, cfg.L, cfg.p, rng)
        else:
            out["Y"] = labels_dense(cfg.m, cfg.L, cfg.p, rng)
    return out


def make_many(count: int = 256, seed: int = 0, lo: int = 1000, hi: int = 50_000,
              L: int = 200, p: int = 5, gamma: float = 2.1):
    """Many independent instances: m log-uniform in [lo, hi], n = m/4, nnz = 10 m,
    r = n/10.  Instance i uses SeedSequence(seed).spawn(count)[i]."""
    out = []
    for ss in np.random.SeedSequence(seed).spawn(count):
        rng = np.random.default_rng(ss)
        m = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = max(1, m // 4)
        nnz = min(10 * m, m * n)
        rowptr, col, val = chung_lu_csr(m, n, nnz, gamma, rng)
        Y = labels_dense(m, L, p, rng)
        out.append({"m": m, "n": n, "rowptr": rowptr, "col": col, "val": val, "Y": Y,
                    "r": max(1, n // 10)})
    return out


def make_tiny_random(m: int, n: int, density: float, rng: np.random.Generator,
                     binary: bool = False):
    """Uniform random sparse matrix for small unit tests (CSR)."""
    mask = rng.random((m, n)) < density
    vals = np.where(mask, 1.0 if binary else 1.0 - rng.random((m, n)), 0.0)
    rows, cols = np.nonzero(mask)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals[rows, cols].astype(np.float64)


def _coo_to_csr(m: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """CSR with sorted, duplicate-free columns per row (first occurrence kept)."""
    keys = rows.astype(np.int64) * (int(cols.max()) + 1 if cols.size else 1) + cols
    _, first = np.unique(keys, return_index=True)
    rows, cols, vals = rows[first], cols[first], vals[first]
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), vals.astype(np.float64)


def make_long_blocks(seed: int = 0):
    """A matrix whose hub-and-spoke reordering (k = 0.0006) has long diagonal
    blocks: spokes of 1500 x 200, 2200 x 150 and 300 x 1500 (random sparse
    rows of 3 entries, columns of 2 entries for the wide one) and a final giant
    component that is a star of 3000 rows on one column.  Five dense "hub" rows
    and two "hub" columns of the highest degrees join everything, so that the
    first iteration removes exactly them and the star, with a single feature,
    ends the loop.  Values uniform(0, 1].  Returns (m, n, rowptr, col, val)."""
    rng = np.random.default_rng(seed)
    specs = [(1500, 200, "rows"), (2200, 150, "rows"), (300, 1500, "cols")]
    r0 = 5                       # hub rows first, then the blocks, then the star
    c0 = 2                       # hub columns first
    R, Cc = [], []
    row_ranges, col_ranges = [], []
    ro, co = r0, c0
    for mb, nb, kind in specs:
        if kind == "rows":
            rr = np.repeat(np.arange(mb), 3)
            cc = np.concatenate([rng.choice(nb, 3, replace=False) for _ in range(mb)])
        else:
            cc = np.repeat(np.arange(nb), 2)
            rr = np.concatenate([rng.choice(mb, 2, replace=False) for _ in range(nb)])
        R.append(rr + ro)
        Cc.append(cc + co)
        row_ranges.append((ro, ro + mb))
        col_ranges.append((co, co + nb))
        ro += mb
        co += nb
    star_rows = np.arange(ro, ro + 3000)
    star_col = co
    R.append(star_rows)
    Cc.append(np.full(3000, star_col))
    m, n = ro + 3000, co + 1
    # hub rows: 600 random columns each; hub columns: 4000 random rows each
    for i in range(r0):
        R.append(np.full(600, i))
        Cc.append(rng.choice(np.arange(c0, n), 600, replace=False))
    for j in range(c0):
        R.append(rng.choice(np.arange(r0, m), 4000, replace=False))
        Cc.append(np.full(4000, j))
    rows = np.concatenate(R)
    cols = np.concatenate(Cc)
    vals = 1.0 - rng.random(rows.size)
    # shuffle row and column ids so nothing is pre-sorted
    prow, pcol = rng.permutation(m), rng.permutation(n)
    rowptr, col, val = _coo_to_csr(m, prow[rows], pcol[cols], vals)
    return m, n, rowptr, col, val
