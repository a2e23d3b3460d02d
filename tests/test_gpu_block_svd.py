"""Eq. 1 on the GPU against LAPACK, block by block.

fastpi_block_svd runs Algorithm 2 and the batched SVD of the diagonal blocks
of A11 and returns the s_i = min(ceil(alpha n_1i), m_1i, n_1i) kept singular
values of every block.  Each block's values are compared with LAPACK's SVD of
that block (numpy.linalg.svd of the dense block of the reordered A; a block
with one row or one column has the single singular value |block|_F).  The
blocks come from the oracle's reordering (Algorithm 2), which the library
must reproduce bit for bit.

Workloads: the 200 000 x 50 000 one (95 924 blocks up to 1 299 x 503: every
register-tile class of the batched Jacobi kernels), and a matrix built to
give long blocks (1 500 x 200, 300 x 1 500, 2 200 x 150 and 3 000 x 1), which
reach the kernels' long-column paths (FP32 beyond 1 408 rows, FP64 beyond
2 048 rows).  Tolerance per block: max |sigma_gpu - sigma_lapack| <= tol *
sigma_max(block), tol = 1e-11 in FP64; in the mixed form the FP32 column
norms and dot products of a block with p rows are p-term FP32 sums, whose
relative error is bounded by p 2^-24, so tol = max(1e-5, 2 p 2^-24).
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from gpu_common import binding
from oracle.reorder import reorder as oracle_reorder

pytestmark = pytest.mark.gpu
TOL = {"fp64": lambda p: 1e-11, "mixed": lambda p: max(1e-5, 2.0 * p * 2.0 ** -24)}


def _lapack_block_sigmas(m, n, rowptr, col, val, R, r):
    """Kept singular values of every A11 block (list, one array per block),
    from LAPACK on the dense block, or |block|_F for a block with one row or
    one column."""
    A = sp.csr_matrix((val, col, rowptr), shape=(m, n))
    A11 = A[R.row_order][:, R.col_order][:R.m1, :R.n1].tocoo()
    ro, co = np.asarray(R.row_off), np.asarray(R.col_off)
    mb, nb = np.diff(ro), np.diff(co)
    s_i = np.minimum(np.minimum((r * nb + n - 1) // n, mb), nb)
    blk_of_row = np.repeat(np.arange(mb.size), mb)
    b = blk_of_row[A11.row]
    order = np.argsort(b, kind="stable")
    b, ri, ci, vi = b[order], A11.row[order], A11.col[order], A11.data[order]
    starts = np.searchsorted(b, np.arange(mb.size + 1))
    out = []
    for k in range(mb.size):
        if s_i[k] == 0:
            out.append(np.zeros(0))
            continue
        e0, e1 = starts[k], starts[k + 1]
        if min(mb[k], nb[k]) == 1:
            out.append(np.array([np.sqrt(np.sum(vi[e0:e1] ** 2))]))
            continue
        D = np.zeros((mb[k], nb[k]))
        D[ri[e0:e1] - ro[k], ci[e0:e1] - co[k]] = vi[e0:e1]
        out.append(np.linalg.svd(D, compute_uv=False)[:s_i[k]])
    return out


def _check(m, n, rowptr, col, val, k, r, prec, R=None, ref=None):
    fp = binding()
    R = R if R is not None else oracle_reorder(m, n, rowptr, col, k)
    ref = ref if ref is not None else _lapack_block_sigmas(m, n, rowptr, col, val, R, r)
    h = fp.FastPI(m, n, rowptr, col, val, device="cuda:0")
    got = h.block_svd(r, k, prec)
    bro, bco = h.blocks()
    ro, co, _, _ = h.perm()
    inf = h.info()
    h.close()
    assert np.array_equal(ro, R.row_order) and np.array_equal(co, R.col_order)
    assert np.array_equal(bro, R.row_off) and np.array_equal(bco, R.col_off)
    assert got.size == sum(x.size for x in ref) == inf["S"]
    pmax = np.maximum(np.diff(R.row_off), np.diff(R.col_off))
    pos, worst = 0, 0.0
    for b, x in enumerate(ref):
        if x.size == 0:
            continue
        g = got[pos:pos + x.size]
        pos += x.size
        assert np.all(np.diff(g) <= 0), "not descending within a block"
        err = float(np.max(np.abs(g - x)) / x[0]) if x[0] > 0 else float(np.max(np.abs(g)))
        assert err <= TOL[prec](int(pmax[b])), f"{prec}: block {b} ({pmax[b]} rows) error {err:.3e}"
        worst = max(worst, err)
    return R, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_svd_long_blocks(prec):
    """Spoke blocks of 1 500, 2 200 and (transposed) 1 500 rows and a star of
    3 000 rows on one column, every singular value kept (r = n)."""
    m, n, rowptr, col, val = workloads.make_long_blocks()
    R, _ = _check(m, n, rowptr, col, val, 0.0006, n, prec)
    sizes = sorted(max(a, b) for a, b in zip(np.diff(R.row_off), np.diff(R.col_off)))
    assert sizes[-3:] == [1500, 2200, 3000] and R.iterations == 1


@pytest.fixture(scope="module")
def large_blocks():
    w = workloads.make("large", with_y=False)
    cfg = w["cfg"]
    R = oracle_reorder(w["m"], w["n"], w["rowptr"], w["col"], cfg.k)
    ref = _lapack_block_sigmas(w["m"], w["n"], w["rowptr"], w["col"], w["val"], R, cfg.r)
    return w, R, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_svd_large_every_block(large_blocks, prec):
    w, R, ref = large_blocks
    cfg = w["cfg"]
    _check(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.k, cfg.r, prec, R=R, ref=ref)


def test_block_svd_arguments():
    fp = binding()
    m, n, rowptr, col, val = workloads.make_long_blocks()
    h = fp.FastPI(m, n, rowptr, col, val, device="cuda:0")
    with pytest.raises(fp.FastPIError) as e:
        h.block_svd(0, 0.01)
    assert e.value.status == 1
    with pytest.raises(fp.FastPIError) as e:
        h.block_svd(10, 1.5)
    assert e.value.status == 1
    h.block_svd(10, 0.0006)
    with pytest.raises(fp.FastPIError) as e:
        h.U()                      # no factors after the block stage alone
    assert e.value.status == 6
    h.close()
