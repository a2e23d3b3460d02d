"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: the permutation and block list are integer results and must match
bit for bit; in FP64 mode the singular values must match to relative
Frobenius error 1e-10 and Z = A^+ Y to 1e-9; the mixed-precision mode must
reach the FP64 residual |AZ - Y|_F to within a relative 1e-3.  Z is compared
only when every truncation gap (sigma_keep_last - sigma_drop_first) / sigma_1
exceeds 1e-8 on the oracle side, because a smaller gap makes the kept
subspace (and Z) ill-determined: several answers are then correct, and only
Sigma and the residual are checked.
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads
from oracle import fastpi as ofp
from oracle.reorder import reorder as oreorder
from tests.gpu_common import binding, dense, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(__file__), "golden")
BIG = 1 << 30   # a chunk at least as large as any border: the single-shot form


def _gap(f):
    if not f.gaps or f.S.size == 0:
        return np.inf
    return min((a - b) for a, b in f.gaps) / f.S[0]


def _handle(w_or_tuple):
    fp = binding()
    m, n, rowptr, col, val = w_or_tuple
    return fp.FastPI(m, n, rowptr, col, val, device=DEV)


def _tiny(seed, m=None, n=None):
    rng = np.random.default_rng(seed)
    m = m or int(rng.integers(4, 40))
    n = n or int(rng.integers(3, 25))
    rowptr, col, val = workloads.make_tiny_random(m, n, float(rng.uniform(0.05, 0.4)), rng)
    return m, n, rowptr, col, val


# ----------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("seed", range(10))
def test_reorder_bitexact_tiny(seed):
    m, n, rowptr, col, val = _tiny(seed)
    k = [0.05, 0.1, 0.2, 0.34, 0.5][seed % 5]
    h = _handle((m, n, rowptr, col, val)).factor(1, k)
    ro, co, m2, n2 = h.perm()
    R = oreorder(m, n, rowptr, col, k)
    assert ro.tolist() == R.row_order.tolist()
    assert co.tolist() == R.col_order.tolist()
    assert (m2, n2) == (R.m2, R.n2)
    bro, bco = h.blocks()
    assert bro.tolist() == R.row_off.tolist() and bco.tolist() == R.col_off.tolist()


@pytest.mark.parametrize("name", ["fig2_toy.json", "star.json", "one_side_stop.json"])
def test_reorder_golden(name):
    g = json.load(open(os.path.join(GOLD, name)))
    m, n = g["m"], g["n"]
    edges = sorted(set(map(tuple, g["edges_row_col"])))
    rowptr = np.zeros(m + 1, dtype=np.int64)
    for r, _ in edges:
        rowptr[r + 1] += 1
    rowptr = np.cumsum(rowptr)
    col = np.array([c for _, c in edges], dtype=np.int32)
    val = np.ones(len(edges))
    h = _handle((m, n, rowptr, col, val)).factor(1, g["k"])
    ro, co, _, _ = h.perm()
    assert ro.tolist() == g["row_order"] and co.tolist() == g["col_order"]
    bro, bco = h.blocks()
    assert bro.tolist() == g["row_off"] and bco.tolist() == g["col_off"]
    assert h.info()["iterations"] == g["iterations"]


@pytest.mark.parametrize("name", ["small", "medium"])
def test_reorder_bitexact_workloads(name):
    w = workloads.make(name, with_y=False)
    h = _handle((w["m"], w["n"], w["rowptr"], w["col"], w["val"])).factor(w["cfg"].r, w["cfg"].k, "mixed")
    ro, co, m2, n2 = h.perm()
    R = oreorder(w["m"], w["n"], w["rowptr"], w["col"], w["cfg"].k)
    assert np.array_equal(ro, R.row_order) and np.array_equal(co, R.col_order)
    bro, bco = h.blocks()
    assert np.array_equal(bro, R.row_off) and np.array_equal(bco, R.col_off)
    inf = h.info()
    assert inf["iterations"] == R.iterations and inf["m1"] == R.m1 and inf["n1"] == R.n1


# ----------------------------------------------------------------- FP64 factor + apply
def _parity(m, n, rowptr, col, val, Y, r, k, cr, cc, ztol=1e-9, stol=1e-10):
    f = ofp.factor(m, n, rowptr, col, val, r, k, chunk_row=cr, chunk_col=cc)
    Zo = ofp.apply(f, Y)
    h = _handle((m, n, rowptr, col, val)).factor(r, k, "fp64", cr or BIG, cc or BIG)
    S = h.S()
    assert S.size == f.S.size
    assert rel(S, f.S) <= stol, f"sigma rel err {rel(S, f.S):.3e}"
    Yd = torch.from_numpy(Y).to(DEV)
    Z = h.apply(Yd).cpu().numpy()
    inf = h.info()
    if _gap(f) > 1e-8:
        assert rel(Z, Zo) <= ztol, f"Z rel err {rel(Z, Zo):.3e}"
    # residual through the library equals the dense residual (when A has full
    # row rank the system is consistent, A Z = Y, and both are rounding noise:
    # hence the absolute floor, relative to |Y|)
    A = dense(m, n, rowptr, col, val)
    res = h.residual(Yd, torch.from_numpy(Z).to(DEV))
    np.testing.assert_allclose(res, np.linalg.norm(A @ Z - Y), rtol=1e-12, atol=1e-12 * np.linalg.norm(Y))
    return h, f, inf


@pytest.mark.parametrize("chunks", [(None, None), (64, 64), (37, 23), (1, 5)])
def test_factor_fp64_small(chunks):
    w = workloads.make("small")
    cfg = w["cfg"]
    _parity(w["m"], w["n"], w["rowptr"], w["col"], w["val"], w["Y"], cfg.r, cfg.k, *chunks)


@pytest.mark.parametrize("shape", [(1, 6), (7, 1), (1, 1), (5, 5)])
@pytest.mark.parametrize("chunks", [(None, None), (1, 1)])
def test_one_sided_empty_a11(shape, chunks):
    """Inputs where Algorithm 2 leaves A11 empty on one side or both (a single
    row, a single column, 1 x 1, a dense 5 x 5 whose nodes all become hubs),
    at r = 2n: FP64 equal to the oracle, and both forms equal to LAPACK's
    pinv (the mixed form to FP32 accuracy)."""
    m, n = shape
    rng = np.random.default_rng(m * 10 + n)
    A = rng.uniform(0.1, 1.0, shape)
    rowptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), m)
    val = A.reshape(-1).copy()
    Y = rng.standard_normal((m, 3))
    Zp = np.linalg.pinv(A) @ Y
    h, f, inf = _parity(m, n, rowptr, col, val, Y, 2 * n, 0.3, *chunks)
    assert (inf["m1"], inf["n1"]) == (f.reo.m1, f.reo.n1)
    assert min(inf["m1"], inf["n1"]) == 0
    assert rel(h.apply(torch.from_numpy(Y).to(DEV)).cpu().numpy(), Zp) <= 1e-12
    g = _handle((m, n, rowptr, col, val)).factor(2 * n, 0.3, "mixed", chunks[0] or BIG, chunks[1] or BIG)
    assert rel(g.apply(torch.from_numpy(Y).to(DEV)).cpu().numpy(), Zp) <= 1e-5


@pytest.mark.parametrize("seed", range(6))
def test_factor_fp64_tiny_truncated(seed):
    m, n, rowptr, col, val = _tiny(100 + seed, m=60, n=25)
    Y = workloads.labels_dense(m, 4, 2, np.random.default_rng(seed))
    r = [3, 5, 8, 12, 20, 25][seed]
    _parity(m, n, rowptr, col, val, Y, r, 0.1, [None, 3, 7, 2, 5, 1][seed], [None, 2, 4, 9, 1, 3][seed])


@pytest.mark.parametrize("seed", range(4))
def test_alpha_one_is_exact_pinv(seed):
    """alpha = 1: Sigma equals the dense SVD and A^+ Y equals the Moore-Penrose solve."""
    rng = np.random.default_rng(7 + seed)
    m, n = 90, 30
    rowptr, col, val = workloads.chung_lu_csr(m, n, 400, 2.1, rng)
    A = dense(m, n, rowptr, col, val)
    Y = workloads.labels_dense(m, 5, 2, rng)
    h = _handle((m, n, rowptr, col, val)).factor(n, 0.05, "fp64", 4, 3)
    sv = np.linalg.svd(A, compute_uv=False)
    S = h.S()
    np.testing.assert_allclose(S[:sv.size], sv, atol=1e-12 * sv[0])
    Z = h.apply(torch.from_numpy(Y).to(DEV)).cpu().numpy()
    Zp = np.linalg.pinv(A) @ Y
    assert rel(Z, Zp) <= 1e-9
    U, V = h.U().cpu().numpy(), h.V().cpu().numpy()
    assert np.linalg.norm(A - (U * S) @ V.T) <= 1e-12 * np.linalg.norm(A)


def test_apply_variants_agree():
    w = workloads.make("small")
    cfg = w["cfg"]
    h = _handle((w["m"], w["n"], w["rowptr"], w["col"], w["val"])).factor(cfg.r, cfg.k, "fp64", 64, 64)
    Yd = torch.from_numpy(w["Y"]).to(DEV)
    Z = h.apply(Yd).cpu().numpy()
    Zh = h.apply_host(w["Y"])
    assert rel(Zh, Z) <= 1e-14
    rp, cl, vl = workloads.labels_csr(w["m"], cfg.L, cfg.p, np.random.default_rng(5))
    Yc = dense(w["m"], cfg.L, rp, cl, vl)
    Zc = h.apply_csr(cfg.L, torch.from_numpy(rp).to(DEV), torch.from_numpy(cl).to(DEV),
                     torch.from_numpy(vl).to(DEV)).cpu().numpy()
    Zd = h.apply(torch.from_numpy(Yc).to(DEV)).cpu().numpy()
    assert rel(Zc, Zd) <= 1e-12


def test_apply_csr_rejects_malformed_labels():
    """A label CSR with a label outside [0, L), or a row whose labels are not
    increasing, is refused with FASTPI_ERR_CSR before anything reads Y by
    label, and the handle keeps working."""
    fp = binding()
    w = workloads.make("small")
    cfg = w["cfg"]
    h = _handle((w["m"], w["n"], w["rowptr"], w["col"], w["val"])).factor(cfg.r, cfg.k, "fp64", 64, 64)
    rp, cl, vl = workloads.labels_csr(w["m"], cfg.L, cfg.p, np.random.default_rng(5))
    good = h.apply_csr(cfg.L, *(torch.from_numpy(a).to(DEV) for a in (rp, cl, vl))).cpu().numpy()
    bad_range = cl.copy()
    bad_range[7] = cfg.L                            # label L in an L-label matrix
    bad_order = cl.copy()
    bad_order[0], bad_order[1] = cl[1], cl[0]       # row 0 decreasing
    for bad in (bad_range, bad_order):
        with pytest.raises(fp.FastPIError) as e:
            h.apply_csr(cfg.L, *(torch.from_numpy(a).to(DEV) for a in (rp, bad, vl)))
        assert e.value.status == 2
    again = h.apply_csr(cfg.L, *(torch.from_numpy(a).to(DEV) for a in (rp, cl, vl))).cpu().numpy()
    assert np.array_equal(again, good)


def test_getters_original_order():
    """U and V come back in the caller's row / column order: A ~ U S V^T."""
    w = workloads.make("small")
    cfg = w["cfg"]
    h = _handle((w["m"], w["n"], w["rowptr"], w["col"], w["val"])).factor(cfg.r, cfg.k, "fp64", 64, 64)
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, 64, 64)
    U, V, S = h.U().cpu().numpy(), h.V().cpu().numpy(), h.S()
    np.testing.assert_allclose(U.T @ U, np.eye(S.size), atol=1e-11)
    np.testing.assert_allclose(V.T @ V, np.eye(S.size), atol=1e-11)
    Xg = (U * S) @ V.T
    Xo = (f.U * f.S) @ f.V.T
    if _gap(f) > 1e-8:
        assert rel(Xg, Xo) <= 1e-9


# ----------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("chunks", [(64, 64), (None, None)])
def test_mixed_residual_within_1e3(chunks):
    w = workloads.make("small")
    cfg = w["cfg"]
    args = (w["m"], w["n"], w["rowptr"], w["col"], w["val"])
    Yd = torch.from_numpy(w["Y"]).to(DEV)
    h64 = _handle(args).factor(cfg.r, cfg.k, "fp64", chunks[0] or BIG, chunks[1] or BIG)
    h32 = _handle(args).factor(cfg.r, cfg.k, "mixed", chunks[0] or BIG, chunks[1] or BIG)
    r64 = h64.residual(Yd, h64.apply(Yd))
    r32 = h32.residual(Yd, h32.apply(Yd))
    assert abs(r32 - r64) / r64 <= 1e-3
    s64, s32 = h64.S(), h32.S()
    assert rel(s32, s64) <= 1e-3


@pytest.mark.parametrize("shape", [(90, 30, 4, 3), (400, 150, 40, 30), (1500, 420, 300, 200)])
def test_mixed_alpha_one_fp32_accuracy(shape):
    """Mixed precision at alpha = 1 reproduces the exact SVD closely: singular
    values, reconstruction A = U S V^T and orthonormal U, V.  The mixed mode
    drops residual directions below 1e-5 of the largest appended column norm;
    accumulated over the chunks this removes a few of the smallest singular
    values and moves the others by up to ~2e-3 sigma_1, so the bounds here are
    5e-3 sigma_1 (the check still exercises the FP32 core SVD end to end,
    including cores wider than the on-chip cluster path holds)."""
    m, n, cr, cc = shape
    rng = np.random.default_rng(11)
    rowptr, col, val = workloads.chung_lu_csr(m, n, 12 * n, 2.1, rng)
    A = dense(m, n, rowptr, col, val)
    h = _handle((m, n, rowptr, col, val)).factor(n, 0.02, "mixed", cr, cc)
    S = h.S()
    sv = np.linalg.svd(A, compute_uv=False)
    big = sv > 1e-2 * sv[0]
    assert S.size >= np.count_nonzero(big)
    np.testing.assert_allclose(S[:np.count_nonzero(big)], sv[big], atol=5e-3 * sv[0])
    U, V = h.U().cpu().numpy(), h.V().cpu().numpy()
    assert np.linalg.norm(A - (U * S) @ V.T) <= 5e-3 * np.linalg.norm(A)
    live = S > 1e-2 * S[0]
    Ul, Vl = U[:, live], V[:, live]
    assert np.abs(Ul.T @ Ul - np.eye(Ul.shape[1])).max() <= 1e-3
    assert np.abs(Vl.T @ Vl - np.eye(Vl.shape[1])).max() <= 1e-3


# ----------------------------------------------------------------- errors / edge cases
def test_errors():
    fp = binding()
    rowptr = np.array([0, 2, 1], dtype=np.int64)   # not monotone
    with pytest.raises(fp.FastPIError) as e:
        fp.FastPI(2, 3, rowptr, np.array([0, 1], dtype=np.int32), np.ones(2), device=DEV)
    assert e.value.status == 2
    with pytest.raises(fp.FastPIError) as e:       # unsorted columns
        fp.FastPI(1, 3, np.array([0, 2]), np.array([2, 1], dtype=np.int32), np.ones(2), device=DEV)
    assert e.value.status == 2
    with pytest.raises(fp.FastPIError) as e:       # column out of range
        fp.FastPI(1, 3, np.array([0, 1]), np.array([3], dtype=np.int32), np.ones(1), device=DEV)
    assert e.value.status == 2
    h = fp.FastPI(2, 2, np.array([0, 1, 2]), np.array([0, 1], dtype=np.int32), np.ones(2), device=DEV)
    with pytest.raises(fp.FastPIError) as e:
        h.S()
    assert e.value.status == 6
    for bad_k in (0.0, 1.0, -0.1):
        with pytest.raises(fp.FastPIError) as e:
            h.factor(1, bad_k)
        assert e.value.status == 1
    with pytest.raises(fp.FastPIError):
        h.factor(0, 0.1)


def test_empty_rows_cols_and_zero_matrix():
    # rows / columns without entries, and a matrix with no nonzero at all
    m, n = 12, 7
    rowptr = np.array([0, 0, 1, 1, 3, 3, 3, 4, 4, 4, 5, 5, 5], dtype=np.int64)
    col = np.array([2, 0, 2, 2, 6], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0, 0.5, 4.0])
    Y = workloads.labels_dense(m, 3, 1, np.random.default_rng(1))
    _parity(m, n, rowptr, col, val, Y, 3, 0.2, None, None)
    h = _handle((m, n, np.zeros(m + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))).factor(2, 0.2)
    assert np.all(h.S() == 0)
    Z = h.apply(torch.from_numpy(Y).to(DEV))
    assert torch.all(Z == 0)
