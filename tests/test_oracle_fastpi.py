"""Pins for the FastPI factorization / solve oracle (Algorithm 1, Eqs. 1-3,
Problem 1, Application 1).

Every check compares the oracle with something fixed by the paper or by
mathematics, not with itself:
  * Problem 1: with r = rank(A) (alpha = 1 here) the pseudoinverse is exact:
    the four Penrose conditions, the normal equations A^T (A Z - Y) = 0,
    Z = lstsq(A, Y) when A has full column rank, singular values equal to
    LAPACK's SVD of the dense A, exact reconstruction A = U Sigma V^T.
  * closed forms: diagonal A (A^+ = diag(1/d)), rank-1 A = a b^T
    (A^+ = b a^T / (|a|^2 |b|^2)), 1 x 1 / p x 1 / 1 x q blocks of Eq. 1.
  * Eq. 1 block-diagonal invariance: the multiset of block singular values is
    the spectrum of A11.
  * Eqs. 2 / 3 single shot (dense M and N as printed) equal the incremental
    form when the whole border is one chunk; at alpha = 1 every chunking gives
    the exact SVD.
  * Eckart-Young: no rank-r factorization beats the optimal residual.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fastpi, pinv
from oracle.reorder import Reordering, reorder


def _dense(m, n, rowptr, col, val):
    return sp.csr_matrix((val, col, rowptr), shape=(m, n)).toarray()


def _csr(A):
    c = sp.csr_matrix(A)
    c.sort_indices()
    return c.indptr.astype(np.int64), c.indices.astype(np.int32), c.data.astype(np.float64)


def _powerlaw(seed, m=120, n=40, nnz=600, gamma=2.1):
    rng = np.random.default_rng(seed)
    return workloads.chung_lu_csr(m, n, nnz, gamma, rng)


def test_ceil_alpha():
    assert fastpi.ceil_alpha(7, 1, 10) == 1        # ceil(0.7)
    assert fastpi.ceil_alpha(10, 1, 10) == 1
    assert fastpi.ceil_alpha(11, 1, 10) == 2       # ceil(1.1)
    assert fastpi.ceil_alpha(0, 3, 10) == 0
    assert fastpi.ceil_alpha(40, 40, 40) == 40     # alpha = 1


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("chunks", [(None, None), (3, 2), (17, 5)])
def test_alpha_one_exact_svd_and_penrose(seed, chunks):
    """alpha = 1: the incremental SVD is exact (r = rank), so A^+ is the Moore-Penrose inverse."""
    m, n = 120, 40
    rowptr, col, val = _powerlaw(seed, m, n)
    A = _dense(m, n, rowptr, col, val)
    f = fastpi.factor(m, n, rowptr, col, val, r=n, k=0.05, chunk_row=chunks[0], chunk_col=chunks[1])
    sv = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(f.S[:sv.size], sv, rtol=0, atol=1e-12 * sv[0])
    assert np.linalg.norm(A - (f.U * f.S) @ f.V.T) <= 1e-12 * np.linalg.norm(A)
    tau = fastpi.pinv_threshold(f.S, m, n)
    inv = np.where(f.S > tau, 1.0 / np.maximum(f.S, tau), 0.0)
    X = (f.V * inv) @ f.U.T
    nA = np.linalg.norm(A)
    nX = np.linalg.norm(X)
    assert np.linalg.norm(A @ X @ A - A) <= 1e-10 * nA
    assert np.linalg.norm(X @ A @ X - X) <= 1e-10 * nX
    assert np.linalg.norm((A @ X).T - A @ X) <= 1e-10
    assert np.linalg.norm((X @ A).T - X @ A) <= 1e-10
    np.testing.assert_allclose(X, pinv.dense_pinv(A), atol=1e-10 * nX)


@pytest.mark.parametrize("seed", range(3))
def test_alpha_one_lstsq_and_normal_equations(seed):
    m, n = 150, 30
    rng = np.random.default_rng(50 + seed)
    # a dense diagonal guarantees full column rank; extra power-law entries on top
    rowptr, col, val = _powerlaw(50 + seed, m, n, 500)
    A = _dense(m, n, rowptr, col, val)
    A[np.arange(n), np.arange(n)] += 1.0 + rng.random(n)
    rowptr, col, val = _csr(A)
    Y = workloads.labels_dense(m, 7, 2, rng)
    f = fastpi.factor(m, n, rowptr, col, val, r=n, k=0.03, chunk_row=4, chunk_col=3)
    Z = fastpi.apply(f, Y)
    Zl = np.linalg.lstsq(A, Y, rcond=None)[0]
    np.testing.assert_allclose(Z, Zl, atol=1e-10 * np.linalg.norm(Zl))
    assert np.linalg.norm(A.T @ (A @ Z - Y)) <= 1e-10 * np.linalg.norm(A) * np.linalg.norm(Y)


def test_diagonal_matrix_closed_form():
    d = np.array([3.0, 0.5, 2.0, 7.0, 1.25, 0.1])
    A = np.zeros((8, 6))
    A[np.arange(6), np.arange(6)] = d
    rowptr, col, val = _csr(A)
    f = fastpi.factor(8, 6, rowptr, col, val, r=6, k=0.2)
    np.testing.assert_allclose(np.sort(f.S)[::-1], np.sort(d)[::-1], rtol=1e-15)
    Y = np.eye(8)
    X = fastpi.apply(f, Y)                       # = A^+
    Xd = np.zeros((6, 8))
    Xd[np.arange(6), np.arange(6)] = 1.0 / d
    np.testing.assert_allclose(X, Xd, atol=1e-14)


def test_rank_one_closed_form():
    rng = np.random.default_rng(3)
    a = rng.random(9) + 0.1
    b = rng.random(5) + 0.1
    A = np.outer(a, b)
    rowptr, col, val = _csr(A)
    f = fastpi.factor(9, 5, rowptr, col, val, r=5, k=0.2, chunk_row=2, chunk_col=1)
    X = fastpi.apply(f, np.eye(9))
    Xc = np.outer(b, a) / (a @ a * (b @ b))
    np.testing.assert_allclose(X, Xc, atol=1e-12 * np.linalg.norm(Xc))
    assert f.S[0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b), rel=1e-14)
    assert np.all(f.S[1:] <= 1e-12 * f.S[0])


def test_block_svd_closed_forms_and_invariance():
    """Eq. 1 on hand-made blocks: 1x1 -> |a|, p x 1 -> column norm, 1 x q -> row norm;
    untruncated, the block singular values are the spectrum of A11."""
    m, n = 30, 20
    rowptr, col, val = _powerlaw(7, m, n, 70)
    A = _dense(m, n, rowptr, col, val)
    R = reorder(m, n, rowptr, col, 0.1)
    _, A11, _, _ = fastpi.split(sp.csr_matrix(A), R)
    U1, s1, V1, si = fastpi.block_svd(A11, R, r=n, n=n)
    A11d = A11.toarray()
    sv = np.linalg.svd(A11d, compute_uv=False) if A11d.size else np.zeros(0)
    sv = np.sort(sv[sv > 1e-12])[::-1]
    got = np.sort(s1[s1 > 1e-12])[::-1]
    np.testing.assert_allclose(got, sv, rtol=1e-13)
    assert np.linalg.norm(A11d - (U1 * s1) @ V1.T) <= 1e-12 * max(1.0, np.linalg.norm(A11d))
    ro, co = R.row_off, R.col_off
    pos = np.concatenate([[0], np.cumsum(si)])
    for b in range(len(ro) - 1):
        blk = A11d[ro[b]:ro[b + 1], co[b]:co[b + 1]]
        if si[b] == 0:
            continue
        if blk.shape == (1, 1):
            assert s1[pos[b]] == pytest.approx(abs(blk[0, 0]), rel=1e-15)
        elif blk.shape[1] == 1:
            assert s1[pos[b]] == pytest.approx(np.linalg.norm(blk), rel=1e-14)
        elif blk.shape[0] == 1:
            assert s1[pos[b]] == pytest.approx(np.linalg.norm(blk), rel=1e-14)


def test_block_truncation_rule():
    """s_i = min(ceil(alpha n_1i), m_1i, n_1i) with alpha = r / n."""
    m, n = 200, 60
    rowptr, col, val = _powerlaw(11, m, n, 500)
    R = reorder(m, n, rowptr, col, 0.05)
    A = sp.csr_matrix((val, col, rowptr), shape=(m, n))
    _, A11, _, _ = fastpi.split(A, R)
    r = 13
    _, _, _, si = fastpi.block_svd(A11, R, r=r, n=n)
    mi, ni = np.diff(R.row_off), np.diff(R.col_off)
    expect = np.minimum(np.minimum(np.ceil(r * ni / n - 1e-12).astype(int), mi), ni)
    assert np.array_equal(si, expect)


def test_block_ranks_hand_computed():
    """Eq. 1 on hand-made blocks of A11 (m_1i x n_1i): 2 x 10, 10 x 2, 3 x 3,
    4 x 5, 1 x 1, with alpha = r / n = 21 / 42 = 0.5.  The kept rank of a block
    is set by its column count: ceil(0.5 * 10) = 5 capped by 2 rows -> 2;
    ceil(0.5 * 2) = 1; ceil(1.5) = 2; ceil(2.5) = 3; ceil(0.5) = 1.  Each block
    keeps its s_i largest singular values (LAPACK on the block alone) with
    singular vectors supported on the block's rows and columns."""
    shapes = [(2, 10), (10, 2), (3, 3), (4, 5), (1, 1)]
    expect = [2, 1, 2, 3, 1]
    ro = np.concatenate([[0], np.cumsum([a for a, _ in shapes])])
    co = np.concatenate([[0], np.cumsum([b for _, b in shapes])])
    m1, n1 = int(ro[-1]), int(co[-1])
    rng = np.random.default_rng(3)
    A11 = np.zeros((m1, n1))
    for b, (p, q) in enumerate(shapes):
        A11[ro[b]:ro[b + 1], co[b]:co[b + 1]] = rng.uniform(0.1, 1.0, (p, q))
    R = Reordering(m1, n1, np.arange(m1), np.arange(n1), ro, co, m1, n1, 1, [])
    U1, s1, V1, si = fastpi.block_svd(sp.csr_matrix(A11), R, r=21, n=42)
    assert si.tolist() == expect
    pos = np.concatenate([[0], np.cumsum(expect)])
    for b in range(len(shapes)):
        blk = A11[ro[b]:ro[b + 1], co[b]:co[b + 1]]
        sv = np.linalg.svd(blk, compute_uv=False)[:expect[b]]
        np.testing.assert_allclose(s1[pos[b]:pos[b + 1]], sv, rtol=1e-13)
        outside_r = np.delete(U1[:, pos[b]:pos[b + 1]], np.s_[ro[b]:ro[b + 1]], axis=0)
        outside_c = np.delete(V1[:, pos[b]:pos[b + 1]], np.s_[co[b]:co[b + 1]], axis=0)
        assert not outside_r.any() and not outside_c.any()
        Ub = U1[ro[b]:ro[b + 1], pos[b]:pos[b + 1]]
        Vb = V1[co[b]:co[b + 1], pos[b]:pos[b + 1]]
        np.testing.assert_allclose(blk @ Vb, Ub * sv[None, :], atol=1e-13)


def test_alpha_above_one_caps_the_phase_ranks():
    """r = 2n (alpha = 2) on a matrix of full column rank: no phase can hold
    more triplets than its matrix has columns, so the row phase keeps
    rank [A11; A21] = n1 triplets (M has n1 columns) and the result has
    rank(A) = n, with A's singular values exactly (LAPACK on the dense A)."""
    m, n = 90, 30
    rowptr, col, val = _powerlaw(17, m, n, 400)
    A = _dense(m, n, rowptr, col, val)
    A[np.arange(n), np.arange(n)] += 1.0          # full column rank
    rowptr, col, val = _csr(A)
    f = fastpi.factor(m, n, rowptr, col, val, r=2 * n, k=0.05, chunk_row=5, chunk_col=3)
    Ap = A[f.reo.row_order][:, f.reo.col_order]
    n1 = f.reo.n1
    assert np.linalg.matrix_rank(Ap[:, :n1]) == n1
    assert f.s_row == n1
    assert f.rank == n and f.S.size == n
    np.testing.assert_allclose(f.S, np.linalg.svd(A, compute_uv=False), rtol=1e-12)


@pytest.mark.parametrize("shape", [(1, 6), (7, 1), (1, 1), (5, 5)])
@pytest.mark.parametrize("chunk", [None, 1])
def test_degenerate_shapes_equal_lapack_pinv(shape, chunk):
    """A single row, a single column, a 1 x 1 and a fully dense matrix, with
    r = 2n (alpha >= 1): Algorithm 2 leaves A11 empty on one side (m1 = 0 or
    n1 = 0) or entirely, and the factorization must still give Z = A^+ Y
    exactly (LAPACK's pinv of the dense A)."""
    m, n = shape
    rng = np.random.default_rng(m * 10 + n)
    A = rng.uniform(0.1, 1.0, shape)
    rowptr, col, val = _csr(A)
    f = fastpi.factor(m, n, rowptr, col, val, r=2 * n, k=0.3, chunk_row=chunk, chunk_col=chunk)
    Y = rng.standard_normal((m, 3))
    np.testing.assert_allclose(fastpi.apply(f, Y), np.linalg.pinv(A) @ Y, atol=1e-13)
    np.testing.assert_allclose(f.S, np.linalg.svd(A, compute_uv=False), rtol=1e-13)


@pytest.mark.parametrize("alpha_r", [5, 12, 25])
def test_single_shot_equals_one_chunk(alpha_r):
    """Eqs. 2 and 3 as printed (dense M, N) equal the incremental form with one chunk."""
    m, n = 160, 50
    rowptr, col, val = _powerlaw(21, m, n, 800)
    f1 = fastpi.factor(m, n, rowptr, col, val, r=alpha_r, k=0.03, single_shot=True)
    f2 = fastpi.factor(m, n, rowptr, col, val, r=alpha_r, k=0.03)
    np.testing.assert_allclose(f2.S, f1.S, rtol=1e-12, atol=1e-13 * f1.S[0])
    Y = workloads.labels_dense(m, 6, 2, np.random.default_rng(0))
    Z1, Z2 = fastpi.apply(f1, Y), fastpi.apply(f2, Y)
    assert np.linalg.norm(Z1 - Z2) <= 1e-10 * np.linalg.norm(Z1)


@pytest.mark.parametrize("chunks", [(None, None), (8, 4)])
def test_eckart_young_and_orthonormality(chunks):
    m, n = 200, 60
    rowptr, col, val = _powerlaw(31, m, n, 900)
    A = _dense(m, n, rowptr, col, val)
    r = 15
    f = fastpi.factor(m, n, rowptr, col, val, r=r, k=0.03, chunk_row=chunks[0], chunk_col=chunks[1])
    sv = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - (f.U * f.S) @ f.V.T)
    assert err >= np.sqrt(np.sum(sv[r:] ** 2)) * (1 - 1e-12)
    assert f.S.size == r
    assert np.all(np.diff(f.S) <= 1e-14 * f.S[0])
    np.testing.assert_allclose(f.U.T @ f.U, np.eye(r), atol=1e-12)
    np.testing.assert_allclose(f.V.T @ f.V, np.eye(r), atol=1e-12)


def test_dependent_hub_rows_are_dropped():
    """Duplicate and all-zero border rows give a rank-deficient residual; the
    factorization is still exact at alpha = 1 (the dropped directions carry nothing)."""
    m, n = 60, 20
    rowptr, col, val = _powerlaw(41, m, n, 250)
    A = _dense(m, n, rowptr, col, val)
    hub = np.argmax((A != 0).sum(1))
    A = np.vstack([A, A[hub], A[hub], np.zeros((1, n))])
    rowptr, col, val = _csr(A)
    f = fastpi.factor(A.shape[0], n, rowptr, col, val, r=n, k=0.05, chunk_row=2, chunk_col=2)
    assert np.linalg.norm(A - (f.U * f.S) @ f.V.T) <= 1e-12 * np.linalg.norm(A)
    sv = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(f.S[:sv.size], sv, atol=1e-12 * sv[0])


def test_small_workload_residual_close_to_optimal():
    """On the 2000 x 500 workload the FastPI residual is no better than the
    unrestricted least-squares optimum (Application 1: Z = A^+ Y minimises
    |AZ - Y|_F) and within 1% of the residual of the exact rank-r truncated
    SVD (Section 4.2 reports FastPI's accuracy as near-optimal)."""
    w = workloads.make("small")
    m, n, r, k = w["m"], w["n"], w["cfg"].r, w["cfg"].k
    f = fastpi.factor(m, n, w["rowptr"], w["col"], w["val"], r=r, k=k)
    A = _dense(m, n, w["rowptr"], w["col"], w["val"])
    Z = fastpi.apply(f, w["Y"])
    res = np.linalg.norm(A @ Z - w["Y"])
    res_r = np.linalg.norm(A @ pinv.dense_solve(A, w["Y"], r) - w["Y"])
    res_full = np.linalg.norm(A @ np.linalg.lstsq(A, w["Y"], rcond=None)[0] - w["Y"])
    assert res_full <= res * (1 + 1e-12)
    assert abs(res - res_r) <= 0.01 * res_r


def test_multi_append_row_phase_is_the_running_svd_of_all_rows_of_M():
    """Reading of Eq. 2 with several appends: the oracle starts the row phase
    from the s largest block triplets.  Pin: the same result comes out of the
    incremental SVD run over ALL rows of M = [Sigma1 V1^T ; A21] from an empty
    state -- the block rows (mutually orthogonal) appended first, in descending
    sigma, a chunk at a time, then A21 -- truncating to s after every append."""
    m, n = 300, 90
    rowptr, col, val = _powerlaw(5, m, n, 1500)
    A = sp.csr_matrix((val, col, rowptr), shape=(m, n))
    r, k, chunk = 24, 0.03, 7
    R = reorder(m, n, rowptr, col, k)
    _, A11, A21, _ = fastpi.split(A, R)
    U1, sig1, V1, _ = fastpi.block_svd(A11, R, r, n)
    S, n1, m2 = sig1.size, R.n1, m - R.m1
    s = int(min(fastpi.ceil_alpha(n1, r, n), S + m2, n1))
    assert S > s and m2 > chunk          # the reading applies
    # the oracle's row phase (factor(): pre-truncation, then the appends)
    keep = fastpi._truncate(sig1, s)
    _, sig_a, V_a = fastpi.row_update_chunked(U1[:, keep], sig1[keep], V1[:, keep], A21, s, chunk)
    # from an empty state over all rows of M (the transposed problem: columns)
    Uc, sg, W = np.zeros((n1, 0)), np.zeros(0), np.zeros((0, 0))
    order = fastpi._truncate(sig1, S)
    cols = V1[:, order] * sig1[order][None, :]
    for a in range(0, S, chunk):
        Uc, sg, W = fastpi.brand_append(Uc, sg, W, cols[:, a:a + chunk], s)
    A21d = A21.toarray()
    for a in range(0, m2, chunk):
        Uc, sg, W = fastpi.brand_append(Uc, sg, W, A21d[a:a + chunk].T, s)
    np.testing.assert_allclose(sg, sig_a, rtol=1e-10, atol=1e-12 * sig_a[0])
    # the same right subspace
    np.testing.assert_allclose(np.abs(Uc.T @ V_a), np.eye(s), atol=1e-8)
    # and factor() itself (its own start of the row phase): its result is the
    # empty-state row phase above followed by the column phase (Eq. 3).  The
    # coefficients W index the rows of M: the S block rows in the order they
    # were appended, then the rows of A21, so U_row = bdiag(U1, I) W.
    f = fastpi.factor(m, n, rowptr, col, val, r, k, chunk_row=chunk, chunk_col=chunk)
    Urow = np.vstack([U1[:, order] @ W[:S], W[S:]])
    _, _, _, T = fastpi.split(A, R)
    rr = int(min(r, m, s + R.n2))
    U_e, S_e, V_e = fastpi.col_update_chunked(Urow, sg, Uc, T, rr, chunk)
    np.testing.assert_allclose(f.S, S_e, rtol=1e-10, atol=1e-12 * S_e[0])
    np.testing.assert_allclose(np.abs(U_e[R.row_pos].T @ f.U), np.eye(rr), atol=1e-7)
    np.testing.assert_allclose(np.abs(V_e[R.col_pos].T @ f.V), np.eye(rr), atol=1e-7)
