"""Oracle for FastPI (Algorithm 1): block SVD of A11, row and column
incremental SVD updates, and the pseudoinverse apply.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain FP64 NumPy.

Notation (Section 3.3, Table 1): after the reordering of Algorithm 2,
A = [[A11, A12], [A21, A22]] with A11 m1 x n1 block diagonal, A21 m2 x n1 (hub
rows), T = [A12; A22] m x n2 (hub columns).  The target rank ratio is
alpha = r / n exactly, so every ceil(alpha * x) is evaluated in integers as
(r * x + n - 1) // n.

Stages (Algorithm 1):
  Eq. 1  per diagonal block of A11 an SVD truncated to
         s_i = min(ceil(alpha n_1i), m_1i, n_1i); U1 = bdiag(U^(i)),
         Sigma1 = bdiag(Sigma^(i)), V1 = bdiag(V^(i)), S = sum_i s_i columns.
  Eq. 2  rank-s SVD of M = [Sigma1 V1^T ; A21], s = min(ceil(alpha n1), S+m2, n1);
         U_row = [[U1 Ut_top] ; [Ut_bot]], V_row = Vt.
  Eq. 3  rank-r' SVD of N = [U_row Sigma_row , T], r' = min(r, m, s+n2);
         U = Ut, V = [[V_row Vt_top] ; [Vt_bot]].
  Problem 1 / Application 1: Z = V Sigma^+ U^T Y.

Two forms of Eqs. 2 and 3 are provided:
  * single shot, exactly as printed: form M (resp. N) densely and take its SVD;
  * chunked: the border (rows of A21, resp. columns of T) is appended ``chunk``
    at a time by the incremental SVD the paper cites for these equations
    (Brand's update): project the new columns on the current basis (two
    projection passes), orthogonalise the residual by Householder QR with column
    pivoting, dropping directions below DROP_TOL times the largest appended
    column norm, take the SVD of the small core [[Sigma, P], [0, R_R]] and
    truncate to the target rank after every chunk.  With ``chunk`` >= the border size this is one chunk and equals
    the single-shot form; with smaller chunks the result depends on the chunk
    schedule, and the library's parity is checked against this function with the
    same schedule.

Readings where the paper is silent: exact SVDs instead of frPCA (Section 3.3
allows any low-rank SVD); the pseudoinverse threshold
tau = max(m, n) * 2^-52 * sigma_1 (sigma_i <= tau is treated as zero).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from .reorder import Reordering, reorder

__all__ = ["ceil_alpha", "Factorization", "split", "block_svd", "brand_append",
           "row_update_single", "row_update_chunked", "col_update_single",
           "col_update_chunked", "factor", "pinv_threshold", "apply"]

EPS = 2.0 ** -52
# residual directions below DROP_TOL x (largest appended column norm) are dropped
DROP_TOL = 1e-7


def ceil_alpha(x, r: int, n: int):
    """ceil(alpha * x) with alpha = r / n (Table 1: r = ceil(alpha n))."""
    return (r * np.asarray(x, dtype=np.int64) + n - 1) // n


@dataclasses.dataclass
class Factorization:
    reo: Reordering
    U: np.ndarray        # m x r', ORIGINAL row order
    S: np.ndarray        # r', descending
    V: np.ndarray        # n x r', ORIGINAL column order
    S1: np.ndarray       # block-stage singular values (block order)
    s_row: int           # rank kept by the row update
    rank: int            # r'
    gaps: list           # (sigma_keep_last, sigma_drop_first) at each truncation


def split(A_csr: sp.csr_matrix, reo: Reordering):
    """Permute A by the reordering and cut it at (m1, n1) (Section 3.3)."""
    Ap = A_csr[reo.row_order][:, reo.col_order].tocsr()
    m1, n1 = reo.m1, reo.n1
    return Ap, Ap[:m1, :n1], Ap[m1:, :n1], Ap[:, n1:]


def block_svd(A11: sp.csr_matrix, reo: Reordering, r: int, n: int):
    """Eq. 1: SVD of every diagonal block of A11, truncated to s_i.

    Returns dense U1 (m1 x S), sigma1 (S), V1 (n1 x S) with the columns of
    each block contiguous, in block order, singular values descending within
    a block.  Also returns per-block s_i."""
    m1, n1 = A11.shape
    ro, co = reo.row_off, reo.col_off
    B = len(ro) - 1
    mi = np.diff(ro)
    ni = np.diff(co)
    s_i = np.minimum(np.minimum(ceil_alpha(ni, r, n), mi), ni)
    S = int(s_i.sum())
    U1 = np.zeros((m1, S))
    V1 = np.zeros((n1, S))
    sig = np.zeros(S)
    A11d = A11.tocsr()
    pos = 0
    for b in range(B):
        if s_i[b] == 0:
            continue
        blk = A11d[ro[b]:ro[b + 1], co[b]:co[b + 1]].toarray()
        u, s, vt = np.linalg.svd(blk, full_matrices=False)
        k = int(s_i[b])
        U1[ro[b]:ro[b + 1], pos:pos + k] = u[:, :k]
        V1[co[b]:co[b + 1], pos:pos + k] = vt[:k].T
        sig[pos:pos + k] = s[:k]
        pos += k
    return U1, sig, V1, s_i


def _truncate(s: np.ndarray, target: int):
    """Indices of the `target` largest values, descending (ties: lower index first)."""
    order = np.lexsort((np.arange(s.size), -s))
    return order[:target]


def brand_append(Uc: np.ndarray, sig: np.ndarray, W: np.ndarray, D: np.ndarray,
                 target: int, gaps: list | None = None, drop_tol: float = DROP_TOL):
    """Append the columns D (p x c) to the thin SVD Uc diag(sig) W^T and keep
    `target` triplets (the incremental SVD cited for Eqs. 2 and 3).

    Uc: p x k orthonormal, sig: k, W: q x k coefficient matrix.  Returns
    (Uc', sig', W') with W' of q + c rows: [[W, 0], [0, I_c]] times the right
    singular vectors of the core.

    The residual R = D - Uc Uc^T D is orthogonalised with column pivoting;
    a direction whose remaining norm is at most ``drop_tol`` times the largest
    column norm of D is dropped (it lies in span(Uc) up to rounding, e.g. a
    hub row with no entry outside the current basis).  The core is then
    (k + rank) x (k + c) and at most k + rank triplets exist."""
    p, k = Uc.shape
    c = D.shape[1]
    P = Uc.T @ D
    R = D - Uc @ P
    P2 = Uc.T @ R                      # second projection pass
    R = R - Uc @ P2
    P = P + P2
    dmax = float(np.max(np.linalg.norm(D, axis=0))) if c else 0.0
    Q, RRp, piv = scipy.linalg.qr(R, mode="economic", pivoting=True)
    d = np.abs(np.diag(RRp))
    rank = int(np.count_nonzero(d > drop_tol * dmax)) if dmax > 0 else 0
    Q = Q[:, :rank]
    RR = np.zeros((rank, c))
    RR[:, piv] = RRp[:rank]
    K = np.zeros((k + rank, k + c))
    K[:k, :k] = np.diag(sig)
    K[:k, k:] = P
    K[k:, k:] = RR
    Uk, sk, Vkt = np.linalg.svd(K, full_matrices=False)
    kk = min(target, sk.size)
    if gaps is not None and kk < sk.size:
        gaps.append((float(sk[kk - 1]) if kk > 0 else float("inf"), float(sk[kk])))
    Unew = np.hstack([Uc, Q]) @ Uk[:, :kk]
    Vk = Vkt.T[:, :kk]
    q = W.shape[0]
    Wnew = np.zeros((q + c, kk))
    Wnew[:q] = W @ Vk[:k]
    Wnew[q:] = Vk[k:]
    return Unew, sk[:kk].copy(), Wnew


def row_update_single(U1, sig1, V1, A21: sp.csr_matrix, s: int):
    """Eq. 2, single shot: rank-s SVD of [Sigma1 V1^T ; A21]."""
    S = sig1.size
    M = np.vstack([sig1[:, None] * V1.T, A21.toarray()])
    u, sv, vt = np.linalg.svd(M, full_matrices=False)
    Urow = np.vstack([U1 @ u[:S, :s], u[S:, :s]])
    return Urow, sv[:s].copy(), vt[:s].T.copy()


def row_update_chunked(U1, sig1, V1, A21: sp.csr_matrix, s: int, chunk: int, gaps=None):
    """Eq. 2 by incremental appends of `chunk` rows of A21 at a time.

    Works on the transpose M^T = [V1 Sigma1, A21^T]: the current right basis V
    plays the role of the basis being extended, and the coefficient matrix W
    gives U_row = bdiag(U1, I_m2) W."""
    S = sig1.size
    m2 = A21.shape[0]
    Vc, sig, W = V1, sig1, np.eye(S)
    A21d = A21.tocsr()
    if chunk is None or chunk <= 0:
        chunk = max(m2, 1)
    for a in range(0, m2, chunk):
        D = A21d[a:a + chunk].toarray().T
        Vc, sig, W = brand_append(Vc, sig, W, D, s, gaps)
    if sig.size > s:                   # no chunk ran: Eq. 2 still keeps rank s
        keep = _truncate(sig, s)
        Vc, sig, W = Vc[:, keep], sig[keep], W[:, keep]
    Urow = np.vstack([U1 @ W[:S], W[S:]])
    return Urow, sig, Vc


def col_update_single(Urow, sig_row, Vrow, T: sp.csr_matrix, r: int):
    """Eq. 3, single shot: rank-r SVD of [U_row Sigma_row , T]."""
    s = sig_row.size
    N = np.hstack([Urow * sig_row[None, :], T.toarray()])
    u, sv, vt = np.linalg.svd(N, full_matrices=False)
    v = vt[:r].T
    V = np.vstack([Vrow @ v[:s], v[s:]])
    return u[:, :r].copy(), sv[:r].copy(), V


def col_update_chunked(Urow, sig_row, Vrow, T: sp.csr_matrix, r: int, chunk: int, gaps=None):
    """Eq. 3 by incremental appends of `chunk` columns of T at a time."""
    s = sig_row.size
    n2 = T.shape[1]
    Tc = T.tocsc()
    Uc, sig, W = Urow, sig_row, np.eye(s)
    if chunk is None or chunk <= 0:
        chunk = max(n2, 1)
    for a in range(0, n2, chunk):
        D = Tc[:, a:a + chunk].toarray()
        Uc, sig, W = brand_append(Uc, sig, W, D, r, gaps)
    if sig.size > r:
        keep = _truncate(sig, r)
        Uc, sig, W = Uc[:, keep], sig[keep], W[:, keep]
    V = np.vstack([Vrow @ W[:s], W[s:]])
    return Uc, sig, V


def factor(m: int, n: int, rowptr, col, val, r: int, k: float,
           chunk_row: int | None = None, chunk_col: int | None = None,
           single_shot: bool = False) -> Factorization:
    """Algorithm 1 up to the solve: reorder, SVD of A11, row update, column update.

    ``chunk_row`` / ``chunk_col``: border rows / columns appended per
    incremental step (None or 0: the whole border at once).  ``single_shot``
    forms M and N densely as printed in Eqs. 2 and 3 instead."""
    if r < 1:
        raise ValueError("target rank must be >= 1")
    A = sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(m, n))
    reo = reorder(m, n, rowptr, col, k)
    _, A11, A21, T = split(A, reo)
    m1, n1 = reo.m1, reo.n1
    m2, n2 = m - m1, n - n1
    U1, sig1, V1, _ = block_svd(A11, reo, r, n)
    S = sig1.size
    s = int(min(ceil_alpha(n1, r, n), S + m2, n1))
    sig1_blocks = sig1
    if not single_shot and chunk_row and 0 < chunk_row < m2 and S > s:
        # several appends: the running SVD of Eq. 2 holds rank s between
        # appends, and the block SVD is its initial state, so it starts as the
        # s largest block triplets (descending; equal values: lower index first)
        keep = _truncate(sig1, s)
        U1, sig1, V1 = U1[:, keep], sig1[keep], V1[:, keep]
    gaps: list = []
    if single_shot:
        Urow, sig_row, Vrow = row_update_single(U1, sig1, V1, A21, s)
    else:
        Urow, sig_row, Vrow = row_update_chunked(U1, sig1, V1, A21, s, chunk_row, gaps)
    rr = int(min(r, m, s + n2))
    if single_shot:
        U, sig, V = col_update_single(Urow, sig_row, Vrow, T, rr)
    else:
        U, sig, V = col_update_chunked(Urow, sig_row, Vrow, T, rr, chunk_col, gaps)
    # back to the caller's row / column order
    U_orig = U[reo.row_pos]
    V_orig = V[reo.col_pos]
    return Factorization(reo, U_orig, sig, V_orig, sig1_blocks, s, rr, gaps)


def pinv_threshold(S: np.ndarray, m: int, n: int) -> float:
    """tau = max(m, n) * eps * sigma_1 (singular values <= tau count as zero)."""
    if S.size == 0:
        return 0.0
    return max(m, n) * EPS * float(np.max(S))


def apply(fac: Factorization, Y: np.ndarray) -> np.ndarray:
    """Problem 1 / Application 1: Z = V Sigma^+ U^T Y (n x L)."""
    m, n = fac.U.shape[0], fac.V.shape[0]
    tau = pinv_threshold(fac.S, m, n)
    inv = np.where(fac.S > tau, 1.0 / np.where(fac.S > tau, fac.S, 1.0), 0.0)
    W = fac.U.T @ Y
    return fac.V @ (inv[:, None] * W)
