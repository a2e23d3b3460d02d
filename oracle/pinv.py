"""Dense Moore-Penrose pseudoinverse from a full SVD (Problem 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For A = U Sigma V^T (thin SVD, FP64 LAPACK), the rank-r pseudoinverse of
Problem 1 is A^+ ~= V_r Sigma_r^+ U_r^T, exact when r >= rank(A).  Singular
values at or below tau = max(m, n) * 2^-52 * sigma_1 count as zero.
"""
from __future__ import annotations

import numpy as np

__all__ = ["dense_pinv", "dense_solve"]


def dense_pinv(A: np.ndarray, r: int | None = None) -> np.ndarray:
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    if r is not None:
        U, s, Vt = U[:, :r], s[:r], Vt[:r]
    tau = max(A.shape) * 2.0 ** -52 * (s[0] if s.size else 0.0)
    inv = np.where(s > tau, 1.0 / np.where(s > tau, s, 1.0), 0.0)
    return (Vt.T * inv[None, :]) @ U.T


def dense_solve(A: np.ndarray, Y: np.ndarray, r: int | None = None) -> np.ndarray:
    """Z* = A_r^+ Y (Application 1)."""
    return dense_pinv(A, r) @ Y
