"""Accuracy diagnostics of a factorization on synthetic data (evaluation
tooling around the library, not part of the method's hot path).

- ``reconstruction_error``: ||A - U diag(S) V^T||_F / ||A||_F, the accuracy
  measure of the low-rank approximation behind the pseudoinverse (Section 4),
  computed by the library (fastpi_recon_error).
- ``precision_at_k``: P@k of multi-label scores, the measure of the
  multi-label linear regression application (Application 1, Section 4): the
  fraction of the k highest-scored labels of a row that are true labels,
  averaged over rows.
- ``heldout_eval``: the application's protocol on a seeded 90% / 10% split of
  the rows: Z = A_train^+ Y_train and the scores A_test Z (fastpi_spmm) from
  the library, P@k on the held-out rows.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fastpi


def reconstruction_error(h: "fastpi.FastPI") -> float:
    """||A - U S V^T||_F / ||A||_F from the handle's factors (computed by the
    library, fastpi_recon_error)."""
    return h.recon_error()


def precision_at_k(scores: np.ndarray, labels: np.ndarray, k: int) -> float:
    """Mean over rows of |top-k(scores_row) intersect true(labels_row)| / k;
    ties among scores are broken towards the lower label index."""
    scores = np.asarray(scores, dtype=np.float64)
    labels = np.asarray(labels) != 0
    n_rows, L = scores.shape
    if n_rows == 0:
        return 0.0
    k = min(k, L)
    order = np.lexsort((np.broadcast_to(np.arange(L), scores.shape), -scores), axis=1)[:, :k]
    hits = np.take_along_axis(labels, order, axis=1).sum(axis=1)
    return float(hits.mean() / k)


def _rows(rowptr, col, val, rows):
    rp = np.asarray(rowptr)
    counts = rp[rows + 1] - rp[rows]
    new_rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(counts, out=new_rp[1:])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows]) if rows.size else np.zeros(0, np.int64)
    return new_rp, np.asarray(col)[idx], np.asarray(val)[idx]


def heldout_eval(m: int, n: int, rowptr, col, val, Y: np.ndarray, r: int, k_hub: float, precision="mixed",
                 test_frac: float = 0.1, seed: int = 0, ks=(1, 3, 5), chunk: int = 256, device="cuda:0") -> dict:
    """Application 1 on a seeded row split: factor A_train with target rank r,
    Z = V S^+ U^T Y_train (fastpi_apply), scores = A_test Z, P@k on the held-out
    rows; also the reconstruction error of the training factorization."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(m)
    n_test = int(round(test_frac * m))
    test, train = np.sort(perm[:n_test]), np.sort(perm[n_test:])
    tr = _rows(rowptr, col, val, train)
    te = _rows(rowptr, col, val, test)
    h = fastpi.FastPI(train.size, n, *tr, device=device)
    h.factor(r, k_hub, precision, chunk, chunk)
    Z = h.apply(torch.from_numpy(np.ascontiguousarray(Y[train])).to(device))
    g = fastpi.FastPI(test.size, n, *te, device=device)   # held-out rows: scores A_test Z (fastpi_spmm)
    scores = g.spmm(Z).cpu().numpy()
    g.close()
    out = {f"P@{k}": precision_at_k(scores, Y[test], k) for k in ks}
    out["reconstruction_error"] = reconstruction_error(h)
    out["rank"] = h.rank
    out["train_rows"], out["test_rows"] = int(train.size), int(test.size)
    h.close()
    return out
