"""GPU parity of the FP64 factorization at the benched configuration, and of
every apply variant, against the FP64 oracle.

- The 20 000 x 5 000 workload (500k nonzeros, r = 500, k = 0.01) with the
  bench's chunk schedule (256 rows / columns per append): singular values to
  relative Frobenius error 1e-10 and Z = A^+ Y to 1e-9 (Z is compared when
  every truncation gap exceeds 1e-8 sigma_1 on the oracle side, as in the other
  parity tests).
- The dense apply, the host-buffer apply and the sparse-label apply (labels
  given as CSR) of the same factorization, each against oracle.fastpi.apply of
  the densified labels, element by element (relative Frobenius 1e-9).
- A handle made from saved factors (save / load) serving the three applies,
  against the oracle on the 2 000 x 500 workload.
- The mixed form at the benched configuration: every apply variant's
  |AZ - Y|_F within 1e-3 of the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads
from gpu_common import binding, rel
from oracle import fastpi as ofp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gap(f):
    if not f.gaps or f.S.size == 0:
        return np.inf
    return min((a - b) for a, b in f.gaps) / f.S[0]


def _labels_as_csr(Y):
    rows, cols = np.nonzero(Y)
    rowptr = np.zeros(Y.shape[0] + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), Y[rows, cols].astype(np.float64)


def _apply_variants(h, Y):
    """Z from the dense, host-buffer and sparse-label applies (numpy)."""
    Yd = torch.from_numpy(Y).to(DEV)
    rp, cl, vl = _labels_as_csr(Y)
    out = {"dense": h.apply(Yd).cpu().numpy(), "host": h.apply_host(Y)}
    out["csr"] = h.apply_csr(Y.shape[1], torch.from_numpy(rp).to(DEV), torch.from_numpy(cl).to(DEV),
                             torch.from_numpy(vl).to(DEV)).cpu().numpy()
    return out


@pytest.fixture(scope="module")
def medium():
    w = workloads.make("medium")
    cfg = w["cfg"]
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, chunk_row=256, chunk_col=256)
    Zo = ofp.apply(f, w["Y"])
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(w["m"], w["n"]))
    res_o = float(np.linalg.norm(A @ Zo - w["Y"]))
    return w, f, Zo, A, res_o


def test_fp64_medium_bench_schedule(medium):
    w, f, Zo, _, _ = medium
    cfg = w["cfg"]
    fp = binding()
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
    h.factor(cfg.r, cfg.k, "fp64", 256, 256)
    S = h.S()
    assert S.size == f.S.size
    assert rel(S, f.S) <= 1e-10, f"sigma rel err {rel(S, f.S):.3e}"
    assert _gap(f) > 1e-8, "truncation gap too small for a Z comparison on this workload"
    for name, Z in _apply_variants(h, w["Y"]).items():
        assert rel(Z, Zo) <= 1e-9, f"{name}: Z rel err {rel(Z, Zo):.3e}"
    h.close()


def test_mixed_medium_every_apply_residual(medium):
    w, _, _, A, res_o = medium
    cfg = w["cfg"]
    fp = binding()
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
    h.factor(cfg.r, cfg.k, "mixed", 256, 256)
    for name, Z in _apply_variants(h, w["Y"]).items():
        res = float(np.linalg.norm(A @ Z - w["Y"]))
        assert abs(res - res_o) / res_o <= 1e-3, f"{name}: residual gap {abs(res - res_o) / res_o:.3e}"
    h.close()


def test_saved_factors_serve_oracle_applies(tmp_path):
    w = workloads.make("small")
    cfg = w["cfg"]
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, chunk_row=64, chunk_col=64)
    Zo = ofp.apply(f, w["Y"])
    fp = binding()
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
    h.factor(cfg.r, cfg.k, "fp64", 64, 64)
    path = str(tmp_path / "factors.npz")
    h.save(path)
    h.close()
    g = fp.FastPI.load(path)
    if _gap(f) > 1e-8:
        for name, Z in _apply_variants(g, w["Y"]).items():
            assert rel(Z, Zo) <= 1e-9, f"{name}: Z rel err {rel(Z, Zo):.3e}"
    assert rel(g.S(), f.S) <= 1e-10
    g.close()


def test_small_sparse_labels_vs_oracle():
    """Sparse labels drawn as CSR (p positives per row): apply_csr against the
    oracle's apply of the densified labels, FP64."""
    w = workloads.make("small")
    cfg = w["cfg"]
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, chunk_row=64, chunk_col=64)
    rp, cl, vl = workloads.labels_csr(w["m"], cfg.L, cfg.p, np.random.default_rng(11))
    Yc = sp.csr_matrix((vl, cl, rp), shape=(w["m"], cfg.L)).toarray()
    Zo = ofp.apply(f, Yc)
    fp = binding()
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
    h.factor(cfg.r, cfg.k, "fp64", 64, 64)
    Zc = h.apply_csr(cfg.L, torch.from_numpy(rp).to(DEV), torch.from_numpy(cl).to(DEV),
                     torch.from_numpy(vl).to(DEV)).cpu().numpy()
    if _gap(f) > 1e-8:
        assert rel(Zc, Zo) <= 1e-9, f"Z rel err {rel(Zc, Zo):.3e}"
    h.close()
