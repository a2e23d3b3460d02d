"""Accuracy diagnostics: P@k (Application 1's measure) pinned on a hand-made
example, and on the GPU the reconstruction error of an FP64 factorization
against the oracle's dense computation, plus the held-out protocol."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads


def test_precision_at_k_hand_example():
    from paper_2011_04235_gb300.diagnostics import precision_at_k
    scores = np.array([[0.9, 0.1, 0.5], [0.2, 0.8, 0.8]])
    labels = np.array([[1, 0, 0], [0, 0, 1]])
    # row 0: top-1 label 0 (true); row 1: 0.8 tie -> lower index 1 (false)
    assert precision_at_k(scores, labels, 1) == pytest.approx(0.5)
    # top-2: row 0 {0, 2} one hit; row 1 {1, 2} one hit
    assert precision_at_k(scores, labels, 2) == pytest.approx(0.5)
    assert precision_at_k(scores, labels, 3) == pytest.approx(1.0 / 3.0)


@pytest.mark.gpu
def test_reconstruction_error_matches_oracle():
    from gpu_common import binding
    from oracle import fastpi as ofp
    fp = binding()
    from paper_2011_04235_gb300.diagnostics import reconstruction_error
    w = workloads.make("small")
    cfg = w["cfg"]
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    h.factor(cfg.r, cfg.k, "fp64", 64, 64)
    e_gpu = reconstruction_error(h)
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, chunk_row=64, chunk_col=64)
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(w["m"], w["n"])).toarray()
    e_ref = np.linalg.norm(A - (f.U * f.S) @ f.V.T) / np.linalg.norm(A)
    assert abs(e_gpu - e_ref) <= 1e-8 * max(e_ref, 1e-300)
    # the mixed form's factors: FP32 U, V, their reconstruction error within
    # 1e-3 of the oracle's
    g = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    g.factor(cfg.r, cfg.k, "mixed", 64, 64)
    assert abs(reconstruction_error(g) - e_ref) <= 1e-3 * e_ref
    g.close()
    h.close()


@pytest.mark.gpu
def test_spmm_matches_scipy():
    from gpu_common import binding
    fp = binding()
    w = workloads.make("small")
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    X = np.random.default_rng(3).standard_normal((w["n"], 300))
    got = h.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(w["m"], w["n"]))
    ref = A @ X
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    h.close()


@pytest.mark.gpu
def test_heldout_protocol_mixed_vs_fp64():
    from gpu_common import binding
    binding()
    from paper_2011_04235_gb300.diagnostics import heldout_eval
    w = workloads.make("small")
    cfg = w["cfg"]
    res = {p: heldout_eval(w["m"], w["n"], w["rowptr"], w["col"], w["val"], w["Y"], cfg.r, cfg.k, p, chunk=64)
           for p in ("fp64", "mixed")}
    for p in res:
        for k in (1, 3, 5):
            assert 0.0 <= res[p][f"P@{k}"] <= 1.0
        assert 0.0 < res[p]["reconstruction_error"] < 1.0
    for k in (1, 3, 5):
        assert abs(res["mixed"][f"P@{k}"] - res["fp64"][f"P@{k}"]) <= 0.01
