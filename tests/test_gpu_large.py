"""Full-size checks of the two larger workloads.

- 200 000 x 50 000 (5M nonzeros, r = 1 000) and 10^6 x 2*10^5 (20M binary
  nonzeros, k = 0.005): the permutation of Algorithm 2 is bit-exact against
  the oracle's at full size.
- 200 000 x 50 000: the mixed-precision factorization in the bench's launch
  configuration (chunk 256) and the FP64 one, checked through properties that
  hold at any size (descending positive spectrum, orthonormal U and V, the
  apply equal to V diag(sigma^+) U^T Y on sampled columns, ||AZ - Y||_F at most
  ||Y||_F) and the mixed residual within 1e-3 of the FP64 residual.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads
from gpu_common import binding
from oracle.reorder import reorder as oracle_reorder

pytestmark = pytest.mark.gpu


def _reorder_bit_exact(name):
    fp = binding()
    w = workloads.make(name, with_y=False)
    cfg = w["cfg"]
    R = oracle_reorder(w["m"], w["n"], w["rowptr"], w["col"], cfg.k)
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    h.reorder(cfg.k)
    ro, co, m2, n2 = h.perm()
    bro, bco = h.blocks()
    h.close()
    assert np.array_equal(ro, R.row_order)
    assert np.array_equal(co, R.col_order)
    assert (m2, n2) == (w["m"] - R.m1, w["n"] - R.n1)
    assert np.array_equal(bro, R.row_off) and np.array_equal(bco, R.col_off)


def test_reorder_bit_exact_200k_x_50k():
    _reorder_bit_exact("large")


def test_reorder_bit_exact_1m_x_200k():
    _reorder_bit_exact("xlarge")


@pytest.fixture(scope="module")
def large_runs():
    fp = binding()
    w = workloads.make("large")
    cfg = w["cfg"]
    dev = "cuda:0"
    rp = torch.from_numpy(w["rowptr"]).to(dev)
    cl = torch.from_numpy(w["col"]).to(dev)
    vl = torch.from_numpy(w["val"]).to(dev)
    Y = torch.from_numpy(w["Y"]).to(dev)
    out = {"w": w, "Y": Y}
    for prec in ("mixed", "fp64"):
        h = fp.FastPI(w["m"], w["n"], rp, cl, vl, device=dev)
        h.factor(cfg.r, cfg.k, prec, 256, 256)
        Z = h.apply(Y)
        out[prec] = {"S": h.S(), "U": h.U(), "V": h.V(), "Z": Z, "res": h.residual(Y, Z), "info": h.info()}
        h.close()
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_large_factor_properties(large_runs, prec):
    r = large_runs[prec]
    S, U, V = r["S"], r["U"], r["V"]
    rank = S.size
    assert rank == large_runs["w"]["cfg"].r
    assert np.all(S > 0) and np.all(np.diff(S) <= 0)
    tol = 1e-3 if prec == "mixed" else 1e-10
    eye = torch.eye(rank, dtype=torch.float64, device=U.device)
    assert (U.T @ U - eye).abs().max().item() <= tol
    assert (V.T @ V - eye).abs().max().item() <= tol
    Y = large_runs["Y"]
    assert r["res"] <= torch.linalg.norm(Y).item()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_large_apply_sampled_columns(large_runs, prec):
    """Z = V diag(sigma^+) U^T Y (Problem 1) on 8 sampled columns of Y, with
    the threshold tau = max(m, n) eps sigma_1."""
    r = large_runs[prec]
    w = large_runs["w"]
    S = torch.from_numpy(r["S"]).to(r["U"].device)
    tau = max(w["m"], w["n"]) * np.finfo(np.float64).eps * float(r["S"][0])
    inv = torch.where(S > tau, 1.0 / S, torch.zeros_like(S))
    cols = np.random.default_rng(7).choice(large_runs["Y"].shape[1], 8, replace=False)
    y = large_runs["Y"][:, cols]
    z_ref = r["V"] @ (inv[:, None] * (r["U"].T @ y))
    z = r["Z"][:, cols]
    rel = (torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref)).item()
    # mixed: U^T Y sums m = 200 000 FP32 products in FP32 (tensor-core
    # accumulation): a typical relative error of sqrt(m) 2^-24 ~ 3e-5
    assert rel <= (1e-4 if prec == "mixed" else 1e-12), rel


def test_large_mixed_residual_matches_fp64(large_runs):
    a, b = large_runs["mixed"]["res"], large_runs["fp64"]["res"]
    assert abs(a - b) / b <= 1e-3
    s_m, s_d = large_runs["mixed"]["S"], large_runs["fp64"]["S"]
    assert np.max(np.abs(s_m[:50] - s_d[:50])) <= 1e-3 * s_d[0]
