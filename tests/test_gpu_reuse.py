"""Factor reuse (stored factors serving applies) and the sweep over smaller
target ranks from one factorization (truncation)."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads
from gpu_common import binding, rel
from oracle import fastpi as ofp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return workloads.make("small")


def _factored(fp, w, prec, r=None):
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    h.factor(r or w["cfg"].r, w["cfg"].k, prec, 64, 64)
    return h


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_save_load_serves_identical_applies(small, prec, tmp_path):
    fp = binding()
    h = _factored(fp, small, prec)
    Y = torch.from_numpy(small["Y"]).cuda()
    Z1 = h.apply(Y)
    path = str(tmp_path / "factors.npz")
    h.save(path)
    g = fp.FastPI.load(path)
    Z2 = g.apply(Y)
    Zh = g.apply_host(small["Y"])
    torch.cuda.synchronize()
    assert torch.equal(Z1, Z2)                       # same factors, same kernels
    assert np.array_equal(Zh, Z2.cpu().numpy())
    assert np.array_equal(g.S(), h.S())
    assert torch.equal(g.U(), h.U()) and torch.equal(g.V(), h.V())
    assert g.info()["precision"] == h.info()["precision"]
    h.close()
    g.close()


def test_factor_handle_has_no_matrix(small):
    fp = binding()
    h = _factored(fp, small, "fp64")
    g = fp.FastPI.from_factors(h.S(), h.U(), h.V(), "fp64")
    Y = torch.from_numpy(small["Y"]).cuda()
    Z = g.apply(Y)
    for call in (lambda: g.residual(Y, Z), lambda: g.factor(10, 0.01), lambda: g.reorder(0.01)):
        with pytest.raises(fp.FastPIError) as e:
            call()
        assert e.value.status == 6   # FASTPI_ERR_STATE
    with pytest.raises(fp.FastPIError):
        fp.FastPI.from_factors(h.S()[::-1].copy(), h.U(), h.V(), "fp64")   # ascending S
    h.close()
    g.close()


def test_truncation_sweep(small):
    """alpha sweep from one rank-100 FP64 factorization: each truncated handle
    applies exactly V_r diag(sigma^+) U_r^T Y of the leading r triplets, and
    its residual is within 1e-3 of the oracle's FastPI run at that rank (the
    oracle shows 3e-5 for this workload)."""
    fp = binding()
    w = small
    h = _factored(fp, w, "fp64")
    S, U, V = h.S(), h.U().cpu().numpy(), h.V().cpu().numpy()
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(w["m"], w["n"]))
    Y = w["Y"]
    for r2 in (10, 25, 50, 75):
        g = fp.FastPI.from_factors(S, h.U(), h.V(), "fp64").truncate(r2)
        assert g.rank == r2
        Z = g.apply_host(Y)
        tau = max(w["m"], w["n"]) * np.finfo(np.float64).eps * S[0]
        s = S[:r2]
        inv = np.where(s > tau, 1.0 / s, 0.0)
        assert rel(Z, V[:, :r2] @ (inv[:, None] * (U[:, :r2].T @ Y))) <= 1e-12
        d = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], r2, w["cfg"].k, chunk_row=64, chunk_col=64)
        res_t = np.linalg.norm(A @ Z - Y)
        res_d = np.linalg.norm(A @ ofp.apply(d, Y) - Y)
        assert abs(res_t / res_d - 1.0) <= 1e-3, (r2, res_t, res_d)
        g.close()
    h.close()
