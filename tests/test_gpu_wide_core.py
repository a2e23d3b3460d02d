"""Cores wider than the staged-panel limit of the FP32 block Jacobi (k + c ~
2 256 columns, as in the 10^6 x 2*10^5 workload at r = 2 000): the mixed form,
whose core SVD then streams V from L2, against the FP64 form and the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads
from gpu_common import binding, rel
from oracle import fastpi as ofp

pytestmark = pytest.mark.gpu

M, N, DENSITY, R, K, CHUNK = 5000, 2400, 0.003, 2000, 0.01, 256


@pytest.fixture(scope="module")
def runs():
    fp = binding()
    rng = np.random.default_rng(11)
    rowptr, col, val = workloads.make_tiny_random(M, N, DENSITY, rng)
    Y = workloads.labels_dense(M, 40, 3, rng)
    Yd = torch.from_numpy(Y).cuda()
    out = {"Y": Y, "csr": (rowptr, col, val)}
    for prec in ("fp64", "mixed"):
        h = fp.FastPI(M, N, rowptr, col, val, device="cuda:0")
        h.factor(R, K, prec, CHUNK, CHUNK)
        Z = h.apply(Yd)
        torch.cuda.synchronize()
        out[prec] = {"S": h.S(), "Z": Z.cpu().numpy(), "res": h.residual(Yd, Z), "U": h.U(), "V": h.V(),
                     "info": h.info()}
        h.close()
    return out


def test_wide_core_sizes(runs):
    inf = runs["mixed"]["info"]
    assert inf["rank"] == R and inf["col_chunks"] >= 1   # column appends ran at r + c = 2 256


def test_wide_core_mixed_vs_fp64(runs):
    a, b = runs["mixed"]["res"], runs["fp64"]["res"]
    assert abs(a - b) / b <= 1e-3
    s_m, s_d = runs["mixed"]["S"], runs["fp64"]["S"]
    assert np.max(np.abs(s_m - s_d)) <= 5e-3 * s_d[0]
    U, V = runs["mixed"]["U"], runs["mixed"]["V"]
    eye = torch.eye(U.shape[1], dtype=torch.float64, device=U.device)
    assert (U.T @ U - eye).abs().max().item() <= 1e-3
    assert (V.T @ V - eye).abs().max().item() <= 1e-3


def test_wide_core_fp64_vs_oracle(runs):
    rowptr, col, val = runs["csr"]
    f = ofp.factor(M, N, rowptr, col, val, R, K, chunk_row=CHUNK, chunk_col=CHUNK)
    assert rel(runs["fp64"]["S"], f.S) <= 1e-10
    if not f.gaps or min(a - b for a, b in f.gaps) > 1e-8 * f.S[0]:
        assert rel(runs["fp64"]["Z"], ofp.apply(f, runs["Y"])) <= 1e-9
