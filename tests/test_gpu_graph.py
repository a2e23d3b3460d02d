"""The dense apply (Problem 1, fastpi_apply) is capture-safe: no host synchronisation and only
stream-ordered allocations, so a caller can record it into a CUDA graph once
and replay it for every new Y of the same shape (the serving path of
Application 1)."""
from __future__ import annotations

import pytest
import torch

import workloads
from gpu_common import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_apply_replays_from_a_cuda_graph(prec):
    fp = binding()
    w = workloads.make("small")
    cfg = w["cfg"]
    f = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    f.factor(cfg.r, cfg.k, prec, 64, 64)
    s = torch.cuda.Stream()
    h = fp.FastPI.from_factors(f.S(), f.U(), f.V(), prec, stream=s.cuda_stream)
    Y = torch.from_numpy(w["Y"]).cuda()
    Z_eager = f.apply(Y)
    torch.cuda.synchronize()
    Ys = torch.zeros_like(Y)
    Zs = torch.empty_like(Z_eager)
    with torch.cuda.stream(s):
        h.apply(Ys, out=Zs)          # warm-up outside the capture (one-time setup)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.apply(Ys, out=Zs)
    for scale in (1.0, 2.0, -0.5):
        Ys.copy_(Y * scale)
        g.replay()
        torch.cuda.synchronize()
        assert torch.allclose(Zs, Z_eager * scale, rtol=1e-12 if prec == "fp64" else 1e-5,
                              atol=1e-12 * Z_eager.abs().max().item())
    f.close()
    h.close()
