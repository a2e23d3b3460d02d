"""fastpi_factor_batched: many independent factorizations (the many-instance
workload: m log-uniform, n = m / 4, nnz = 10 m, r = n / 10), with the A11
block SVDs of every instance in one batched launch.  Each batched result must
equal the result of factoring that instance alone (the same algorithm; only
the Jacobi kernel's register tile, chosen from the largest block of the whole
batch, may change the rounding order), and the FP64 results must match the
oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads
from gpu_common import binding, rel
from oracle import fastpi as ofp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def instances():
    # the first instances of the many-instance workload, with m capped so that
    # the single-instance references stay quick
    return workloads.make_many(count=10, lo=1000, hi=8000)


def _handles(fp, insts, streams):
    hs = []
    for w, s in zip(insts, streams):
        hs.append(fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0",
                            stream=s.cuda_stream))
    return hs


def _factor_alone(fp, w, prec, k):
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    h.factor(w["r"], k, prec, 64, 64)
    Y = torch.from_numpy(w["Y"]).cuda()
    Z = h.apply(Y)
    torch.cuda.synchronize()
    out = (h.S(), Z.cpu().numpy(), h.residual(Y, Z))
    h.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_equals_alone(instances, prec):
    fp = binding()
    k = 0.01
    streams = [torch.cuda.Stream() for _ in instances]
    hs = _handles(fp, instances, streams)
    torch.cuda.synchronize()
    st = fp.factor_batched(hs, [w["r"] for w in instances], k, prec, 64, 64, concurrency=4)
    assert st == [0] * len(instances)
    torch.cuda.synchronize()
    for w, h in zip(instances, hs):
        Y = torch.from_numpy(w["Y"]).cuda()
        torch.cuda.synchronize()
        Z = h.apply(Y)
        torch.cuda.synchronize()
        S_b, Z_b, res_b = h.S(), Z.cpu().numpy(), h.residual(Y, Z)
        S_a, Z_a, res_a = _factor_alone(fp, w, prec, k)
        assert S_b.size == S_a.size
        if prec == "fp64":
            assert rel(S_b, S_a) <= 1e-12
            assert rel(Z_b, Z_a) <= 1e-9
            assert abs(res_b - res_a) <= 1e-12 * res_a
        else:
            assert abs(res_b - res_a) <= 1e-5 * res_a
            assert np.max(np.abs(S_b - S_a)) <= 1e-4 * S_a[0]
        h.close()


def test_batched_fp64_matches_oracle(instances):
    """Two members of an FP64 batch against the oracle (Sigma 1e-10, Z 1e-9)."""
    fp = binding()
    k = 0.01
    sub = instances[:2]
    streams = [torch.cuda.Stream() for _ in sub]
    hs = _handles(fp, sub, streams)
    torch.cuda.synchronize()
    fp.factor_batched(hs, [w["r"] for w in sub], k, "fp64", 64, 64, concurrency=2)
    torch.cuda.synchronize()
    for w, h in zip(sub, hs):
        f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], w["r"], k, chunk_row=64, chunk_col=64)
        S = h.S()
        assert rel(S, f.S) <= 1e-10
        if not f.gaps or min(a - b for a, b in f.gaps) > 1e-8 * f.S[0]:
            Y = torch.from_numpy(w["Y"]).cuda()
            Z = h.apply(Y)
            torch.cuda.synchronize()
            assert rel(Z.cpu().numpy(), ofp.apply(f, w["Y"])) <= 1e-9
        h.close()


def test_batched_argument_errors():
    fp = binding()
    w = workloads.make_many(count=1, lo=1000, hi=1000)[0]
    h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
    with pytest.raises(fp.FastPIError):
        fp.factor_batched([h, h], [w["r"], w["r"]], 0.01, "mixed")      # a handle twice
    with pytest.raises(fp.FastPIError):
        fp.factor_batched([h], [0], 0.01, "mixed")                      # rank 0
    with pytest.raises(fp.FastPIError):
        fp.factor_batched([h], [w["r"]], 1.5, "mixed")                  # k outside (0, 1)
    h.close()
