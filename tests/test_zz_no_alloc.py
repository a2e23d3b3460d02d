"""fastpi_residual_noalloc against fastpi_residual.

The no-allocation entry point exists for callers that cannot allocate device
memory when they need the residual (under a locked memory budget, in
allocation-free loops); it keeps its scratch in a static
device array.  This test calls it through the C ABI twice in a row (the second
call finds the previous call's scratch contents) and checks both results
against the handle-based fastpi_residual, with the relative tolerance the
residual parity tests use (1e-12).  The file sorts last so that a run stopping
at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_common import binding

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_residual_noalloc_matches_residual_twice():
    fp = binding()
    w = workloads.make("small")
    cfg = w["cfg"]
    m, n = w["m"], w["n"]
    rp = torch.from_numpy(w["rowptr"]).to(DEV)
    cl = torch.from_numpy(w["col"]).to(DEV)
    vl = torch.from_numpy(w["val"]).to(DEV)
    Y = torch.from_numpy(w["Y"]).to(DEV)
    h = fp.FastPI(m, n, rp, cl, vl, device=DEV).factor(cfg.r, cfg.k, "fp64", 64, 64)
    Z = h.apply(Y)
    ref = h.residual(Y, Z)
    got1 = fp.residual_noalloc(m, n, rp, cl, vl, Y, Z)
    # a second call with a different Z reuses the same scratch
    Z2 = Z * 0.5
    ref2 = h.residual(Y, Z2)
    got2 = fp.residual_noalloc(m, n, rp, cl, vl, Y, Z2)
    assert abs(got1 - ref) <= 1e-12 * ref
    assert abs(got2 - ref2) <= 1e-12 * ref2
    assert abs(ref2 - ref) > 1e-6 * ref     # the two calls really computed different values
    h.close()


def test_residual_noalloc_rejects_too_many_rows():
    fp = binding()
    m = (1 << 20) + 1
    dummy = torch.zeros(1, dtype=torch.float64, device=DEV)
    rp = torch.zeros(m + 1, dtype=torch.int64, device=DEV)
    with pytest.raises(fp.FastPIError) as e:
        fp.residual_noalloc(m, 1, rp, torch.zeros(1, dtype=torch.int32, device=DEV), dummy,
                            torch.zeros((1, 1), dtype=torch.float64, device=DEV),
                            torch.zeros((1, 1), dtype=torch.float64, device=DEV))
    assert e.value.status == 1
