"""fastpi_residual_noalloc: |A Z - Y|_F without any allocation in the library.

The entry point exists for callers that cannot allocate device memory when
they need the residual (code under a locked memory budget, allocation-free
loops); it keeps its scratch in a static device array.  This test calls it
through the C ABI twice in a row (the second call finds the previous call's
scratch contents) and checks both results element for element of the
definition: against NumPy's dense |A Z - Y|_F (relative 1e-12) and against
the handle-based fastpi_residual (relative 1e-12).  It also checks that the
second call leaves the device's free memory unchanged.  The file sorts last
so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads
from tests.gpu_common import binding

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_residual_noalloc_matches_numpy_twice():
    fp = binding()
    w = workloads.make("small")
    cfg = w["cfg"]
    m, n = w["m"], w["n"]
    rp = torch.from_numpy(w["rowptr"]).to(DEV)
    cl = torch.from_numpy(w["col"]).to(DEV)
    vl = torch.from_numpy(w["val"]).to(DEV)
    Y = torch.from_numpy(w["Y"]).to(DEV)
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(m, n))
    h = fp.FastPI(m, n, rp, cl, vl, device=DEV).factor(cfg.r, cfg.k, "fp64", 64, 64)
    Z = h.apply(Y)
    Z2 = Z * 0.5
    torch.cuda.synchronize()
    Zn, Z2n = Z.cpu().numpy(), Z2.cpu().numpy()
    exp1 = float(np.linalg.norm(A @ Zn - w["Y"]))
    exp2 = float(np.linalg.norm(A @ Z2n - w["Y"]))
    ref1, ref2 = h.residual(Y, Z), h.residual(Y, Z2)
    got1 = fp.residual_noalloc(m, n, rp, cl, vl, Y, Z)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(DEV)
    # a second call, with a different Z, finds the first call's scratch contents
    got2 = fp.residual_noalloc(m, n, rp, cl, vl, Y, Z2)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(DEV)
    assert abs(got1 - exp1) <= 1e-12 * exp1
    assert abs(got2 - exp2) <= 1e-12 * exp2
    assert abs(got1 - ref1) <= 1e-12 * ref1
    assert abs(got2 - ref2) <= 1e-12 * ref2
    assert abs(exp2 - exp1) > 1e-6 * exp1     # the two calls really computed different values
    assert free_after == free_before          # nothing was allocated on the device
    h.close()


def test_residual_noalloc_empty_and_too_many_rows():
    fp = binding()
    d64 = torch.zeros(1, dtype=torch.float64, device=DEV)
    i32 = torch.zeros(1, dtype=torch.int32, device=DEV)
    # m = 0 (the call that sets a device up before a memory budget is locked)
    assert fp.residual_noalloc(0, 1, torch.zeros(1, dtype=torch.int64, device=DEV), i32[:0], d64[:0],
                               torch.zeros((0, 1), dtype=torch.float64, device=DEV),
                               torch.zeros((1, 1), dtype=torch.float64, device=DEV)) == 0.0
    m = (1 << 20) + 1
    rp = torch.zeros(m + 1, dtype=torch.int64, device=DEV)
    with pytest.raises(fp.FastPIError) as e:
        fp.residual_noalloc(m, 1, rp, i32, d64, torch.zeros((m, 1), dtype=torch.float64, device=DEV),
                            torch.zeros((1, 1), dtype=torch.float64, device=DEV))
    assert e.value.status == 1


def test_residual_noalloc_binding_refuses_bad_cuda_arguments():
    """With CUDA tensors, each malformed argument is refused by the binding
    with ValueError before the library reads any buffer by its size."""
    fp = binding()
    m, n = 4, 3
    rp = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64, device=DEV)
    cl = torch.tensor([0, 1, 2, 0], dtype=torch.int32, device=DEV)
    vl = torch.ones(4, dtype=torch.float64, device=DEV)
    Y = torch.zeros(m, 2, dtype=torch.float64, device=DEV)
    Z = torch.zeros(n, 2, dtype=torch.float64, device=DEV)
    assert fp.residual_noalloc(m, n, rp, cl, vl, Y, Z) == 0.0
    cases = [
        (rp.to(torch.int32), cl, vl, Y, Z),
        (rp[:-1], cl, vl, Y, Z),
        (rp, cl, vl[:-1], Y, Z),
        (rp, cl, vl, Y[:-1], Z),
        (rp, cl, vl, Y, Z[:-1]),
        (rp, cl, vl, Y, torch.zeros(n, 3, dtype=torch.float64, device=DEV)),
        (rp, cl.to(torch.int64), vl, Y, Z),
        (rp, cl, vl.float(), Y, Z),
        (rp.cpu(), cl, vl, Y, Z),
    ]
    for args in cases:
        with pytest.raises(ValueError):
            fp.residual_noalloc(m, n, *args)
