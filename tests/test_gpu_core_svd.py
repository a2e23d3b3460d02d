"""The FP32 SVD of the update cores (Eqs. 2 and 3) on its own, against LAPACK.

fastpi_core_svd_f32 runs the library's core-SVD kernel (block one-sided
Jacobi) on a square matrix with a chosen tiling: panels of 16 or 32 columns,
the rows of a block pair split over a cluster of 1 to 8 CTAs (0: the default
choice), the resident-block schedule, the Gram sweep in its fast form (one
CTA barrier per inner round, fast rotations) or its IEEE form, or the
single-CTA kernel.  Every tiling must give the SVD of the
FP32 matrix on its live directions -- those ten times above the FP32 Jacobi
noise floor 2 n 2^-23 |K|_F, below which the kernel leaves columns unrotated
and the library never keeps a direction: singular values against numpy.linalg.svd
(FP64 LAPACK on the same FP32 entries) within 3e-4 sigma_1, U diag(S) V^T
(all columns) equal to the matrix within 3e-4 relative (Frobenius), U^T U and V^T V within
3e-4 of I on the live columns; and no tiling may be less accurate than the
single-CTA kernel it stands in for (singular-value error at most twice that
kernel's, plus 1e-5 sigma_1).  The bounds reflect FP32 rotations applied
thousands of times per column (each a few 2^-24 relative), not LAPACK's
backward error.

Matrices: the structure of a core, K = [[diag(sigma), P], [0, R]] (sigma
descending, P dense, R upper triangular: Eqs. 2 / 3 after CholeskyQR), and
plain Gaussian matrices; sizes from 2 to 1 100 columns (tails of odd sizes
included: blocks of 8 / 16 columns that are not full, an odd number of
clusters for the resident schedule).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from gpu_common import binding

pytestmark = pytest.mark.gpu


def _core(n, seed):
    rng = np.random.default_rng(seed)
    k = (2 * n) // 3
    c = n - k
    K = np.zeros((n, n))
    K[:k, :k] = np.diag(np.sort(rng.uniform(0.5, 20.0, k))[::-1])
    K[:k, k:] = rng.standard_normal((k, c))
    K[k:, k:] = np.triu(rng.standard_normal((c, c)))
    return K


def _gauss(n, seed):
    return np.random.default_rng(seed).standard_normal((n, n))


def _errors(K64, **tiling):
    fp = binding()
    Kf = K64.astype(np.float32)
    n = Kf.shape[0]
    ref = np.linalg.svd(Kf.astype(np.float64), compute_uv=False)
    try:
        S, U, V, sweeps, ms = fp.core_svd_f32(torch.from_numpy(Kf).cuda(), **tiling)
    except fp.FastPIError as e:
        # a tiling whose clusters cannot all be resident at once (or whose
        # panels do not fit) is refused, not run: nothing to check
        if e.status == 1 and "does not fit" in str(e):
            pytest.skip(f"tiling does not fit this core: {tiling}")
        raise
    U = U.double().cpu().numpy()
    V = V.double().cpu().numpy()
    s1 = ref[0]
    assert np.all(np.diff(S) <= 0)
    assert 1 <= sweeps <= 30
    floor = 2.0 * n * 2.0 ** -23 * np.linalg.norm(Kf)
    # well above the floor: the noise-level columns of the FP32 kernel (at
    # most ~floor) cannot interleave with these in the sorted order
    live = ref > 10.0 * floor
    e_sig = float(np.max(np.abs(S[live] - ref[live])) / s1) if live.any() else 0.0
    # all columns (those at the noise floor included: U diag(S) V^T = (K J) J^T)
    e_rec = float(np.linalg.norm((U * S) @ V.T - Kf) / np.linalg.norm(Kf))
    e_orth = max(float(np.max(np.abs(X.T @ X - np.eye(X.shape[1])))) for X in (U[:, live], V[:, live]))
    return e_sig, e_rec, e_orth


def _check(K64, **tiling):
    e_sig, e_rec, e_orth = _errors(K64, **tiling)
    assert e_sig <= 3e-4, f"sigma err {e_sig:.2e} {tiling}"
    assert e_rec <= 3e-4, f"reconstruction err {e_rec:.2e} {tiling}"
    assert e_orth <= 3e-4, f"orthonormality {e_orth:.2e} {tiling}"
    if not tiling.get("single_cta"):
        base = _errors(K64, single_cta=True)[0]
        assert e_sig <= 2.0 * base + 1e-5, f"sigma err {e_sig:.2e} vs single-CTA {base:.2e} {tiling}"
    return e_sig


TILINGS = [dict(panel=16), dict(panel=32), dict(panel=16, parts=1), dict(panel=16, parts=2),
           dict(panel=16, parts=4), dict(panel=16, parts=8), dict(panel=32, parts=3),
           dict(panel=16, resident=True), dict(panel=32, resident=True), dict(panel=16, fast=False),
           dict(panel=32, parts=5, resident=True, fast=False), dict(single_cta=True)]


@pytest.mark.parametrize("n", [2, 3, 17, 64, 203])
@pytest.mark.parametrize("ti", range(len(TILINGS)))
def test_core_svd_small_sizes_every_tiling(n, ti):
    _check(_core(n, n), **TILINGS[ti])


@pytest.mark.parametrize("n", [531, 756])
@pytest.mark.parametrize("ti", range(len(TILINGS)))
def test_core_svd_workload_sizes_every_tiling(n, ti):
    """The core sizes of the 20 000 x 5 000 workload (row phase 275 + 256,
    column phase 500 + 256)."""
    _check(_core(n, 1000 + n), **TILINGS[ti])


@pytest.mark.parametrize("n", [300, 1100])
def test_core_svd_gaussian(n):
    for ti in (dict(panel=16), dict(panel=32), dict(panel=16, resident=True)):
        _check(_gauss(n, n), **ti)


def test_core_svd_tilings_agree_bitwise_on_schedule():
    """The resident schedule keeps the pairs and the arithmetic of the default
    one, so with the same panel, parts and Gram sweep the results are equal
    bit for bit."""
    fp = binding()
    K = torch.from_numpy(_core(531, 5).astype(np.float32)).cuda()
    a = fp.core_svd_f32(K, panel=16, parts=4)
    b = fp.core_svd_f32(K, panel=16, parts=4, resident=True)
    assert np.array_equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_core_svd_rejects_bad_tilings():
    fp = binding()
    K = torch.eye(8, device="cuda")
    for kw in (dict(panel=24), dict(parts=9), dict(panel=32, single_cta=True)):
        with pytest.raises(fp.FastPIError) as e:
            fp.core_svd_f32(K, **kw)
        assert e.value.status == 1
