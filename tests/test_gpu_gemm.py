"""Element-wise checks of the FP32 dense kernels behind the mixed-precision
form (SIMT FP32 and the tcgen05 TF32 tensor-core GEMM, one and three passes)
against an FP64 PyTorch CPU product of the same operands."""
from __future__ import annotations

import pytest
import torch

from gpu_common import binding

pytestmark = pytest.mark.gpu

SHAPES = [
    # M, N, K: one element, ragged tails of every tile dimension, the rotation
    # shape of the medium workload, a split-K reduction over many rows
    (1, 1, 1),
    (130, 200, 37),
    (257, 129, 65),
    (1000, 500, 756),
    (256, 300, 20000),
]
# bound on |C - C64| / (|op(A)| |op(B)|), element-wise
TOL = {"simt": 2e-5, "tf32x3": 2e-5, "tf32": 3e-3}


def _operands(M, N, K, ta, tb, seed, pad=0):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((K, M + pad) if ta else (M, K + pad), generator=g, dtype=torch.float64)
    B = torch.randn((N, K + pad) if tb else (K, N + pad), generator=g, dtype=torch.float64)
    opA = (A[:, :M].T if ta else A[:, :K])
    opB = (B[:, :K].T if tb else B[:, :N])
    return A, B, opA, opB


def _check(Cg, opA, opB, beta, C0, tol):
    ref = opA @ opB + beta * C0
    scale = opA.abs() @ opB.abs() + abs(beta) * C0.abs() + 1e-30
    err = ((Cg.double().cpu() - ref).abs() / scale).max().item()
    assert err <= tol, err
    return err


@pytest.mark.parametrize("engine", ["simt", "tf32x3", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_f32_engines(engine, M, N, K, ta, tb):
    if K >= 20000 and (ta, tb) != (True, False):
        pytest.skip("the long-K case is the Gram / U^T Y layout only")
    fp = binding()
    A, B, opA, opB = _operands(M, N, K, ta, tb, seed=M + 7 * N + 13 * K + 2 * ta + tb)
    Ad, Bd = A.float().cuda(), B.float().cuda()
    C = fp.gemm_f32(Ad, Bd, ta, tb, engine)
    torch.cuda.synchronize()
    # reference on the FP32-rounded operands, so only the kernel's own error remains
    _, _, opA32, opB32 = _operands(M, N, K, ta, tb, seed=M + 7 * N + 13 * K + 2 * ta + tb)
    opA32 = opA32.float().double()
    opB32 = opB32.float().double()
    _check(C, opA32, opB32, 0.0, torch.zeros(M, N, dtype=torch.float64), TOL[engine])


@pytest.mark.parametrize("engine", ["simt", "tf32x3"])
def test_gemm_f32_beta_and_padded_ld(engine):
    """beta != 0 reads C; leading dimensions that are not multiples of 4 and an
    output with ldc > N."""
    fp = binding()
    M, N, K = 333, 190, 101
    A, B, opA, opB = _operands(M, N, K, False, False, seed=5, pad=3)
    Ad, Bd = A.float().cuda(), B.float().cuda()
    C0 = torch.randn(M, N + 5, dtype=torch.float64, generator=torch.Generator().manual_seed(9))
    Cd = C0.float().cuda()
    fp.gemm_f32(Ad[:, :K], Bd[:, :N], False, False, engine, alpha=1.0, beta=-0.5, Cout=Cd[:, :N])
    torch.cuda.synchronize()
    _check(Cd[:, :N], opA.float().double(), opB.float().double(), -0.5, C0[:, :N].float().double(),
           TOL[engine])
    # the padding columns of C are untouched
    assert torch.equal(Cd[:, N:].cpu(), C0[:, N:].float())


def test_gemm_tf32_passes_matter_and_repeat():
    """The three-pass form is much more accurate than the one-pass form (the lo
    products are really accumulated), and the result is bitwise repeatable."""
    fp = binding()
    M, N, K = 512, 384, 1024
    A, B, opA, opB = _operands(M, N, K, False, True, seed=3)
    Ad, Bd = A.float().cuda(), B.float().cuda()
    ref = opA.float().double() @ opB.float().double()
    scale = opA.abs() @ opB.abs()
    e1 = ((fp.gemm_f32(Ad, Bd, False, True, "tf32").double().cpu() - ref).abs() / scale).max().item()
    c3a = fp.gemm_f32(Ad, Bd, False, True, "tf32x3")
    c3b = fp.gemm_f32(Ad, Bd, False, True, "tf32x3")
    e3 = ((c3a.double().cpu() - ref).abs() / scale).max().item()
    assert e3 * 20 < e1, (e1, e3)
    assert torch.equal(c3a, c3b)
