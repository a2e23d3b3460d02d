"""Precision study of the mixed form's dense products: the library's TF32
tensor-core GEMM (one pass, or three passes on split hi + lo operands) against
BF16 tensor-core products of split operands, at the shape of the basis
rotation of the 200 000 x 50 000 workload's column update
(U <- [U, Q] Ut: 200 000 x 1 256 times 1 256 x 1 000).

  python -m paper_2011_04235_gb300.precision_study [--m 200000] [--k 1256] [--n 1000]

An FP32 operand x is split into BF16 terms x = x1 + x2 + x3 (each the BF16
rounding of what the earlier terms leave); a product with s terms per operand
keeps the cross products x_i y_j with i + j <= s + 1 (s = 1: 1 product, s = 2:
3, s = 3: 6), accumulated in FP32.  The BF16 products run through PyTorch's
BF16 matmul (a library GEMM: this is a measurement of the arithmetic, not a
library code path); the TF32 rows run the library's own tcgen05 kernel
(fastpi_gemm_f32).  Reported per variant: relative Frobenius error against the
FP64 product of the same FP32 operands, CUDA-event time (best of 3), and the
tensor-core passes.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2011_04235_gb300 import fastpi  # noqa: E402


def _split_bf16(x: torch.Tensor, terms: int):
    out, rest = [], x.clone()
    for _ in range(terms):
        t = rest.to(torch.bfloat16)
        out.append(t)
        rest = rest - t.float()
    return out


OUT_FP32 = True


def _mm_f32(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """BF16 x BF16 with FP32 accumulation and an FP32 result (torch.mm's
    out_dtype); without it the result is rounded to BF16, which this study
    then reports."""
    global OUT_FP32
    if OUT_FP32:
        try:
            return torch.mm(a, b, out_dtype=torch.float32)
        except (TypeError, RuntimeError):
            OUT_FP32 = False
    return torch.mm(a, b).float()


def _timed(fn, reps=3):
    best, out = None, None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return out, best


def run(m: int, k: int, n: int, seed: int = 0):
    dev = "cuda:0"
    g = torch.Generator(device=dev).manual_seed(seed)
    A = torch.randn(m, k, device=dev, generator=g, dtype=torch.float32) / m ** 0.5
    B = torch.randn(k, n, device=dev, generator=g, dtype=torch.float32) / k ** 0.5
    ref = (A.double() @ B.double())
    nref = torch.linalg.norm(ref).item()
    rows = []
    for name, engine, passes in (("tf32 x1 (library)", "tf32", 1), ("tf32 x3 split (library)", "tf32x3", 3)):
        C, ms = _timed(lambda: fastpi.gemm_f32(A, B, engine=engine))
        rows.append({"variant": name, "passes": passes, "ms": ms,
                     "rel_err": (torch.linalg.norm(C.double() - ref).item() / nref)})
    for terms in (1, 2, 3):
        As, Bs = _split_bf16(A, terms), _split_bf16(B, terms)
        pairs = [(i, j) for i in range(terms) for j in range(terms) if i + j <= terms - 1]

        def prod():
            acc = torch.zeros(m, n, device=dev, dtype=torch.float32)
            for i, j in pairs:
                acc += _mm_f32(As[i], Bs[j])
            return acc
        C, ms = _timed(prod)
        rows.append({"variant": f"bf16 split {terms} term(s), {len(pairs)} product(s) (library BF16 GEMM)",
                     "passes": len(pairs), "ms": ms,
                     "rel_err": torch.linalg.norm(C.double() - ref).item() / nref})
    return {"shape": [m, k, n], "bf16_products_fp32_output": OUT_FP32, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=200_000)
    ap.add_argument("--k", type=int, default=1256)
    ap.add_argument("--n", type=int, default=1000)
    a = ap.parse_args(argv)
    from paper_2011_04235_gb300 import build
    build.build()
    print(json.dumps(run(a.m, a.k, a.n)))


if __name__ == "__main__":
    main()
