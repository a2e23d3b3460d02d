"""Run one FastPI factor + apply on a named synthetic workload and print the
factorization statistics (the same call sequence as one bench step).

  python -m paper_2011_04235_gb300.run_workload medium mixed [chunk_row] [chunk_col]
"""
from __future__ import annotations

import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_2011_04235_gb300 import fastpi  # noqa: E402


def main(argv):
    name = argv[1] if len(argv) > 1 else "medium"
    prec = argv[2] if len(argv) > 2 else "mixed"
    cr = int(argv[3]) if len(argv) > 3 else 256
    cc = int(argv[4]) if len(argv) > 4 else 256
    w = workloads.make(name)
    cfg = w["cfg"]
    dev = "cuda:0"
    rp = torch.from_numpy(w["rowptr"]).to(dev)
    cl = torch.from_numpy(w["col"]).to(dev)
    vl = torch.from_numpy(w["val"]).to(dev)
    h = fastpi.FastPI(w["m"], w["n"], rp, cl, vl, device=dev)
    h.factor(cfg.r, cfg.k, prec, cr, cc)
    if "Y" in w:
        Y = torch.from_numpy(w["Y"]).to(dev)
        Z = h.apply(Y)
        res = h.residual(Y, Z)
    else:
        yr, yc, yv = (torch.from_numpy(a).to(dev) for a in w["Y_csr"])
        h.apply_csr(cfg.L, yr, yc, yv)
        res = None
    torch.cuda.synchronize()
    out = h.info()
    out["residual"] = res
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main(sys.argv)
