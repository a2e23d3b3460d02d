"""Run one FastPI factor + apply on a named synthetic workload and print the
factorization statistics (the same call sequence as one bench step).

  python -m paper_2011_04235_gb300.run_workload medium mixed [chunk_row] [chunk_col] [--timed]

With --timed the factor + apply is run once untimed, then timed with CUDA
events while nvidia-smi samples the SM clock and throttle reasons; the JSON
line then carries "seconds" and "clocks".

The many-instance workload (independent matrices, m log-uniform in
[1 000, 50 000], n = m / 4, nnz = 10 m, r = n / 10, Y m x 200) is timed one
instance after another and through fastpi_factor_batched:

  python -m paper_2011_04235_gb300.run_workload many [count] [precision] [concurrency[,concurrency...]]

(concurrency 0: the one-after-another pass only).
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


def run_many(count: int, prec: str, concurrency: list):
    import time
    ws = workloads.make_many(count)
    dev = "cuda:0"
    streams = [torch.cuda.Stream(device=dev) for _ in ws]
    csr = [tuple(torch.from_numpy(a).to(dev) for a in (w["rowptr"], w["col"], w["val"])) for w in ws]
    Ys = [torch.from_numpy(w["Y"]).to(dev) for w in ws]
    torch.cuda.synchronize()
    res = {"instances": count, "rows": int(sum(w["m"] for w in ws)), "nnz": int(sum(w["col"].size for w in ws)),
           "precision": prec, "k": 0.01, "chunk": 256}

    # one after another, one stream
    hs = [fastpi.FastPI(w["m"], w["n"], *c, device=dev) for w, c in zip(ws, csr)]
    torch.cuda.synchronize()
    ck = _Clocks().__enter__()
    t0 = time.perf_counter()
    for w, h, Y in zip(ws, hs, Ys):
        h.factor(w["r"], 0.01, prec, 256, 256)
        h.apply(Y)
    torch.cuda.synchronize()
    res["sequential_s"] = time.perf_counter() - t0
    seq_res = [None] * count
    for i, (h, Y) in enumerate(zip(hs, Ys)):
        seq_res[i] = h.residual(Y, h.apply(Y))
        h.close()

    # batched: one stream per instance, for each requested concurrency (0: none)
    for conc in (c for c in concurrency if c > 0):
        hs = [fastpi.FastPI(w["m"], w["n"], *c, device=dev, stream=s.cuda_stream)
              for w, c, s in zip(ws, csr, streams)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fastpi.factor_batched(hs, [w["r"] for w in ws], 0.01, prec, 256, 256, concurrency=conc)
        Zs = [h.apply(Y) for h, Y in zip(hs, Ys)]
        torch.cuda.synchronize()
        bt = time.perf_counter() - t0
        gap = 0.0
        for h, Y, Z, r0 in zip(hs, Ys, Zs, seq_res):
            gap = max(gap, abs(h.residual(Y, Z) - r0) / max(r0, 1e-300))
            h.close()
        res[f"batched_s_concurrency_{conc}"] = bt
        res[f"speedup_concurrency_{conc}"] = res["sequential_s"] / bt
        res[f"max_rel_residual_diff_concurrency_{conc}"] = gap
    ck.__exit__(None, None, None)
    res["clocks"] = ck.summary()
    res["residuals_sequential"] = [float(x) for x in seq_res]
    print(json.dumps(res))


class _Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons while a run is timed."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __enter__(self):
        import subprocess
        import threading
        self.lines = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--id=0", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=lambda: [self.lines.append(x.strip()) for x in self.p.stdout], daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            self.p.wait(timeout=5)
            self.t.join(timeout=2)

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def main(argv):
    if len(argv) > 1 and argv[1] == "many":
        run_many(int(argv[2]) if len(argv) > 2 else 256, argv[3] if len(argv) > 3 else "mixed",
                 [int(c) for c in (argv[4] if len(argv) > 4 else "8").split(",")])
        return
    timed = "--timed" in argv
    argv = [a for a in argv if a != "--timed"]
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
    if "Y" in w:
        Y = torch.from_numpy(w["Y"]).to(dev)
        step = lambda: h.apply(Y)           # noqa: E731
    else:
        yr, yc, yv = (torch.from_numpy(a).to(dev) for a in w["Y_csr"])
        step = lambda: h.apply_csr(cfg.L, yr, yc, yv)   # noqa: E731
    out = {}
    if timed:
        h.factor(cfg.r, cfg.k, prec, cr, cc)
        step()
        torch.cuda.synchronize()
        with _Clocks() as ck:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h.factor(cfg.r, cfg.k, prec, cr, cc)
            Z = step()
            e1.record()
            torch.cuda.synchronize()
        out["seconds"] = e0.elapsed_time(e1) / 1000.0
        out["clocks"] = ck.summary()
    else:
        h.factor(cfg.r, cfg.k, prec, cr, cc)
        Z = step()
    torch.cuda.synchronize()
    res = h.residual(Y, Z) if "Y" in w else None
    out.update(h.info())
    out["residual"] = res
    out["workload"] = cfg.name
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main(sys.argv)
