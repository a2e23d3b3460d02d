"""Autotuner: picks, on the GPU, the parameters the library reads from its
tuning table (``tuning.txt`` beside ``libfastpi.so``; format in
include/fastpi.h, ``fastpi_load_tuning``).

  python -m paper_2011_04235_gb300.autotune [--workloads medium,large] [--out PATH] [--quick]

Four searches, each timed with CUDA events on the device:

1. Core-SVD tiling (the FP32 block-Jacobi SVD of the update cores of Eqs. 2
   and 3): for core sizes n from 96 to 2 400, every tiling -- panels of 16 or
   32 columns, 1 to 8 CTAs of a cluster sharing a block pair's rows, the
   resident-block schedule on or off -- runs fastpi_core_svd_f32 on a matrix
   with the structure of a core, [[diag(sigma), P], [0, R]]; the fastest
   (kernel time, best of two) wins for that n, and its range reaches half-way
   to the next measured size.
2. Append chunk c (border rows / columns per incremental step, used when
   fastpi_factor gets chunk 0): on each workload, with the tiling table of
   step 1 loaded, the row phase (Eq. 2) is timed for every candidate c with
   the column chunk fixed, then the column phase (Eq. 3) with the best row
   chunk; the fastest c of each phase is stored for that phase's target rank
   (the mixed form; the FP64 form on the smallest workload).
3. Bucket classes of the batched Jacobi SVD of the A11 blocks (Eq. 1): the
   block stage alone (fastpi_block_svd) with the natural register-tile
   classes and with the small classes merged into larger ones (fewer
   launches, larger tiles); the fastest layout per precision.
4. The smallest FP32 product sent to the tensor cores in the mixed form
   (2 M N K flops; below it the SIMT kernel runs it): the mixed factorization
   of every workload, with the tables of steps 1-3, for thresholds from 2^24
   to 2^31 flops; the fastest sum wins.

The table is written to --out (default: the package's tuning.txt) and
printed; the measurements behind it are printed as JSON lines.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_2011_04235_gb300 import fastpi  # noqa: E402

DEV = "cuda:0"
CORE_SIZES = [96, 192, 320, 531, 756, 1000, 1280, 1600, 2000, 2400]
CHUNKS = [128, 192, 256, 320, 384, 512]


def _core_matrix(n: int, seed: int) -> torch.Tensor:
    rng = np.random.default_rng(seed)
    k = (2 * n) // 3
    K = np.zeros((n, n), dtype=np.float32)
    K[:k, :k] = np.diag(np.sort(rng.uniform(0.5, 20.0, k))[::-1])
    K[:k, k:] = rng.standard_normal((k, n - k))
    K[k:, k:] = np.triu(rng.standard_normal((n - k, n - k)))
    return torch.from_numpy(K).to(DEV)


def tune_core(sizes, quick: bool):
    rows, log = [], []
    parts_list = [1, 2, 4, 8] if quick else [1, 2, 3, 4, 6, 8]
    for n in sizes:
        K = _core_matrix(n, n)
        best = None
        for panel in (16, 32):
            for parts in parts_list:
                for res in (False, True):
                    times = []
                    try:
                        for _ in range(2):
                            _, _, _, sweeps, ms = fastpi.core_svd_f32(K, panel=panel, parts=parts, resident=res)
                            times.append(ms)
                    except fastpi.FastPIError:
                        continue           # this tiling does not fit this core
                    t = min(times)
                    log.append({"search": "core", "n": n, "panel": panel, "parts": parts, "resident": res,
                                "ms": t, "sweeps": sweeps})
                    if best is None or t < best[0]:
                        best = (t, panel, parts, res)
        if best is not None:
            rows.append((n, best[1], best[2], best[3]))
    # ranges: up to half-way to the next measured size; the last one open-ended
    table = []
    for i, (n, panel, parts, res) in enumerate(rows):
        n_max = (n + rows[i + 1][0]) // 2 if i + 1 < len(rows) else 1 << 20
        table.append(f"core {n_max} {panel} {parts} {int(res)} 1")
    return table, log


def _factor_ms(h, r, k, prec, cr, cc):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream(DEV)
    e0.record(st)
    h.factor(r, k, prec, cr, cc)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), h.info()


def tune_chunks(names, quick: bool):
    table, log = [], []
    cands = [128, 256, 512] if quick else CHUNKS
    for prec_name, prec_id, wl in (("mixed", 1, names), ("fp64", 0, names[:1])):
        by_phase = {0: [], 1: []}
        for name in wl:
            w = workloads.make(name, with_y=False)
            cfg = w["cfg"]
            h = fastpi.FastPI(w["m"], w["n"], *(torch.from_numpy(w[a]).to(DEV) for a in ("rowptr", "col", "val")),
                              device=DEV)
            fp64_cands = [128, 256, 512] if prec_id == 0 else cands
            _factor_ms(h, cfg.r, cfg.k, prec_name, 256, 256)          # warm-up
            best_row = None
            for c in fp64_cands:
                _, inf = _factor_ms(h, cfg.r, cfg.k, prec_name, c, 256)
                log.append({"search": "chunk_row", "workload": name, "precision": prec_name, "c": c,
                            "ms_row_update": inf["ms_row_update"], "s_row": inf["s_row"]})
                if best_row is None or inf["ms_row_update"] < best_row[0]:
                    best_row = (inf["ms_row_update"], c, inf["s_row"])
            best_col = None
            for c in fp64_cands:
                _, inf = _factor_ms(h, cfg.r, cfg.k, prec_name, best_row[1], c)
                log.append({"search": "chunk_col", "workload": name, "precision": prec_name, "c": c,
                            "ms_col_update": inf["ms_col_update"], "rank": inf["rank"]})
                if best_col is None or inf["ms_col_update"] < best_col[0]:
                    best_col = (inf["ms_col_update"], c, inf["rank"])
            h.close()
            by_phase[0].append((best_row[2], best_row[1]))
            by_phase[1].append((best_col[2], best_col[1]))
        for phase, pts in by_phase.items():
            pts.sort()
            for i, (k_t, c) in enumerate(pts):
                k_max = (k_t + pts[i + 1][0]) // 2 if i + 1 < len(pts) else 1 << 40
                table.append(f"chunk {prec_id} {phase} {k_max} {c}")
    return table, log


# merged layouts of the register-tile classes: (dim_max, class) lines
BUCKET_LAYOUTS = {
    1: {"natural": [], "0->1": [(256, 1)], "0,1->2": [(1024, 2)]},     # FP32: 8 / 16 / 32 / 44 values per lane
    0: {"natural": [], "0->1": [(512, 1)], "0,1->2": [(1024, 2)]},     # FP64: teams of 2 or 4 warps
}


def tune_buckets(names, base_lines, quick: bool):
    table, log = [], []
    for prec_name, prec_id in (("mixed", 1), ("fp64", 0)):
        best = None
        for label, lines in BUCKET_LAYOUTS[prec_id].items():
            tab = base_lines + [f"bucket {prec_id} {d} {c}" for d, c in lines]
            with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as fh:
                fh.write("\n".join(tab) + "\n")
                path = fh.name
            fastpi.load_tuning(path)
            os.unlink(path)
            total = 0.0
            for name in names:
                w = workloads.make(name, with_y=False)
                cfg = w["cfg"]
                h = fastpi.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
                h.block_svd(cfg.r, cfg.k, prec_name)                    # warm-up
                ts = []
                for _ in range(1 if quick else 2):
                    h.block_svd(cfg.r, cfg.k, prec_name)
                    ts.append(h.info()["ms_block_svd"])
                h.close()
                total += min(ts)
                log.append({"search": "bucket", "precision": prec_name, "layout": label, "workload": name,
                            "ms_block_svd": min(ts)})
            if best is None or total < best[0]:
                best = (total, lines)
        table += [f"bucket {prec_id} {d} {c}" for d, c in best[1]]
    return table, log


GEMM_THRESHOLDS = [1 << 24, 1 << 26, 1 << 27, 1 << 28, 1 << 29, 1 << 30, 1 << 31]


def tune_gemm(names, base_lines, quick: bool):
    log, best = [], None
    for thr in ([1 << 24, 1 << 27, 1 << 29] if quick else GEMM_THRESHOLDS):
        with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as fh:
            fh.write("\n".join(base_lines + [f"gemm {thr}"]) + "\n")
            path = fh.name
        fastpi.load_tuning(path)
        os.unlink(path)
        total = 0.0
        for name in names:
            w = workloads.make(name, with_y=False)
            cfg = w["cfg"]
            h = fastpi.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device=DEV)
            _factor_ms(h, cfg.r, cfg.k, "mixed", 0, 0)                     # warm-up
            ms = min(_factor_ms(h, cfg.r, cfg.k, "mixed", 0, 0)[0] for _ in range(1 if quick else 2))
            h.close()
            total += ms
            log.append({"search": "gemm", "tc_min_flops": thr, "workload": name, "ms_factor": ms})
        if best is None or total < best[0]:
            best = (total, thr)
    return [f"gemm {best[1]}"], log


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="medium,large")
    ap.add_argument("--out", default=fastpi.TUNING_PATH)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--skip", default="", help="comma list of searches to skip: core,chunk,bucket,gemm")
    args = ap.parse_args(argv)
    from paper_2011_04235_gb300 import build
    build.build()
    fastpi.load_tuning(None)                      # start from the built-in defaults
    names = [s for s in args.workloads.split(",") if s]
    skip = set(args.skip.split(","))
    core_lines, log = ([], []) if "core" in skip else tune_core(CORE_SIZES, args.quick)
    for r in log:
        print(json.dumps(r))
    with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as fh:
        fh.write("\n".join(core_lines) + "\n")
        path = fh.name
    fastpi.load_tuning(path)
    os.unlink(path)
    chunk_lines, log = ([], []) if "chunk" in skip else tune_chunks(names, args.quick)
    for r in log:
        print(json.dumps(r))
    bucket_lines, log = ([], []) if "bucket" in skip else tune_buckets(names, core_lines + chunk_lines, args.quick)
    for r in log:
        print(json.dumps(r))
    gemm_lines, log = ([], []) if "gemm" in skip else tune_gemm(names, core_lines + chunk_lines + bucket_lines,
                                                                 args.quick)
    for r in log:
        print(json.dumps(r))
    lines = (["# written by python -m paper_2011_04235_gb300.autotune on " + torch.cuda.get_device_name(DEV)]
             + core_lines + chunk_lines + bucket_lines + gemm_lines)
    with open(args.out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    fastpi.load_tuning(args.out)
    print("\n".join(lines))


if __name__ == "__main__":
    main()
