#!/usr/bin/env python
"""Benchmark: FastPI factor + solve (Algorithm 1 + Problem 1) on the seeded
20000 x 5000 power-law workload (500k nonzeros, r = 500, k = 0.01, Y 20000 x 400).

One step = fastpi_factor + fastpi_apply on one GPU with the matrix and Y
already resident in HBM.  The headline `value` is the mixed-precision form
in GFLOP/s of a fixed flop model of the method's shapes (the same count for
every implementation, so FP64, mixed and the CPU oracle compare directly);
the FP64 form is timed beside it and both residuals |AZ - Y|_F are reported.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank factors its own copy of the workload
(replicas: the method does not shard); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "A†Y factor+solve seconds and GFLOP/s at rank r, mixed vs FP64 at same residual"
WORKLOAD = "medium"
TUNING = os.path.join(ROOT, "paper_2011_04235_gb300", "tuning.txt")


def table_chunk(prec_id: int, phase: int, k_target: int, default: int = 256) -> int:
    """The append chunk the library takes for chunk 0: the tuning table's
    value for this precision, phase and target rank (first matching line),
    else 256."""
    try:
        lines = open(TUNING).read().splitlines()
    except OSError:
        return default
    for ln in lines:
        f = ln.split("#")[0].split()
        if len(f) == 5 and f[0] == "chunk" and int(f[1]) == prec_id and int(f[2]) == phase and k_target <= int(f[3]):
            return int(f[4])
    return default


def oracle_chunk_schedule(w):
    """(chunk_row, chunk_col) of the mixed form's autotuned schedule, from the
    phases' target ranks (Algorithm 2 on the host, Eq. 1's s_i), for the CPU
    arm that runs without the library."""
    from oracle.reorder import reorder
    m, n, cfg = w["m"], w["n"], w["cfg"]
    R = reorder(m, n, w["rowptr"], w["col"], cfg.k)
    mb, nb = np.diff(R.row_off), np.diff(R.col_off)
    S = int(np.sum(np.minimum(np.minimum((cfg.r * nb + n - 1) // n, mb), nb)))
    s_row = min((cfg.r * R.n1 + n - 1) // n, S + (m - R.m1), R.n1)
    rank = min(cfg.r, m, s_row + (n - R.n1))
    return table_chunk(1, 0, s_row), table_chunk(1, 1, rank)


# ----------------------------------------------------------------------------- flop model
def flop_model(m, n, nnz_a21, nnz_t, m1, n1, m2, n2, row_off, col_off, r, L, chunk, chunk_col=None):
    """Flops of FastPI factor + solve from the method's shapes (Algorithm 1 with
    the chunked updates of Eqs. 2 / 3).  Dense SVD of a p x q matrix (p >= q)
    with vectors counts 4 p q^2 + 8 q^3.  One append of c columns to a rank-k
    basis of length p (q rows of coefficients, nnzc nonzeros, kk kept):
    2 nnzc k (projection) + 6 p k c (residual, second pass) + 8 p c^2
    (two Gram matrices, two triangular applies) + 12 (k + c)^3 (core SVD)
    + 2 p (k + c) kk + 2 q k kk (rotations)."""
    ceil_a = lambda x: (r * x + n - 1) // n
    chunk_row = chunk
    chunk_col = chunk if chunk_col is None else chunk_col
    mb = np.diff(row_off)
    nb = np.diff(col_off)
    sb = np.minimum(np.minimum(ceil_a(nb), mb), nb)
    p = np.maximum(mb, nb).astype(float)
    q = np.minimum(mb, nb).astype(float)
    live = sb > 0
    F = float(np.sum(4 * p[live] * q[live] ** 2 + 8 * q[live] ** 3))
    S = int(sb.sum())

    def phase(pdim, k, q0, total, target, nnz_total, chunk):
        nonlocal F
        qrows = q0
        for a in range(0, total, chunk):
            c = min(chunk, total - a)
            nnzc = nnz_total * c / max(total, 1)
            kk = min(target, k + c)
            F += (2 * nnzc * k + 6 * pdim * k * c + 8 * pdim * c * c + 12 * (k + c) ** 3
                  + 2 * pdim * (k + c) * kk + 2 * qrows * k * kk)
            k = kk
            qrows += c
        return min(k, target)

    s = int(min(ceil_a(n1), S + m2, n1))
    # with several appends the row phase starts from the s largest block
    # triplets (its coefficient matrix keeps the S block rows)
    k0 = s if (chunk_row < m2 and S > s) else S
    s = phase(n1, k0, S, m2, s, nnz_a21, chunk_row)
    F += 2.0 * float(np.sum(mb * sb)) * s            # U_row = bdiag(U1, I) W
    rr = int(min(r, m, s + n2))
    rr = phase(m, s, s, n2, rr, nnz_t, chunk_col)
    F += 2.0 * n1 * s * rr                           # V = [[V_row W_top], [W_bot]]
    F += 2.0 * m * rr * L + 2.0 * n * rr * L         # Z = V Sigma^+ (U^T Y)
    return F


def workload_flops(w, reo_row_order, reo_col_order, row_off, col_off, m1, n1, chunk, chunk_col=None):
    m, n, cfg = w["m"], w["n"], w["cfg"]
    rows = np.repeat(np.arange(m), np.diff(w["rowptr"]))
    pos_r = np.empty(m, dtype=np.int64)
    pos_r[reo_row_order] = np.arange(m)
    pos_c = np.empty(n, dtype=np.int64)
    pos_c[reo_col_order] = np.arange(n)
    nr, nc = pos_r[rows], pos_c[w["col"]]
    nnz_a21 = int(np.count_nonzero((nr >= m1) & (nc < n1)))
    nnz_t = int(np.count_nonzero(nc >= n1))
    L = w["Y"].shape[1]
    return flop_model(m, n, nnz_a21, nnz_t, m1, n1, m - m1, n - n1, np.asarray(row_off), np.asarray(col_off),
                      cfg.r, L, chunk, chunk_col)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines: list[str] = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(w, chunks, budget_s: float = 60.0):
    """Time the FP64 CPU oracle, as it stands, on the whole workload: reorder,
    block SVD, row and column updates with the same chunk schedule, and the
    apply.  Returns (GFLOP/s under the bench's flop model, seconds,
    description, BLAS threads, the oracle's singular values, its ||AZ - Y||_F)."""
    from oracle import fastpi as ofp

    cfg = w["cfg"]
    t0 = time.perf_counter()
    cr, cc = chunks
    f = ofp.factor(w["m"], w["n"], w["rowptr"], w["col"], w["val"], cfg.r, cfg.k, chunk_row=cr, chunk_col=cc)
    Zo = ofp.apply(f, w["Y"])
    secs = time.perf_counter() - t0
    import scipy.sparse as sp
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(w["m"], w["n"]))
    res_o = float(np.linalg.norm(A @ Zo - w["Y"]))
    reo = f.reo
    F = workload_flops(w, reo.row_order, reo.col_order, reo.row_off, reo.col_off, reo.m1, reo.n1, cr, cc)
    try:
        from threadpoolctl import threadpool_info
        threads = max((d.get("num_threads", 1) for d in threadpool_info()), default=1)
    except Exception:
        threads = len(os.sched_getaffinity(0))
    desc = (f"FP64 oracle (NumPy/SciPy LAPACK) on the whole {cfg.name} workload: reorder, block SVD, "
            f"row and column updates with chunks {cr} / {cc}, apply; flops by the bench's flop model")
    return F / secs / 1e9, secs, desc, threads, np.asarray(f.S), res_o


# ----------------------------------------------------------------------------- main
# DRAM bytes (read + write) per launch of the dominant kernel,
# k_jacobi_cluster<16, 0, 1>, from an ncu capture of the current kernel on
# this workload (dram__bytes_read.sum + dram__bytes_write.sum); None whenever
# the kernel's source changed after the capture, until it is captured again.
JACOBI_TRAFFIC_BYTES = (32 * 3.0310000e6 + 8 * 5.9561920e6) / 40
JACOBI_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_jacobi_cluster<16, 0, 1>: "
                         "3.03 MB per row-phase core (n = 531), 5.96 MB per column-phase core (n = 756), "
                         "weighted 32 : 8 as in one step")


def pinv_threshold_report(S, m, n):
    """Where the singular values sit against the pseudoinverse threshold
    tau = max(m, n) 2^-52 sigma_1 of Problem 1's Sigma^+ (sigma <= tau counts
    as zero): how many are at or below tau, and how many lie within 10 tau
    above it, where the zero / non-zero decision is fragile."""
    S = np.asarray(S, dtype=np.float64)
    tau = float(max(m, n) * 2.0 ** -52 * S.max()) if S.size else 0.0
    return {"tau": tau, "sigma_at_or_below_tau": int(np.count_nonzero(S <= tau)) if S.size else 0,
            "sigma_within_10x_tau": int(np.count_nonzero((S > tau) & (S <= 10.0 * tau))) if S.size else 0}


def factor_accuracy(h):
    """Deviation of the handle's U and V from orthonormal columns (max |entry|
    of U^T U - I and V^T V - I), the singular values against the pseudoinverse
    threshold, and the singular values themselves (host)."""
    import torch
    U, V = h.U(), h.V()
    eye = torch.eye(U.shape[1], dtype=torch.float64, device=U.device)
    S = np.asarray(h.S())
    out = {"UtU_minus_I_max": float((U.T @ U - eye).abs().max().item()),
           "VtV_minus_I_max": float((V.T @ V - eye).abs().max().item()),
           "pinv_threshold": pinv_threshold_report(S, h.m, h.n),
           "S": S}
    del U, V
    return out


def bench_config(w, chunks):
    """The workload description shared by both arms of the bench."""
    cfg = w["cfg"]
    return {"workload": cfg.name, "m": int(w["m"]), "n": int(w["n"]), "nnz": int(w["col"].size), "r": cfg.r,
            "k": cfg.k, "L": int(cfg.L), "chunk": {"row": int(chunks[0]), "col": int(chunks[1]),
                                                   "source": "autotuned (chunk 0: the library's tuning table)"},
            "gamma": cfg.gamma, "seed": 0,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}


def aggregate(world, flops_per_rank, sec_local, pg=None, device=None):
    """Whole-job throughput of `world` replicas: every rank did flops_per_rank
    in sec_local seconds; the job took the slowest rank's time (max over the
    process group).  Returns (GFLOP/s, seconds)."""
    sec_max = sec_local
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([sec_local], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        sec_max = float(t.item())
    return world * flops_per_rank / sec_max / 1e9, sec_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        w = workloads.make(WORKLOAD)
        chunks = oracle_chunk_schedule(w)
        vals, secs = [], []
        desc, threads = "", 1
        for _ in range(args.warmup):        # untimed, as for the GPU arm
            oracle_sample(w, chunks, budget_s=20.0)
        for _ in range(args.steps):
            g, s, desc, threads, _, _ = oracle_sample(w, chunks, budget_s=20.0)
            vals.append(g)
            secs.append(s)
        v = statistics.mean(vals)
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": bench_config(w, chunks),
               "precision": "FP64 CPU oracle (NumPy / SciPy LAPACK)",
               "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": desc},
               "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    import torch

    if not torch.cuda.is_available():
        print(json.dumps({"impl": "ours", "unavailable": "no CUDA device"}))
        return
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2011_04235_gb300 import build as _build
    if rank == 0:
        _build.build()
    if pg:
        pg.barrier()
    from paper_2011_04235_gb300 import fastpi

    w = workloads.make(WORKLOAD)
    cfg = w["cfg"]
    m, n = w["m"], w["n"]
    stream = torch.cuda.current_stream(dev)
    rp = torch.from_numpy(w["rowptr"]).to(dev)
    cl = torch.from_numpy(w["col"]).to(dev)
    vl = torch.from_numpy(w["val"]).to(dev)
    Yd = torch.from_numpy(w["Y"]).to(dev)
    Z = torch.empty((n, Yd.shape[1]), dtype=torch.float64, device=dev)
    h = fastpi.FastPI(m, n, rp, cl, vl, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > 129 MB L2

    chunks = [0, 0]   # mixed: chunk 0, the library's autotuned chunks

    def step(prec):
        cr, cc = chunks if prec == "fp64" else (0, 0)
        h.factor(cfg.r, cfg.k, prec, cr, cc)
        h.apply(Yd, out=Z)

    def timed(prec, steps, warmup, sampler=None):
        for _ in range(warmup):
            flush.fill_(1.0)
            step(prec)
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        fastpi.reset_counters()
        times = []
        for _ in range(steps):
            flush.fill_(2.0)       # L2 flush between steps, outside the timed window
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1) / 1000.0)
        cnt = fastpi.counters()
        clocks = sampler.stop() if sampler else None
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        return times, cnt, clocks

    # mixed precision: the headline
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    t_mixed, cnt_mixed, clocks = timed("mixed", args.steps, max(args.warmup, 3), sampler)
    res_mixed = h.residual(Yd, Z)
    info = h.info()
    chunks[:] = [info["chunk_row"], info["chunk_col"]]   # the FP64 form and the oracle take the same schedule
    acc = {"mixed": factor_accuracy(h), "fp64": None}
    ro, co, _, _ = h.perm()
    bro, bco = h.blocks()
    F = workload_flops(w, ro, co, bro, bco, info["m1"], info["n1"], chunks[0], chunks[1])
    # FP64 form at the same chunk schedule
    t64, _, _ = timed("fp64", max(args.fp64_steps, 1), 1)
    res64 = h.residual(Yd, Z)
    info64 = h.info()
    acc["fp64"] = factor_accuracy(h)

    sec_mixed = statistics.mean(t_mixed)
    value, sec_max = aggregate(world, F, sec_mixed, pg, dev)

    # end to end through the C ABI with host buffers (create + factor + apply_host)
    e2e = None
    if not args.no_e2e:
        e_times, c_times = [], []
        for i in range(2 + args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = fastpi.FastPI(m, n, w["rowptr"], w["col"], w["val"], device=dev)
            tc = time.perf_counter()        # fastpi_create returns after its upload, check and CSC build
            hh.factor(cfg.r, cfg.k, "mixed", 0, 0)
            Zh = hh.apply_host(w["Y"])
            t1 = time.perf_counter()
            hh.close()
            if i >= 2:
                e_times.append(t1 - t0)
                c_times.append(tc - t0)
        h2d = w["rowptr"].nbytes + w["col"].nbytes + w["val"].nbytes + w["Y"].nbytes
        d2h = Zh.nbytes
        e_value, e_sec = aggregate(world, F, statistics.mean(e_times), pg, dev)   # slowest rank's time
        e2e = {"value": e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "seconds_per_step": e_sec,
               "create_seconds_per_step": statistics.mean(c_times)}

    # roofline of the dominant kernel, the FP32 block-Jacobi SVD of the update
    # cores (ALU-bound): algorithmic flops = 12 n^3 per n x n core (the dense
    # SVD model 4 p q^2 + 8 q^3 at p = q = n), over the kernel's own CUDA-event
    # time on the launching stream.  The rotation work it did (sweeps x
    # n(n-1)/2 pair visits x 18 n) is reported beside it.
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12        # TFLOP/s: SMs x FP32 lanes x 2 flop x clock
    core = cnt_mixed["core32"]
    jl = max(core["launches"], 1)
    avg_ms = core["ms"] / jl
    achieved = core["flops"] / (core["ms"] / 1000.0) / 1e12 if core["ms"] > 0 else 0.0
    achieved_rot = core["flops_rot"] / (core["ms"] / 1000.0) / 1e12 if core["ms"] > 0 else 0.0
    step_s = max(sum(t_mixed), 1e-9)
    roofline = {"kernel": "k_jacobi_cluster (block one-sided Jacobi SVD of the update cores, a block pair's rows "
                          "split over a thread-block cluster, FP32)", "bound": "alu",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": JACOBI_TRAFFIC_BYTES, "traffic_source": JACOBI_TRAFFIC_SOURCE,
                "work_per_launch": "12 n^3 flops for an n x n core (n = k + c)",
                "flops_per_step": core["flops"] / args.steps,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz of MEASURED_PEAKS.json "
                               "(the file has no FP32 figure)",
                "rotation_flops_achieved": achieved_rot,
                "time_share": core["ms"] / 1000.0 / step_s,
                "avg_launch_ms": avg_ms, "launches_per_step": core["launches"] / args.steps}
    svd_kernels = {kind: {"launches_per_step": cnt_mixed[kind]["launches"] / args.steps,
                          "ms_per_step": cnt_mixed[kind]["ms"] / args.steps,
                          "share": cnt_mixed[kind]["ms"] / 1000.0 / step_s}
                   for kind in ("blocks", "core32")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the host-core baseline: N = 1 only
        g, s, desc, threads, S_o, res_o = oracle_sample(w, chunks, budget_s=20.0)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": desc, "seconds": s}
        for form, res in (("mixed", res_mixed), ("fp64", res64)):
            S_g = acc[form].pop("S")
            acc[form]["sigma_rel_err_vs_oracle"] = (float(np.linalg.norm(S_g - S_o) / np.linalg.norm(S_o))
                                                    if S_g.size == S_o.size else None)
            acc[form]["residual_gap_vs_oracle"] = abs(res - res_o) / res_o
    for form in acc:
        acc[form].pop("S", None)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1000 * sec_mixed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(w, chunks),
            "precision": "mixed: FP32 storage, TF32 tensor-core products (split hi/lo, 3 passes) with FP32 "
                         "accumulation, float-float residual Gram and FP64 pivoted Cholesky, FP32 block-Jacobi "
                         "core SVD (cluster form, Newton-Schulz re-orthonormalised rotations)",
            "mixed": {"seconds": sec_mixed, "gflops": F / sec_mixed / 1e9, "residual": res_mixed,
                      "stage_ms": {k: info[k] for k in info if k.startswith("ms_")}},
            "fp64": {"seconds": statistics.mean(t64), "gflops": F / statistics.mean(t64) / 1e9,
                     "residual": res64, "stage_ms": {k: info64[k] for k in info64 if k.startswith("ms_")}},
            "residual_gap_rel": abs(res_mixed - res64) / res64,
            "speedup_mixed_vs_fp64": statistics.mean(t64) / sec_mixed,
            "flops_per_step": F,
            "reorder": {k: info[k] for k in ("m1", "n1", "m2", "n2", "num_blocks", "iterations", "S", "s_row",
                                               "rank", "row_chunks", "col_chunks", "jacobi_sweeps_max")},
            "accuracy": acc,
            "roofline": roofline,
            "svd_kernels": svd_kernels,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(cnt_mixed["kernel_launches"]),
            "clocks": clocks,
        }
        print(json.dumps(out))
    h.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
