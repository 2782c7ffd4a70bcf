#!/usr/bin/env python
"""Throughput of the GLRM alternating proximal-gradient sweep on one GB300.

A step is one full sweep (X-step over all rows, Y-step over all columns, FP64
objective) of the mixed-type table: m = 100,000 rows, n = 1,000 columns,
k = 20; 500 Huber, 300 hinge (Boolean) and 200 ordinal-hinge (7 levels)
columns; 40% of cells missing at random (|Omega| ~ 6.0e7); l1 (0.01) on X,
nonnegativity on Y; FP32.  The metric is observed entries per second per
sweep.  The inputs (CSR + CSC, ~0.96 GB) are larger than L2, so no L2 flush
is needed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU runs (torchrun, one rank per GPU) run independent replicas of the
same fit; value is the entries all ranks processed over the slowest rank's
time.  --impl reference times the FP64 CPU oracle (the correctness
reference, not a tuned program) on a row sample of the same table.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1410_0342_gb300 import workloads as W  # noqa: E402

METRIC = "observed entries/s per alternating prox-grad sweep"
UNIT = "entries/s"
WORKLOAD = "mixed-type table m={m} n=1000 k=20 (500 Huber, 300 hinge, 200 ordinal d=7), " \
           "40% missing, l1(0.01) on X, nonneg on Y, FP32"
ORACLE_SAMPLE_ROWS = 10_000
TOL_WINDOW = 10  # sweeps over which the relative objective decrease is averaged


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="glrm", choices=["glrm", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the sparse (masked-tile) path measurement on the same table")
    ap.add_argument("--time-to-tol", type=int, default=1,
                    help="1: measure the time to a 1e-4 relative objective (GPU and oracle)")
    ap.add_argument("--rows", type=int, default=100_000,
                    help="rows of the mixed table (smaller for profiling runs)")
    ap.add_argument("--path", default="auto",
                    help="kernel paths 'X,Y' (auto, chunked, fused, blocked, masked, split)")
    ap.add_argument("--form-rows", type=int, default=0,
                    help="rows of the completion form's table (0: its full 1,000,000)")
    ap.add_argument("--count", type=int, default=4096, help="instances of the batched form")
    ap.add_argument("--no-autotune", action="store_true", help="batched form: default work items")
    ap.add_argument("--form", default="sweep",
                    choices=["sweep", "batched", "autograd", "completion", "dense", "features", "pieces"],
                    help="sweep: the benchmark line; the others measure the batched, differentiable, "
                         "matrix-completion, dense (fully observed, tensor-core) and feature-table "
                         "(categorical / ordinal embeddings) forms on their own workloads")
    return ap.parse_args()


PATH_CODES = {"auto": 0, "chunked": 1, "fused": 2, "blocked": 3, "masked": 4, "split": 5}


# ---------------------------------------------------------------- helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(world: int, units_per_rank: float, steps: int, ms_max: float) -> float:
    """Whole-job units per second: every rank processes units_per_rank per step
    (replicas, weak scaling), timed by the slowest rank."""
    return world * units_per_rank * steps / (ms_max / 1000.0)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.file.read())) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4)
                          if r[5 + q].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_digest(files=None) -> str:
    """Digest of the kernel sources (all of csrc/, or the named files)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_0342_gb300", "csrc")
    for name in sorted(files if files is not None else os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it
    was taken from the current sources of that kernel (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    try:
        if d.get("source_digest") != source_digest(d.get("source_files")):
            return None
    except OSError:
        return None
    v = d.get("bytes_per_launch", {}).get(kernel)
    return float(v) if v is not None else None


def algorithmic_bytes(name: str, t: W.Table, k: int) -> float:
    """Bytes a kernel must move at minimum per launch, counted as the method's
    own work: every observed entry's index and value once (8 bytes, int32 and
    FP32), every factor row it reads once and every row it writes once.  A
    fused half-step reads the entries once and both factors, and writes the
    updated factor and step sizes; a gradient or loss pass (sparse or dense)
    reads the entries and both factors, and a gradient pass writes per-segment
    partial gradients; prox / decide kernels touch per-segment state only.
    The dense form reads every cell of its table instead of the observed
    entries; that figure is dense_cell_bytes."""
    nnz, m, n = t.nnz, t.m, t.n
    fb = 4 * k
    x = name.endswith("_x")
    nseg, other = (m, n) if x else (n, m)
    if "fused" in name:
        return nnz * 8 + (nseg + other) * fb + nseg * (fb + 4)
    if "grad" in name or "loss" in name:
        return nnz * 8 + (nseg + other) * fb + (nseg * fb if "grad" in name else 0)
    if "prox" in name or "decide" in name:
        return nseg * (2 * fb + 4)
    return 0.0


def dense_cell_bytes(name: str, t: W.Table, k: int) -> float:
    """What a dense pass actually has to read: every cell of the m x n table
    (4 bytes; a missing cell is a NaN), both factors, and for a gradient pass
    the per-row partial gradients it writes."""
    m, n = t.m, t.n
    nseg, other = (m, n) if name.endswith("_x") else (n, m)
    return 4.0 * m * n + (nseg + other) * 4 * k + (nseg * 4 * k if "grad" in name else 0)


def sweep_bytes(t: W.Table, k: int) -> float:
    """Algorithmic bytes of one whole sweep: each observed entry's index and
    value read once per half-step (16 bytes), every factor row read and
    written once per half-step, row / column pointers, step sizes and counts."""
    return 16.0 * t.nnz + 4 * 4 * (t.m + t.n) * k + 4 * (t.m + t.n) + 8 * (t.m + t.n)


def sweep_flops(t: W.Table, k: int) -> float:
    """FP32 flops of one sweep: per observed entry and half-step a dot product,
    the gradient update and the re-evaluating dot product (2k each)."""
    return 12.0 * k * t.nnz


def algorithmic_flops(name: str, t: W.Table, k: int) -> float:
    """FP32 multiply-adds x 2 the method needs per launch: per observed entry
    a dot product (2k), the gradient update (2k) and, after the prox, the
    re-evaluating dot product (2k)."""
    if "fused" in name:
        return t.nnz * 6.0 * k
    if "grad" in name:
        return t.nnz * 4.0 * k
    if "loss" in name:
        return t.nnz * 2.0 * k
    return 0.0


def table_rows(t: W.Table, rows: int) -> W.Table:
    """The first `rows` rows of a table with all their entries (a sample of
    the same workload for the CPU oracle)."""
    e = int(t.rowptr[rows])
    rowptr = t.rowptr[:rows + 1].copy()
    colidx = t.colidx[:e]
    val = t.val[:e]
    colptr, rowidx, cval = W.csc_from_csr(rows, t.n, rowptr, colidx, val)
    return W.Table(t.name + f"[:{rows}]", rows, t.n, t.k, rowptr, colidx, val, colptr, rowidx,
                   cval, t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0[:rows],
                   t.Yt0)


def oracle_rate(t: W.Table, steps: int, warmup: int = 0, nthreads: int = 0):
    """Entries/s of the oracle's sweep (with its objective) on table t, on
    nthreads host threads (0: all)."""
    import oracle
    oracle.build()
    p = oracle.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val,
                                loss_kind=t.loss_kind, loss_param=t.loss_param,
                                loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)
    X, Yt = t.X0.copy(), t.Yt0.copy()
    ax, ay = p.initial_alphas()
    if warmup:
        X, Yt, ax, ay, _, _ = p.proxgrad(X, Yt, warmup, ax, ay, nthreads=nthreads)
    t0 = time.perf_counter()
    X, Yt, ax, ay, hist, _ = p.proxgrad(X, Yt, steps, ax, ay, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return t.nnz * steps / dt, dt, oracle.num_threads(nthreads)


def cpu_model() -> str:
    """The host CPU's model name (lscpu / /proc/cpuinfo), for the baselines."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_time_to_tol(t: W.Table, rtol: float, f_ref=None, max_sweeps=3000, chunk=10,
                       nthreads=0, window=TOL_WINDOW):
    """Wall time of the oracle's sweeps from the table's initial factors up to
    the first sweep that meets the test glrm_sweep_until applies: average
    relative decrease F_{t-w} - F_t <= w rtol |F_t| over the last w = window
    sweeps (f_ref None; F_0 the initial objective) or F_t - f_ref <= rtol
    |f_ref|.  Sweeps run in chunks; the time of a chunk's sweeps past the
    stopping sweep is not counted."""
    import oracle
    oracle.build()
    p = oracle.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val,
                                loss_kind=t.loss_kind, loss_param=t.loss_param,
                                loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)
    X, Yt = t.X0.copy(), t.Yt0.copy()
    ax, ay = p.initial_alphas()
    Fs = [p.objective(X, Yt, nthreads)] if f_ref is None else [None]
    done, total = 0, 0.0
    while done < max_sweeps:
        c = min(chunk, max_sweeps - done)
        t0 = time.perf_counter()
        X, Yt, ax, ay, hist, _ = p.proxgrad(X, Yt, c, ax, ay, nthreads=nthreads)
        dt = time.perf_counter() - t0
        for q, F in enumerate(hist):
            Fs.append(F)
            s = len(Fs) - 1
            if f_ref is None:
                ok = s >= window and Fs[s - window] - F <= window * rtol * abs(F)
            else:
                ok = F - f_ref <= rtol * abs(f_ref)
            if ok:
                return {"sweeps": s, "seconds": total + dt * (q + 1) / c,
                        "objective": float(F), "threads": oracle.num_threads(nthreads)}
        done += c
        total += dt
    return {"sweeps": None, "seconds": total, "objective": float(Fs[-1]) if Fs[-1] is not None else None,
            "threads": oracle.num_threads(nthreads), "note": f"not reached in {max_sweeps} sweeps"}


def qpca_fstar(t: W.Table) -> float:
    """Closed-form optimum of quadratically regularised PCA on a fully observed
    table: ||A||^2 - sum_{i<=k} ((s_i - gamma)_+)^2 (Appendix A)."""
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    return float(np.sum(A * A) - np.sum(np.maximum(s[:t.k] - t.rx[1], 0.0) ** 2))


# ------------------------------------------------------------------- arms

def run_reference(args, world, rank):
    if rank != 0:
        return
    t = W.mixed()
    sample = table_rows(t, ORACLE_SAMPLE_ROWS)
    rate, dt, cores = oracle_rate(sample, args.steps, args.warmup)
    sample_desc = (f"first {ORACLE_SAMPLE_ROWS} rows of the table (all columns, "
                   f"{sample.nnz} observed entries), {args.steps} sweeps")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(m=t.m), "l2": "CPU run"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_desc, "cpu_model": cpu_model(),
                         "nproc": os.cpu_count()},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_roofline(name, ms, count, t, fp32_tflops, peaks, peak_src):
    """Roofline of one kernel from its per-launch CUDA-event time: HBM with the
    method's algorithmic bytes, and the FP32 pipe (sparse passes) or the BF16
    tensor pipe (dense passes) with the method's flops."""
    avg_s = ms / count / 1000.0
    abytes = algorithmic_bytes(name, t, t.k)
    achieved = abytes / avg_s / 1e9
    r = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
         "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(name),
         "algorithmic_bytes_per_launch": abytes, "avg_launch_us": avg_s * 1e6,
         "peak_source": peak_src}
    if name.startswith("dense_"):
        cb = dense_cell_bytes(name, t, t.k)
        r["dense_cell"] = {"bytes_per_launch": cb, "achieved_gbs": cb / avg_s / 1e9,
                           "frac": cb / avg_s / 1e9 / peaks["hbm_gbs"]}
        # 2 m n k flop for U (+ 2 m n k for R W in a gradient pass) against the
        # measured BF16 peak (the six split products are not counted)
        tflops = (4.0 if "grad" in name else 2.0) * t.m * t.n * t.k / avg_s / 1e12
        r["tensor"] = {"achieved_tflops": tflops, "peak_tflops": peaks["bf16_tflops"],
                       "frac": tflops / peaks["bf16_tflops"], "peak_source": peak_src}
    else:
        af = algorithmic_flops(name, t, t.k)
        r["alu"] = {"achieved_tflops": af / avg_s / 1e12, "peak_tflops": fp32_tflops,
                    "frac": af / avg_s / 1e12 / fp32_tflops,
                    "peak_source": "measured FP32 FMA probe (glrm_fma_peak)"}
    return r


def run_glrm(args, world, rank, local):
    import torch
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm as G

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t = W.mixed(m=args.rows)
    stream = torch.cuda.current_stream(dev)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP32, device=dev, stream=stream)
    if args.path != "auto":
        px, py = (PATH_CODES[v] for v in args.path.split(","))
        G.glrm_set_path(g.h, px, py)
    paths = G.glrm_get_path(g.h)
    torch.cuda.synchronize(dev)
    fp32_tflops, sms = G.glrm_fma_peak(stream=stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up
    g.sweep(args.warmup, history=False)
    torch.cuda.synchronize(dev)

    # timed region: K sweeps, CUDA events on the library's stream, per-kernel
    # events recorded by the library on the same stream
    G.glrm_timing_enable(g.h, True)
    launches0 = G.glrm_launch_count(g.h)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.sweep(args.steps, history=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    launches = G.glrm_launch_count(g.h) - launches0
    kern = G.glrm_timing_read(g.h)
    G.glrm_timing_enable(g.h, False)
    hist = g.sweep(1, history=True)
    ms_max = max_over_ranks(ms, world, dev)
    value = job_throughput(world, t.nnz, args.steps, ms_max)

    # dominant kernel and its roofline; the whole sweep against section 8(d)'s bytes and flops
    peaks, peak_src = measured_peaks()
    tname, (tms, tcount) = max(kern.items(), key=lambda kv: kv[1][0])
    roofline = kernel_roofline(tname, tms, tcount, t, fp32_tflops, peaks, peak_src)
    roofline["share_of_step"] = tms / ms
    sw_s = ms / args.steps / 1000.0
    sweep_rf = {"algorithmic_bytes": sweep_bytes(t, t.k), "algorithmic_flops": sweep_flops(t, t.k),
                "hbm_frac": sweep_bytes(t, t.k) / sw_s / 1e9 / peaks["hbm_gbs"],
                "fp32_frac": sweep_flops(t, t.k) / sw_s / 1e12 / fp32_tflops,
                "fp32_peak_tflops": fp32_tflops, "sms": sms}
    roofline["sweep"] = sweep_rf
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / ms}
               for k, v in sorted(kern.items(), key=lambda kv: -kv[1][0])}

    # the sparse sampled-residual path (masked tiles) on the same table
    sparse = None
    if rank == 0 and args.path == "auto" and not args.no_sparse:
        gs = G.GLRM.from_table(t, precision=G.GLRM_FP32, device=dev, stream=stream)
        # masked tiles in both half-steps, split over the GPU's warps by the planner
        G.glrm_set_path(gs.h, PATH_CODES["masked"], PATH_CODES["masked"])
        spaths = G.glrm_get_path(gs.h)
        gs.sweep(args.warmup, history=False)
        G.glrm_timing_enable(gs.h, True)
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        gs.sweep(args.steps, history=False)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        sms_ = s0.elapsed_time(s1)
        sk = G.glrm_timing_read(gs.h)
        G.glrm_timing_enable(gs.h, False)
        sn, (sms_k, scnt) = max(sk.items(), key=lambda kv: kv[1][0])
        srf = kernel_roofline(sn, sms_k, scnt, t, fp32_tflops, peaks, peak_src)
        srf["share_of_step"] = sms_k / sms_
        sparse = {"paths": {"x": spaths[0], "y": spaths[1]}, "value": t.nnz * args.steps / (sms_ / 1e3),
                  "unit": UNIT, "ms_per_step": sms_ / args.steps, "roofline": srf,
                  "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / sms_}
                              for k, v in sorted(sk.items(), key=lambda kv: -kv[1][0])}}
        gs.close()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
        # the CSR arrays alone: the library builds the CSC orientation on the
        # device (glrm_set_observed_csr_host), half the bytes over the host link
        hb = [pin(t.rowptr, np.int32), pin(t.colidx, np.int32), pin(t.val, np.float32)]
        hX, hY = pin(t.X0, np.float32), pin(t.Yt0, np.float32)
        h2d = sum(x.numel() * x.element_size() for x in hb + [hX, hY])
        out = np.empty(1, np.float64)
        ge = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry,
                    G.GLRM_FP32, dev, stream)

        def e2e_step():
            G.glrm_set_observed_csr_host(ge.h, t.nnz, *[x.numpy() for x in hb])
            G.glrm_set_factors_host(ge.h, hX.numpy(), hY.numpy())
            G._check(G._lib.glrm_sweep(ge.h, 1, G._ptr(out)), ge.h)

        # the host link this box gives: the same bytes copied by plain
        # asynchronous copies from the pinned buffers (context for e2e, which
        # varies with it between hosts)
        dbufs = [torch.empty_like(x, device=dev) for x in hb + [hX, hY]]
        link = []
        for rep in range(6):  # the first is a warm-up, not recorded
            torch.cuda.synchronize(dev)
            c0 = time.perf_counter()
            for d_, h_ in zip(dbufs, hb + [hX, hY]):
                d_.copy_(h_, non_blocking=True)
            torch.cuda.synchronize(dev)
            if rep:
                link.append(h2d / (time.perf_counter() - c0) / 1e9)
        del dbufs
        for _ in range(max(3, args.warmup)):  # the pool reaches its steady size
            e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, world, dev)
        e2e = {"value": world * t.nnz * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8,
               "steps": args.e2e_steps, "h2d_link_gbs": float(np.median(link)),
               "includes": "set_observed_csr_host (H2D copy of the CSR arrays + device validation + "
                           "the CSC orientation built on the device + chunk tables + the chosen path's "
                           "layout), set_factors_host, one sweep, objective D2H"}
        ge.close()

    # time to a 1e-4 relative objective: the device-side convergence test
    # (glrm_sweep_until) from the initial factors, beside the oracle's time to
    # the same test on the same table (row sample) and on the qPCA table
    ttt = None
    if rank == 0 and world == 1 and args.time_to_tol and args.rows == 100_000:
        ttt = {"rtol": 1e-4}

        def gpu_ttt(table, rtol, f_ref=float("nan"), prec=G.GLRM_FP32, max_sweeps=3000, window=TOL_WINDOW):
            gg = G.GLRM.from_table(table, precision=prec, device=dev, stream=stream)
            # capture the graph with the same history size (one sweep: any objective is
            # below the reference 1e300), then restart the fit from the initial factors
            gg.sweep_until(max_sweeps, 0.0, 1e300, window)
            gg.set_factors(torch.as_tensor(table.X0, dtype=gg.dtype, device=dev),
                           torch.as_tensor(table.Yt0, dtype=gg.dtype, device=dev))
            G.glrm_reset_steps(gg.h)
            torch.cuda.synchronize(dev)
            w0 = time.perf_counter()
            h = gg.sweep_until(max_sweeps, rtol, f_ref, window)
            wall = time.perf_counter() - w0
            gg.close()
            return {"sweeps": int(len(h)), "seconds": wall, "objective": float(h[-1]),
                    "reached": bool(len(h) < max_sweeps)}

        rel_test = f"average relative decrease over the last {TOL_WINDOW} sweeps <= 1e-4"
        ttt["mixed_full"] = {"test": rel_test,
                             "gpu": gpu_ttt(t, 1e-4)}
        sample = table_rows(t, ORACLE_SAMPLE_ROWS)
        ttt["mixed_rows_10k"] = {"test": rel_test,
                                 "gpu": gpu_ttt(sample, 1e-4),
                                 "oracle": oracle_time_to_tol(sample, 1e-4)}
        q = W.qpca_dense()
        fq = qpca_fstar(q)
        ttt["qpca_200x100"] = {"test": "(F - f*) / f* <= 1e-4, f* the closed-form optimum", "f_star": fq,
                               "gpu_fp64": gpu_ttt(q, 1e-4, fq, prec=G.GLRM_FP64),
                               "oracle": oracle_time_to_tol(q, 1e-4, f_ref=fq, chunk=50)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the whole table, as many oracle sweeps as fit in about 15 s, on all
        # host cores; then one sweep on one core
        _, dt1, _ = oracle_rate(t, 1, 0)
        nsw = max(1, min(50, int(15.0 / max(dt1, 1e-3))))
        rate, dt, cores = oracle_rate(t, nsw, 0)
        rate1, dt_1, _ = oracle_rate(t, 1, 0, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the full table ({t.nnz} entries) from the same initial factors, "
                         f"{nsw} sweeps with the objective after each, {dt:.1f} s",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"one sweep of the full table, {dt_1:.1f} s"},
               "cpu_model": cpu_model(), "nproc": os.cpu_count()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.format(m=t.m), "nnz": t.nnz, "m": t.m, "n": t.n, "k": t.k,
                       "paths": {"x": paths[0], "y": paths[1]},
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (CSR+CSC 0.96 GB; stored densely for the dense "
                             "path, 0.40 GB); no flush"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "kernels": kernels,
            "sparse": sparse,
            "time_to_tol": ttt,
            "objective_after": float(hist[-1]),
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _events(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_form(args):
    """Measurements of the other forms, one JSON line each (single GPU)."""
    import torch
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm as G
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    line = {"form": args.form, "steps": args.steps, "warmup": args.warmup, "data": "synthetic"}
    if args.form == "batched":
        t0 = time.time()
        wb = W.batch_torch(args.count, device=dev)
        gen_s = time.time() - t0
        meth = [G.GLRM_BATCH_ALS if s % 2 == 0 else G.GLRM_BATCH_PROXGRAD for s in range(wb.count)]
        B = G.Batch(wb, meth, stream=st)
        tx, ty = (np.zeros(32, np.int32), np.zeros(32, np.int32)) if args.no_autotune else B.autotune(reps=2)
        nnz = int(wb.nnz.sum())
        B.sweep(args.steps, G.GLRM_BATCH_GRAPH, history=False)  # capture + warm-up
        for _ in range(max(0, args.warmup - 1)):
            B.sweep(args.steps, G.GLRM_BATCH_GRAPH, history=False)
        ms_graph = _events(torch, st, lambda: B.sweep(args.steps, G.GLRM_BATCH_GRAPH, history=False))
        ms_stream = _events(torch, st, lambda: B.sweep(args.steps, G.GLRM_BATCH_STREAM, history=False))
        ms_inst = _events(torch, st, lambda: B.sweep(args.steps, G.GLRM_BATCH_PER_INSTANCE, history=False))
        line.update({
            "metric": METRIC, "unit": UNIT, "value": nnz * args.steps / (ms_graph / 1e3),
            "config": {"workload": f"{wb.count} instances, m~U[50,5000], n~U[20,500], k in {{4,8,16}}, even "
                                   "quadratic (ALS, FP64 Cholesky), odd Huber (prox-grad), 30% missing, "
                                   "gamma=0.1, FP32", "nnz": nnz, "generate_s": gen_s},
            "ms_per_sweep": {"graph": ms_graph / args.steps, "stream": ms_stream / args.steps,
                             "per_instance_launches": ms_inst / args.steps},
            "speedup_vs_per_instance": ms_inst / ms_graph,
            "tiles_x": tx.tolist(), "tiles_y": ty.tolist()})
    elif args.form == "autograd":
        from paper_1410_0342_gb300 import autograd as AG
        t = W.logistic_bool()
        g = G.GLRM.from_table(t, factors=False, stream=st)
        X = torch.as_tensor(t.X0, dtype=torch.float32, device=dev).requires_grad_()
        Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device=dev).requires_grad_()

        def step():
            X.grad = None
            Yt.grad = None
            AG.glrm_objective(X, Yt, g).backward()

        for _ in range(args.warmup):
            step()
        ms = _events(torch, st, lambda: [step() for _ in range(args.steps)])
        line.update({"metric": "observed entries/s per forward+backward", "unit": UNIT,
                     "value": t.nnz * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                     "config": {"workload": "logistic Boolean table m=50000 n=2000 k=32, 20% "
                                            "missing, gamma=0.1, FP32", "nnz": t.nnz}})
    elif args.form == "dense":
        t = W.mixed_dense()
        # the BF16 form on the same table: R W as one BF16 product per chunk
        gb = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry,
                    G.GLRM_BF16, dev, st)
        gb.set_dense(torch.as_tensor(t.A, dtype=torch.float32, device=dev))
        gb.set_factors(torch.as_tensor(t.X0, dtype=torch.float32, device=dev),
                       torch.as_tensor(t.Yt0, dtype=torch.float32, device=dev))
        gb.sweep(args.warmup, history=False)
        G.glrm_timing_enable(gb.h, True)
        ms_b = _events(torch, st, lambda: gb.sweep(args.steps, history=False))
        kern_b = G.glrm_timing_read(gb.h)
        G.glrm_timing_enable(gb.h, False)
        hb = gb.sweep(1)
        gb.close()
        g = G.GLRM.from_dense_table(t, stream=st)
        g.sweep(args.warmup, history=False)
        G.glrm_timing_enable(g.h, True)
        ms = _events(torch, st, lambda: g.sweep(args.steps, history=False))
        kern = G.glrm_timing_read(g.h)
        G.glrm_timing_enable(g.h, False)
        hf = g.sweep(1)
        line["bf16"] = {"ms_per_step": ms_b / args.steps, "objective_after": float(hb[-1]),
                        "fp32_objective_after": float(hf[-1]),
                        "kernels_ms": {k: v[0] / v[1] for k, v in kern_b.items()},
                        "what": "GLRM_BF16 model: gradient contraction R W as one BF16 tensor-core product "
                                "(FP32 accumulation); U, losses, objective and decisions at FP32 quality"}
        per = {k: v[0] / v[1] for k, v in kern.items()}
        nent = t.m * t.n
        # dominant kernel: the X-step gradient pass; algorithmic bytes = A once
        # (4 m n) + both factors (4 (m + n) k) + the partial gradients (4 m k)
        top = max((k for k in per if k.startswith("dense_")), key=lambda k: per[k])
        bytes_pass = 4.0 * nent + 4.0 * (t.m + t.n) * t.k + (4.0 * t.m * t.k if "grad" in top else 0.0)
        flops_pass = (4.0 if "grad" in top else 2.0) * nent * t.k
        peaks, source = measured_peaks()
        hbm = peaks.get("hbm_gbs")
        tc = peaks.get("bf16_tflops")
        ach = bytes_pass / (per[top] / 1e3) / 1e9
        line.update({
            "metric": METRIC, "unit": UNIT, "value": nent * args.steps / (ms / 1e3),
            "ms_per_step": ms / args.steps, "dtype": "fp32 (bf16 three-way split products, fp32 accumulation)",
            "config": {"workload": "mixed-type table, fully observed: m=100000 n=1000 k=20 (500 Huber, "
                                   "300 hinge, 200 ordinal d=7), l1(0.01) on X, nonneg on Y",
                       "entries": nent, "inputs_vs_L2": "A is 400 MB > L2"},
            "kernels_ms": per,
            "roofline": {"kernel": top, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm if hbm else None, "peak_source": source,
                         "tensor_tflops": flops_pass / (per[top] / 1e3) / 1e12,
                         "tensor_frac_of_bf16": (flops_pass / (per[top] / 1e3) / 1e12) / tc if tc else None}})
        g.close()
    elif args.form == "pieces":
        # the method pieces around the sweep, timed on the benchmark's mixed
        # table (and on quadratic-regularised / quadratic-loss variants of it
        # where the piece needs one)
        t = W.mixed(m=args.rows)
        g = G.GLRM.from_table(t, stream=st)
        G.glrm_set_path(g.h, 1, 1)  # the sparse observed set (the pieces read CSR / CSC)
        res = {}
        mu = torch.empty(t.n, dtype=torch.float64, device=dev)
        s2 = torch.empty_like(mu)
        G.glrm_column_stats(g.h, mu, s2)
        res["column_stats_ms"] = _events(torch, st, lambda: G.glrm_column_stats(g.h, mu, s2))
        g.set_offset(True)
        g.svd_init(power_iters=4, offset=True)
        res["svd_init_ms"] = _events(torch, st, lambda: g.svd_init(power_iters=4, offset=True))
        g.set_offset(False)
        g.close()
        tq = W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, t.val, t.colptr, t.rowidx, t.cval, t.loss_kind,
                     t.loss_param, t.loss_levels, (W.REG_QUAD, 0.1), (W.REG_QUAD, 0.1), t.X0, t.Yt0)
        g = G.GLRM.from_table(tq, stream=st)
        G.glrm_set_path(g.h, 1, 1)
        g.sweep(5, history=False)
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        val, its = g.certificate(max_iters=50, tol=0.0)
        res["certificate_50_iterations_ms"] = (time.perf_counter() - c0) * 1e3
        res["certificate_value_after_5_sweeps"] = val
        c0 = time.perf_counter()
        obj, sw, _ = g.regularization_path([1.0, 0.3, 0.1], max_sweeps=20, rtol=1e-4, window=5)
        res["regularization_path_3_weights_ms"] = (time.perf_counter() - c0) * 1e3
        res["regularization_path_sweeps"] = sw.tolist()
        g.close()
        tc = W.completion(m=100_000, k=32)
        gq = G.GLRM.from_table(tc, stream=st)
        gq.proxprox_sweep(1, 1.0, 3, history=False)
        res["proxprox_sweep_completion_100k_ms"] = _events(torch, st,
                                                           lambda: gq.proxprox_sweep(3, 1.0, 3, history=False)) / 3
        gq.als_sweep(1, history=False)
        res["als_sweep_completion_100k_ms"] = _events(torch, st, lambda: gq.als_sweep(3, history=False)) / 3
        gq.close()
        line.update({"metric": "milliseconds per call", "unit": "ms", "higher_is_better": False,
                     "config": {"workload": f"mixed table m={t.m} n=1000 k=20 (quadratic-regularised copy for "
                                            "the certificate and the path); completion m=100000 n=20000 k=32 "
                                            "(2e7 entries) for prox-prox and ALS", "nnz": t.nnz},
                     "results": res})
    elif args.form == "features":
        # a census-like table of features (Sec. 6): real, Boolean, categorical
        # (6 labels) and ordinal (7 levels) features, embedded on the device
        m = args.form_rows or 100_000
        t0 = time.time()
        t = W.features_mixed(m=m, n_real=300, n_bool=200, n_cat=150, n_ord=100, classes=6, levels=7, k=20,
                             p_obs=0.6, cyclic=False, rx=(W.REG_QUAD, 0.1), ry=(W.REG_QUAD, 0.1))
        gen_s = time.time() - t0
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        g = G.GLRM.from_feature_table(t, stream=st)
        torch.cuda.synchronize(dev)
        setup_ms = (time.perf_counter() - c0) * 1e3
        paths = G.glrm_get_path(g.h)
        g.sweep(args.warmup, history=False)
        ms = _events(torch, st, lambda: g.sweep(args.steps, history=False))
        hist = g.sweep(1)
        rng = np.random.default_rng(7)
        cnt = 1_000_000
        rows = torch.as_tensor(rng.integers(0, t.m, cnt).astype(np.int32), device=dev)
        feats = torch.as_tensor(rng.integers(0, t.nf, cnt).astype(np.int32), device=dev)
        g.decode_features(rows, feats)
        ms_dec = _events(torch, st, lambda: g.decode_features(rows, feats))
        D = int(t.widths().sum())
        ennz = int(np.sum(t.widths()[t.featidx]))
        line.update({
            "metric": "observed feature entries/s per alternating prox-grad sweep", "unit": UNIT,
            "value": t.nnz * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
            "embedded_entries_per_s": ennz * args.steps / (ms / 1e3),
            "objective_after": float(hist[-1]), "paths": paths,
            "setup_ms": setup_ms, "decode_1e6_ms": ms_dec,
            "config": {"workload": f"feature table m={t.m}: 300 Huber, 200 hinge, 150 categorical (6 labels), "
                                   "100 ordinal (7 levels) features, 60% observed, k=20, gamma=0.1, FP32",
                       "nnz": t.nnz, "embedded_columns": D, "embedded_nnz": ennz, "generate_s": gen_s}})
        g.close()
    else:
        t = W.completion(m=args.form_rows) if args.form_rows else W.completion()
        res = {}
        for name, prec in (("fp32", G.GLRM_FP32), ("bf16", G.GLRM_BF16)):
            g = G.GLRM.from_table(t, precision=prec, stream=st)
            paths = G.glrm_get_path(g.h)
            g.sweep(args.warmup, history=False)
            G.glrm_timing_enable(g.h, True)
            ms = _events(torch, st, lambda: g.sweep(args.steps, history=False))
            kern = G.glrm_timing_read(g.h)
            G.glrm_timing_enable(g.h, False)
            hist = g.sweep(1)
            res[name] = {"value": t.nnz * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                         "objective_after": float(hist[-1]), "paths": paths,
                         "kernels": {k: v[0] / v[1] for k, v in kern.items()}}
            g.close()
        line.update({"metric": METRIC, "unit": UNIT, "value": res["bf16"]["value"],
                     "dtype": "bf16 gathers, fp32 accumulation and re-evaluation",
                     "config": {"workload": f"matrix completion m={t.m} n=20000 k=64, 200 entries "
                                            "per row, quadratic loss, gamma=0.05", "nnz": t.nnz},
                     "forms": res})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.form != "sweep":
        if rank == 0:
            run_form(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_glrm(args, world, rank, local)


if __name__ == "__main__":
    main()
