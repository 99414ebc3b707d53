#!/usr/bin/env python
"""Benchmark: simultaneous Krylov solves on the 3D convection-diffusion workload.

Workload (stand-in for Examples 2-3 of the paper): 7-point convection-diffusion
on a 128^3 grid (n = 2,097,152, 14,581,760 stored entries), cell Peclet number
0.8 along each axis, complex shift 0.05i, s = 8 Gaussian right-hand sides
(seed 0), X_0 = 0, FP64, relative residual 1e-8, at most 3000 iterations.

First every one of the ten methods (Bl-BiCG, Bl-BiCG-rQ, Gl-BiCG, eGl-BiCG,
Bl-BiCGStab, Bl-BiCGStab-rQ, Gl-BiCGStab, Bl-QMR, Gl-QMR, eGl-QMR) solves the
system: its time to 1e-8 (CUDA events, median of three solves after an untimed
3-iteration solve that allocates its workspace), iterations and status go to
per_method.  The methods that reached the tolerance form the headline set; one
step runs the first --window (50) iterations from X0 = 0 of each of them, and the
metric is RHS*iterations per second over the timed steps (no per-launch
instrumentation in that region).  A
separate profiled step gives the per-kernel-class rates for the roofline, whose
FP64 peak is measured in the same run by an FMA probe kernel.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (torchrun): every rank solves its own copy (independent replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METHODS10 = ["bl_bicg", "bl_bicg_rq", "gl_bicg", "egl_bicg", "bl_bicgstab", "bl_bicgstab_rq", "gl_bicgstab",
             "bl_qmr", "gl_qmr", "egl_qmr"]
# the methods that reach 1e-8 on the 128^3 s = 8 workload within the iteration limit (measured; the
# GPU arm re-derives the set from its per-method pass, the reference arm uses this list)
HEADLINE_METHODS = ["bl_bicg", "bl_bicg_rq", "gl_bicg", "egl_bicg", "bl_bicgstab", "bl_bicgstab_rq", "gl_bicgstab",
                    "gl_qmr", "egl_qmr"]
HBM_FALLBACK_GBS = 6800.0
# nominal FP64 FMA rate for context only (152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz); the
# roofline divides by the rate of the FMA probe measured in the same run
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--s", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=3000)
    ap.add_argument("--methods", default="",
                    help="comma-separated methods (default: the ten of the workload; reference arm: the headline set)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--per-method-reps", type=int, default=3,
                    help="timed solves per method in the per-method pass (median reported)")
    ap.add_argument("--skip-per-method", action="store_true",
                    help="profiling captures: no per-method pass; every method of --methods is a headline method")
    ap.add_argument("--window", type=int, default=50,
                    help="iterations per headline method in one step of the timed region")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--operator", choices=("lattice", "csr"), default="lattice",
                    help="config-4 operator: matrix-free lattice (kr_op_create_lattice4d) or its CSR storage")
    ap.add_argument("--ilu", action="store_true",
                    help="time to 1e-8 with and without ILU(0) right preconditioning on 3D convection-diffusion (--grid, --s)")
    ap.add_argument("--config1", action="store_true",
                    help="time to 1e-8 per method on the 2D 32x32 problem (s = 4), eager launches vs CUDA-graph replay")
    ap.add_argument("--config3", action="store_true",
                    help="time to 1e-8 per method on the 4D lattice (16^4 x 12, s = 12 point sources and 12 Gaussian)")
    ap.add_argument("--config4", action="store_true",
                    help="mixed precision vs FP64 on the 4D lattice (24^4 x 12, s = 32, eGl-BiCG to 1e-10)")
    ap.add_argument("--spmm-rates", action="store_true",
                    help="fused product + trace kernel rates only (complex64 and complex128) on 3D "
                         "convection-diffusion (--grid, --s)")
    ap.add_argument("--cpu-sample-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-iters", type=int, default=5)
    ap.add_argument("--spec", default="", help=argparse.SUPPRESS)
    ap.add_argument("--config2-sweep", action="store_true",
                    help="time to 1e-8 of every method on the 128^3 workload for s in {1, 4, 8, 16}")
    ap.add_argument("--config5", action="store_true",
                    help="differentiation: forward eGl-BiCG + adjoint solve + gradient on 3D convection-diffusion "
                         "64^3 with learnable Peclet numbers, s = 16; gradient checked against finite differences")
    return ap.parse_args()


def workload(grid, s):
    from workloads import ConvDiff, convdiff_csr, gaussian_block
    op = ConvDiff((grid, grid, grid), (0.8, 0.8, 0.8), 0.05j)
    rp, ci, v = convdiff_csr(op)
    B = gaussian_block(op.n, s, seed=0)
    return op, rp, ci, v, B


def workload_name(grid, s, n, nnz):
    return ("3D convection-diffusion %d^3 (n=%d, nnz=%d), Pe 0.8, shift 0.05i, s=%d Gaussian RHS, "
            "FP64 to relative residual 1e-8, X0=0" % (grid, n, nnz, s))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------------------------------
# CPU oracle samples (fresh processes from the spawn start method, single-threaded BLAS each)
# ------------------------------------------------------------------------------------------
#
# The oracle runs as it stands; the only addition is a clock read at the start of its first
# iteration and at the end of each iteration (its iteration monitor's begin / step), so that
# the per-iteration time excludes the set-up product R_0 = B - A X_0 and the final true
# residual.  Each method runs in its own process; processes run concurrently on the host's
# cores.

_ORACLE = {}


def convdiff_spec(grid, s, pe=(0.8, 0.8, 0.8), shift=0.05, seed=0):
    """A 3D convection-diffusion workload: grid^3, cell Peclet numbers pe, diagonal shift i*shift,
    s Gaussian right-hand sides from `seed`."""
    return {"grid": int(grid), "s": int(s), "pe": [float(x) for x in pe], "shift": float(shift), "seed": int(seed)}


def _oracle_init(spec):
    """Pool initializer: the workload's matrix, its adjoint and B, once per process."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[k] = "1"
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    import oracle.methods as om
    from workloads import ConvDiff, convdiff_csr, gaussian_block
    g = spec["grid"]
    op = ConvDiff((g, g, g), tuple(spec["pe"]), 1j * spec["shift"])
    rp, ci, v = convdiff_csr(op)
    B = gaussian_block(op.n, spec["s"], seed=spec["seed"])
    A = oracle.csr_matrix_from_arrays(op.n, rp, ci, v)
    _ORACLE.update(A=A, AH=oracle.adjoint(A), B=B, s=spec["s"], stamps=[])
    stamps = _ORACLE["stamps"]
    begin, step = om._Monitor.begin, om._Monitor.step

    def timed_begin(self, nrm0):
        stamps.append(time.time())
        return begin(self, nrm0)

    def timed_step(self, rnorm):
        r = step(self, rnorm)
        stamps.append(time.time())
        return r

    om._Monitor.begin, om._Monitor.step = timed_begin, timed_step


def _oracle_iterations(task):
    """Run `iters` iterations of one method from X_0 = 0; returns the wall-clock stamps of the
    timed iterations (the first `skip` iterations are run but not timed)."""
    method, iters, skip = task
    import oracle
    st = _ORACLE["stamps"]
    st.clear()
    r = oracle.solve(method, _ORACLE["A"], _ORACLE["B"], tol=0.0, maxit=iters, AH=_ORACLE["AH"])
    stamps = list(st)  # begin, then one stamp per completed iteration
    done = r.iters
    t0, t1 = stamps[skip], stamps[done]
    return {"method": method, "units": _ORACLE["s"] * (done - skip), "start": t0, "end": t1,
            "seconds": t1 - t0, "iters": done - skip, "status": r.status.name}


def host_description():
    cores = os.cpu_count() or 1
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model


def oracle_sample(spec, methods, iters, skip, procs):
    """Concurrent oracle runs, one process per method: per-method seconds per timed iteration,
    the single-thread rate (all timed units over the summed per-process times) and the
    all-core rate (the same units over the wall-clock span of the concurrent timed sections)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=procs, initializer=_oracle_init, initargs=(spec,)) as pool:
        rows = pool.map(_oracle_iterations, [(m, iters, skip) for m in methods])
    units = sum(r["units"] for r in rows)
    serial = sum(r["seconds"] for r in rows)
    span = max(r["end"] for r in rows) - min(r["start"] for r in rows)
    return {"units": units, "single_thread_value": units / serial, "all_core_value": units / span,
            "serial_seconds": serial, "wall_seconds": span, "procs": procs,
            "per_method": {r["method"]: {"s_per_iter": r["seconds"] / max(r["iters"], 1), "iters": r["iters"]}
                           for r in rows}}


def cpu_sample_worker(args):
    methods = args.methods.split(",")
    procs = min(len(methods), os.cpu_count() or 1)
    spec = json.loads(args.spec) if args.spec else convdiff_spec(args.grid, args.s)
    d = oracle_sample(spec, methods, args.sample_iters + 1, 1, procs)
    cores, model = host_description()
    d.update(cores=cores, cpu_model=model, iters_per_method=args.sample_iters, methods=methods)
    print(json.dumps(d))


def run_cpu_sample(args, methods, spec=None):
    """The oracle baseline in a fresh interpreter (no CUDA state is inherited)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample-worker", "--grid", str(args.grid), "--s",
           str(args.s), "--methods", ",".join(methods), "--sample-iters", str(args.sample_iters)]
    if spec is not None:
        cmd += ["--spec", json.dumps(spec)]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("CPU oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_sample_desc(args, d):
    return ("oracle (numpy/scipy FP64) on the full %d^3 s=%d workload: %d timed iterations of each of %d methods "
            "(%s) after one untimed iteration from X0=0, the set-up product R0 and the final true residual "
            "excluded; one single-threaded process per method, %d processes at once on %d cores (%s); value = "
            "all-core rate (units over the wall-clock span of the concurrent timed iterations), single_thread = "
            "units over the summed per-process times"
            % (args.grid, args.s, d["iters_per_method"], len(d["methods"]), ",".join(d["methods"]), d["procs"],
               d["cores"], d["cpu_model"]))


def reference_arm(args):
    """The oracle as the reference arm: each step runs one iteration of every headline method,
    one process per method at once (a persistent pool that built the matrix once); the step's
    time is the wall-clock span of those concurrent iterations (R_0 and the final residual of
    each run excluded)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    methods = args.methods.split(",") if args.methods else list(HEADLINE_METHODS)
    procs = min(len(methods), os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    units, secs = 0, 0.0
    with ctx.Pool(processes=procs, initializer=_oracle_init, initargs=(convdiff_spec(args.grid, args.s),)) as pool:
        for i in range(args.warmup + args.steps):
            rows = pool.map(_oracle_iterations, [(m, 1, 0) for m in methods])
            if i >= args.warmup:
                units += sum(r["units"] for r in rows)
                secs += max(r["end"] for r in rows) - min(r["start"] for r in rows)
    value = units / secs
    cores, model = host_description()
    from workloads import grid_nnz
    n = args.grid ** 3
    sample = ("oracle (numpy/scipy FP64) on the full %d^3 s=%d workload: per step one iteration of each of %d "
              "methods (%s) from X0=0, one single-threaded process per method, %d at once on %d cores (%s); "
              "step time = wall-clock span of the concurrent iterations, R0 and the final residual excluded"
              % (args.grid, args.s, len(methods), ",".join(methods), procs, cores, model))
    line = {
        "impl": "reference", "metric": "RHS·iters/s", "value": value, "unit": "RHS·iters/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.grid, args.s, n, grid_nnz((args.grid,) * 3)), "s": args.s,
                   "methods": methods, "sample": "one iteration per method per step"},
        "cpu_baseline": {"value": value, "unit": "RHS·iters/s", "cores": procs, "kind": "oracle", "sample": sample,
                         "host_cores": cores, "cpu_model": model},
        "e2e": {"value": value, "unit": "RHS·iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# multi-rank aggregation (independent replicas: no data-path collective)
# ------------------------------------------------------------------------------------------

def aggregate_over_ranks(elapsed_s, units, dist=None, device="cpu"):
    """Whole-job throughput: all ranks' units over the slowest rank's time (max over ranks)."""
    if dist is None:
        return units / elapsed_s, elapsed_s, units
    import torch
    t = torch.tensor([elapsed_s, float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tsum[1]) / float(tmax[0]), float(tmax[0]), float(tsum[1])


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                    pw.append(float(p[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(pw) if pw else None}


def fma_peaks(kr, torch):
    """Measured FMA rates (TFLOP/s) of the probe kernel: FP64 and FP32, best of 5 launches of
    about 0.3 s each after about a second of warm-up launches (clocks settle), CUDA events on
    the launching stream."""
    out = {}
    for prec, iters in (("fp64", 1 << 20), ("fp32", 1 << 23)):
        for _ in range(3):
            kr.kr_probe_fma(prec, iters)
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fl, _ = kr.kr_probe_fma(prec, iters)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) / 1000.0) / 1e12)
        out[prec] = best
    return out


def solve_timed(kr, torch, A, m, Bd, Xd, tol, maxit, stream, check_every=8):
    """One kr_solve from X_0 = 0 bracketed by CUDA events on the launching stream: (info, ms)."""
    Xd.zero_()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    _, info = kr.kr_solve(A, m, Bd, Xd, tol=tol, maxit=maxit, check_every=check_every)
    t1.record(stream)
    t1.synchronize()
    return info, t0.elapsed_time(t1)


def gpu_arm(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    op_, rp, ci, v, B = workload(args.grid, args.s)
    n, s = op_.n, args.s
    methods = args.methods.split(",") if args.methods else list(METHODS10)
    A = kr.Operator(n, rp, ci, v, device=local)
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    stream = torch.cuda.current_stream()
    peaks = fma_peaks(kr, torch)

    # time to 1e-8 of every method (median of --per-method-reps solves after an untimed 3-iteration
    # solve that allocates the method's workspace).  Methods that
    # stall or break down are reported here and left out of the headline value.
    per_method = {}
    for m in ([] if args.skip_per_method else methods):
        kr.kr_solve(A, m, Bd, Xd, tol=args.tol, maxit=3)  # the method's workspace, untimed
        runs = [solve_timed(kr, torch, A, m, Bd, Xd, args.tol, args.maxit, stream)
                for _ in range(max(1, args.per_method_reps))]
        info = runs[0][0]
        ms = statistics.median(r[1] for r in runs)
        per_method[m] = {"status": info.status, "iters": info.iters, "relres_true": info.relres_true,
                         "time_to_tol_ms": ms if info.status == "OK" else None,
                         "ms_to_exit": ms, "rhs_iters_per_s": s * info.iters / (ms / 1000.0),
                         "timed_solves": len(runs)}
        if info.status == "BREAKDOWN":
            per_method[m]["breakdown_iter"] = info.breakdown_iter
    headline = [m for m in methods if args.skip_per_method or per_method[m]["status"] == "OK"]
    if not headline:
        raise RuntimeError("no method reached the tolerance: %s" % per_method)

    # one step: the first `window` iterations from X0 = 0 of every headline method (each iteration
    # costs the same whichever it is; the whole solves are timed in per_method above)
    def step(record=None):
        for m in headline:
            Xd.zero_()
            _, info = kr.kr_solve(A, m, Bd, Xd, tol=0.0, maxit=args.window)
            if record is not None:
                record.append((m, info))

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    recs = []
    for _ in range(args.steps):
        step(recs)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    units_rank = sum(s * info.iters for (_, info) in recs)
    value, elapsed_s, _ = aggregate_over_ranks(e0.elapsed_time(e1) / 1000.0, units_rank, dist, "cuda")
    ms_per_step = 1000.0 * elapsed_s / args.steps

    # per kernel class: one more step with every launch bracketed by CUDA events (separate from
    # the timed region, whose launches are not instrumented)
    kr.kr_profile_read(reset=True)
    kr.kr_profile_enable(True, time_kernels=True)
    step()
    torch.cuda.synchronize()
    prof = kr.kr_profile_read(reset=True)
    kr.kr_profile_enable(False)
    launches_per_step = int(sum(c["launches"] for c in prof.values()))
    dom = max(("spmm", "lincomb", "spmm_c64", "lincomb_c64"), key=lambda k: prof[k]["ms"])
    total_kernel_ms = sum(c["ms"] for c in prof.values())
    hbm_peak, hbm_src = measured_peaks()
    fp64_peak = peaks["fp64"]
    pd = prof[dom]
    achieved = pd["flops"] / (pd["ms"] / 1000.0) / 1e12 if pd["ms"] > 0 else None
    roofline = {
        "kernel": dom, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
        "frac": (achieved / fp64_peak) if achieved else None, "traffic": None,
        "peak_source": "measured: FP64 FMA probe kr_probe_fma (16 independent DFMA chains per thread, 4x256 "
                       "threads per SM, best of 5 launches after 3 warm-up launches, CUDA events), this run",
        "nominal_fp64_tflops": FP64_NOMINAL_TFLOPS, "measured_fp32_tflops": peaks["fp32"],
        "timing": "per-launch CUDA events in a separate profiled step after the timed region",
        "launches": pd["launches"], "avg_launch_ms": pd["ms"] / max(pd["launches"], 1),
        "hbm_achieved_gbs": pd["bytes"] / (pd["ms"] / 1000.0) / 1e9 if pd["ms"] > 0 else None,
        "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
        "share_of_kernel_time": {k: c["ms"] / total_kernel_ms for k, c in prof.items()} if total_kernel_ms else {},
        "per_class": {k: {"launches": c["launches"], "ms": c["ms"],
                          "tflops": c["flops"] / (c["ms"] / 1000.0) / 1e12 if c["ms"] > 0 else None,
                          "fp64_frac": c["flops"] / (c["ms"] / 1000.0) / 1e12 / fp64_peak if c["ms"] > 0 else None,
                          "gbs": c["bytes"] / (c["ms"] / 1000.0) / 1e9 if c["ms"] > 0 else None}
                      for k, c in prof.items()},
    }
    # DRAM traffic per launch from the committed ncu capture, only while the files that define
    # the kernel and its launch are the ones that capture measured (otherwise null)
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        key = "%s_%d_%d" % (dom, args.grid, s)
        if key in tr and tr[key].get("kernel_digest") == build.kernel_digest(tr[key]["kernel_sources"]):
            roofline["traffic"] = tr[key]["bytes_per_launch"]
            roofline["traffic_instance"] = tr[key]["instance"]
            roofline["traffic_algorithmic_bytes"] = tr[key]["algorithmic_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass

    # ---- end-to-end through the C interface with host buffers (pinned), copies in the timed region
    e2e = None
    if not args.no_e2e:
        Bh = torch.from_numpy(B).pin_memory()
        Xh = torch.zeros_like(Bh).pin_memory()
        step_bytes = n * s * 16
        barrier()
        t0 = time.perf_counter()
        e2e_units = 0
        for _ in range(args.e2e_steps):
            for m in headline:
                Xh.zero_()
                _, info = kr.kr_solve(A, m, Bh, Xh, tol=0.0, maxit=args.window)
                e2e_units += s * info.iters
        barrier()
        e2e_value, _, _ = aggregate_over_ranks(time.perf_counter() - t0, e2e_units, dist, "cuda")
        e2e = {"value": e2e_value, "unit": "RHS·iters/s", "steps": args.e2e_steps,
               "h2d_bytes_per_step": 2 * step_bytes * len(headline), "d2h_bytes_per_step": step_bytes * len(headline)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            d = run_cpu_sample(args, headline)
            cpu = {"value": d["all_core_value"], "unit": "RHS·iters/s", "cores": d["procs"], "kind": "oracle",
                   "sample": cpu_sample_desc(args, d), "single_thread": d["single_thread_value"],
                   "host_cores": d["cores"], "cpu_model": d["cpu_model"],
                   "s_per_iter": {m: r["s_per_iter"] for m, r in d["per_method"].items()}}
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "unit": "RHS·iters/s", "cores": None, "kind": "oracle", "sample": "failed: %s" % e}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = bench_extras(kr, A, n, s, B, rp, ci, v, args, hbm_peak)

    if rank == 0:
        line = {
            "metric": "RHS·iters/s", "value": value, "unit": "RHS·iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.grid, s, n, len(ci)), "s": s, "tol": args.tol,
                       "maxit": args.maxit, "methods": methods, "headline_methods": headline,
                       "step": "the first %d iterations from X0=0 (R0, the iterations and the final true residual) "
                               "of each headline method: the methods that reached tol within maxit in the "
                               "per-method pass, whose whole solves are timed there (time_to_tol_ms); the others "
                               "are in per_method with their status" % args.window,
                       "window": args.window,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (one n x s complex128 block = %.0f MB > 129 MB)"
                             % (n * s * 16 / 1e6)},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "per_method": per_method,
            "fma_peaks_tflops": peaks,
        }
        line.update(extras)
        print(json.dumps(line))
    A.close()
    if dist is not None:
        dist.destroy_process_group()


def bench_extras(kr, A, n, s, B, rp, ci, v, args, hbm_peak):
    """SpMM kernel rates for s in {1, 4, 8, 16} (plain, and fused with a Gram / trace reduction in
    complex128 and complex64) and FP32+refine vs FP64 eGl-BiCG."""
    import torch
    out = {"spmm": {}}
    nnz = len(ci)
    info = A.info()
    for ss in (1, 4, 8, 16):
        V = torch.randn(n, ss, dtype=torch.complex128, device="cuda")
        Y = torch.empty_like(V)
        for _ in range(3):
            kr.kr_op_apply(A, V, Y)
        torch.cuda.synchronize()
        reps = 20
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            kr.kr_op_apply(A, V, Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if info["real_offdiag"]:
            noff = nnz - n
            mbytes = 8 * (n + 1) + 4 * noff + 8 * noff + 16 * n
            flops = ss * (4.0 * noff + 6.0 * n)
        else:
            mbytes = 8 * (n + 1) + 4 * nnz + 16 * nnz
            flops = ss * 8.0 * nnz
        byts = mbytes + 2 * 16 * n * ss
        out["spmm"][str(ss)] = {"ms": ms, "gbs": byts / ms / 1e6, "hbm_frac": byts / ms / 1e6 / hbm_peak,
                                "tflops": flops / ms / 1e9, "fp64_frac_nominal": flops / ms / 1e9 / FP64_NOMINAL_TFLOPS}
        del V, Y
    # fused SpMM + reduction (the product with the s x s Gram U^H (A V) or the trace of it in its
    # epilogue), complex128 and complex64, rates from the library's launch profile
    out["spmm_fused"] = {}
    for ss in (1, 4, 8, 16):
        for dt, cls, kinds in ((torch.complex128, "spmm", ("gram",)), (torch.complex64, "spmm_c64", ("gram", "trace"))):
            V = torch.randn(n, ss, dtype=dt, device="cuda")
            U = torch.randn_like(V)
            Y = torch.empty_like(V)
            for kind in kinds:
                if dt == torch.complex128:
                    def fn():
                        kr.kr_op_apply_reduce(A, V, U, kind=kind, Y=Y)
                else:
                    def fn():
                        kr.kr_op_apply_reduce_c64(A, V, U, kind=kind, Y=Y)
                for _ in range(3):
                    fn()
                torch.cuda.synchronize()
                kr.kr_profile_read(reset=True)
                kr.kr_profile_enable(True, time_kernels=True)
                for _ in range(20):
                    fn()
                torch.cuda.synchronize()
                c = kr.kr_profile_read(reset=True)[cls]
                kr.kr_profile_enable(False)
                ms = c["ms"] / c["launches"]
                gbs = c["bytes"] / c["ms"] / 1e6
                out["spmm_fused"]["%s_%s_s%d" % ("c128" if cls == "spmm" else "c64", kind, ss)] = {
                    "ms": ms, "gbs": gbs, "hbm_frac": gbs / hbm_peak, "tflops": c["flops"] / c["ms"] / 1e9}
            del V, U, Y
    # mixed precision: complex64 inner solves (tol 1e-4) in FP64 defect correction, eGl-BiCG to 1e-8
    Bd = torch.from_numpy(B).cuda()
    res = {}
    for prec, name in ((kr.FP64, "fp64"), (kr.FP32_REFINE, "fp32_refine")):
        X = torch.zeros_like(Bd)
        kr.kr_solve(A, "egl_bicg", Bd, X, tol=args.tol, maxit=args.maxit, precision=prec, check_every=1)
        times = []
        for _ in range(3):
            X.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf = kr.kr_solve(A, "egl_bicg", Bd, X, tol=args.tol, maxit=2000, precision=prec, check_every=1)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        res[name] = {"time_to_tol_ms": 1000 * statistics.median(times), "iters": inf.iters,
                     "outer": inf.outer_iters, "relres_true": inf.relres_true, "status": inf.status, "X": X.clone()}
        # per kernel class rates of one more solve, CUDA events around every launch
        X.zero_()
        kr.kr_profile_read(reset=True)
        kr.kr_profile_enable(True, time_kernels=True)
        kr.kr_solve(A, "egl_bicg", Bd, X, tol=args.tol, maxit=2000, precision=prec, check_every=1)
        torch.cuda.synchronize()
        prof = kr.kr_profile_read(reset=True)
        kr.kr_profile_enable(False)
        res[name]["per_class"] = {
            k: {"launches": c["launches"], "ms": c["ms"],
                "gbs": c["bytes"] / (c["ms"] / 1000.0) / 1e9 if c["ms"] > 0 else None,
                "hbm_frac": c["bytes"] / (c["ms"] / 1000.0) / 1e9 / hbm_peak if c["ms"] > 0 else None,
                "tflops": c["flops"] / (c["ms"] / 1000.0) / 1e12 if c["ms"] > 0 else None}
            for k, c in prof.items() if c["launches"]}
    diff = float(torch.linalg.norm(res["fp32_refine"]["X"] - res["fp64"]["X"]) / torch.linalg.norm(res["fp64"]["X"]))
    for r in res.values():
        r.pop("X")
    # the same solves with the literal schedule of Algorithm 4 (alpha from A P, separate update)
    kr.kr_set_fused_products(False)
    try:
        for prec, name in ((kr.FP64, "fp64"), (kr.FP32_REFINE, "fp32_refine")):
            times = []
            for _ in range(3):
                X = torch.zeros_like(Bd)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, inf = kr.kr_solve(A, "egl_bicg", Bd, X, tol=args.tol, maxit=2000, precision=prec, check_every=1)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            res[name]["literal_schedule"] = {"time_to_tol_ms": 1000 * statistics.median(times), "iters": inf.iters,
                                             "status": inf.status, "relres_true": inf.relres_true}
    finally:
        kr.kr_set_fused_products(True)
    out["mixed"] = {"method": "egl_bicg", **res,
                    "speedup": res["fp64"]["time_to_tol_ms"] / res["fp32_refine"]["time_to_tol_ms"],
                    "rel_diff_vs_fp64_gpu": diff}
    # the same problem as a matrix-free stencil operator (complex64 products on the plane kernel,
    # FP64 products from the stencil's coefficients): the same solves, timed the same way
    from workloads import ConvDiff
    cd = ConvDiff((args.grid,) * 3, (0.8, 0.8, 0.8), 0.05j)
    St = kr.Operator.stencil(cd.dims, *cd.coefficients())
    try:
        sres = {}
        for prec, name in ((kr.FP64, "fp64"), (kr.FP32_REFINE, "fp32_refine")):
            X = torch.zeros_like(Bd)
            kr.kr_solve(St, "egl_bicg", Bd, X, tol=args.tol, maxit=2000, precision=prec, check_every=1)
            times = []
            for _ in range(3):
                X.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, inf = kr.kr_solve(St, "egl_bicg", Bd, X, tol=args.tol, maxit=2000, precision=prec, check_every=1)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            sres[name] = {"time_to_tol_ms": 1000 * statistics.median(times), "iters": inf.iters,
                          "outer": inf.outer_iters, "relres_true": inf.relres_true, "status": inf.status}
        out["mixed_stencil"] = {"method": "egl_bicg", "operator": "matrix-free 7-point stencil of the same A", **sres,
                                "speedup": sres["fp64"]["time_to_tol_ms"] / sres["fp32_refine"]["time_to_tol_ms"]}
    finally:
        St.close()
    return out


def config4(args):
    """Mixed precision (complex64 inner solves, tol 1e-4, FP64 defect correction to 1e-10) against the
    pure-FP64 GPU path on the 4D lattice operator, 24^4 sites x 12 dof (n = 3,981,312, 49 entries per
    row), s = 32 Gaussian right-hand sides, eGl-BiCG (Algorithm 4)."""
    import torch
    from workloads import Lattice4D, gaussian_block, lattice_csr
    from workloads.lattice import GAMMA, LATTICE_MASS, haar_links
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    L = args.grid if args.grid != 128 else 24
    s = args.s if args.s != 8 else 32
    lat = Lattice4D((L,) * 4, LATTICE_MASS, seed=0)
    t0 = time.perf_counter()
    links = haar_links(lat.dims, lat.seed)
    if args.operator == "csr":
        rp, ci, v = lattice_csr(lat, links)
        nnz = len(ci)
    else:
        nnz = 49 * lat.n
    gen_s = time.perf_counter() - t0
    if args.operator == "csr":
        A = kr.Operator(lat.n, rp, ci, v)
    else:
        A = kr.Operator.lattice4d(lat.dims, 4.0 + LATTICE_MASS, -0.5, GAMMA, links)
    B = torch.from_numpy(gaussian_block(lat.n, s, seed=32)).cuda()
    hbm_peak, _ = measured_peaks()
    out = {"workload": "4D lattice %d^4 x 12 (n=%d, nnz=%d), m=%.2f, s=%d Gaussian RHS, eGl-BiCG to 1e-10, %s operator"
                       % (L, lat.n, nnz, LATTICE_MASS, s, "matrix-free" if args.operator == "lattice" else "CSR"),
           "mass_reading": "diagonal 4 + m with m = %.2f, the spectrum kept in the right half-plane as the paper "
                           "states for Example 4 (kappa about 54 on 4^4) rather than kappa = 1e3" % LATTICE_MASS,
           "generation_s": gen_s}
    X = {}
    for prec, name in ((kr.FP64, "fp64"), (kr.FP32_REFINE, "fp32_refine")):
        # first call: device copies (complex64 operator for the mixed path) and workspaces
        t0 = time.perf_counter()
        kr.kr_solve(A, "egl_bicg", B, torch.zeros_like(B), tol=1e-10, maxit=2, precision=prec, inner_tol=1e-4)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        Xd = torch.zeros_like(B)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf = kr.kr_solve(A, "egl_bicg", B, Xd, tol=1e-10, maxit=5000, precision=prec, inner_tol=1e-4,
                             check_every=8)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        # the same solve again with every launch timed (events add host work: not the headline)
        kr.kr_profile_read(reset=True)
        kr.kr_profile_enable(True, time_kernels=True)
        kr.kr_solve(A, "egl_bicg", B, torch.zeros_like(B), tol=1e-10, maxit=5000, precision=prec, inner_tol=1e-4,
                    check_every=8)
        torch.cuda.synchronize()
        prof = kr.kr_profile_read(reset=True)
        kr.kr_profile_enable(False)
        X[name] = Xd
        out[name] = {"time_to_tol_s": el, "first_call_setup_s": setup, "status": inf.status, "iters": inf.iters,
                     "outer": inf.outer_iters, "fp64_iters": inf.fp64_iters, "relres_true": inf.relres_true,
                     "kernel_ms": round(sum(c["ms"] for c in prof.values()), 3),
                     "per_class": {k: {"launches": c["launches"], "ms": round(c["ms"], 3),
                                       "gbs": c["bytes"] / (c["ms"] / 1e3) / 1e9 if c["ms"] > 0 else None,
                                       "hbm_frac": c["bytes"] / (c["ms"] / 1e3) / 1e9 / hbm_peak if c["ms"] > 0
                                       else None,
                                       "tflops": c["flops"] / (c["ms"] / 1e3) / 1e12 if c["ms"] > 0 else None}
                                   for k, c in prof.items() if c["launches"]}}
    out["speedup"] = out["fp64"]["time_to_tol_s"] / out["fp32_refine"]["time_to_tol_s"]
    out["rel_diff_mixed_vs_fp64"] = float(torch.linalg.norm(X["fp32_refine"] - X["fp64"]) / torch.linalg.norm(X["fp64"]))
    print(json.dumps(out))
    A.close()


def ilu_mode(args):
    """Sec. 5's second set of experiments on the config-2 problem: 3D convection-diffusion
    (--grid^3, Pe 0.8, shift 0.05i, --s Gaussian right-hand sides), time to a relative
    residual of 1e-8 without and with ILU(0) right preconditioning, for the methods of
    --methods.  The factorisation (host, FP64) is timed separately."""
    import torch
    from workloads import ConvDiff, convdiff_csr, gaussian_block
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    L, s = args.grid, args.s
    op = ConvDiff((L, L, L), (0.8, 0.8, 0.8), 0.05j)
    rp, ci, v = convdiff_csr(op)
    A = kr.Operator(op.n, rp, ci, v)
    B = torch.from_numpy(gaussian_block(op.n, s, seed=0)).cuda()
    methods = ["egl_bicg", "gl_bicg", "bl_bicgstab", "gl_bicgstab"]
    if args.methods:
        methods = args.methods.split(",")
    out = {"workload": "3D convection-diffusion %d^3 (n=%d), Pe 0.8, shift 0.05i, s=%d Gaussian RHS, to 1e-8"
                       % (L, op.n, s), "results": {}}
    for prec in (None, "ilu0"):
        t0 = time.perf_counter()
        A.set_preconditioner(prec)
        torch.cuda.synchronize()
        if prec:
            out["ilu0_setup_s"] = time.perf_counter() - t0
        for method in methods:
            kr.kr_solve(A, method, B, torch.zeros_like(B), tol=1e-8, maxit=3)  # workspaces
            X = torch.zeros_like(B)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf = kr.kr_solve(A, method, B, X, tol=1e-8, maxit=args.maxit)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            out["results"]["%s_%s" % (method, prec or "none")] = {
                "time_to_tol_ms": 1000 * el, "iters": inf.iters, "status": inf.status,
                "relres_true": inf.relres_true}
    print(json.dumps(out))
    A.close()


def config1(args):
    """Config 1 (2D convection-diffusion 32 x 32, n = 1024, Pe 0.5, shift 0.1i, s = 4 Gaussian RHS,
    seed 0, X0 = 0, relative residual 1e-8): time to tolerance per method with eager launches and
    with the iterations replayed as a CUDA graph.  At this size a kernel takes a few
    microseconds, so launch overhead, not the GPU, sets the pace without graphs."""
    import statistics
    import torch
    from workloads import ConvDiff, convdiff_csr, gaussian_block
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    op = ConvDiff((32, 32), (0.5, 0.5), 0.1j)
    rp, ci, v = convdiff_csr(op)
    A = kr.Operator(op.n, rp, ci, v)
    B = torch.from_numpy(gaussian_block(op.n, 4, seed=0)).cuda()
    out = {"workload": "2D convection-diffusion 32^2 (n=1024), Pe 0.5, shift 0.1i, s=4 Gaussian RHS, to 1e-8",
           "results": {}}
    methods = ["bl_bicg", "bl_bicg_rq", "gl_bicg", "egl_bicg", "bl_bicgstab", "gl_bicgstab", "bl_qmr", "egl_qmr"]
    for method in methods:
        row = {}
        for mode in ("off", "on"):
            kr.kr_solve(A, method, B, torch.zeros_like(B), tol=1e-8, maxit=1000, graphs=mode)
            times = []
            for _ in range(5):
                X = torch.zeros_like(B)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, inf = kr.kr_solve(A, method, B, X, tol=1e-8, maxit=1000, graphs=mode)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            row["time_to_tol_ms_graphs_" + mode] = 1000 * statistics.median(times)
            row["iters"] = inf.iters
            row["status"] = inf.status
        row["graph_speedup"] = row["time_to_tol_ms_graphs_off"] / row["time_to_tol_ms_graphs_on"]
        out["results"][method] = row
    print(json.dumps(out))
    A.close()


def config3(args):
    """Time to a relative residual of 1e-8 per method on the 4D lattice operator, 16^4 sites x 12
    (n = 786,432), s = 12 point sources at one seeded site and s = 12 Gaussian right-hand sides:
    eGl-BiCG and eGl-QMR (Algorithm 4 and its QMR counterpart) and Bl-BiCGStab-rQ.  For the
    point sources every method takes a seeded Gaussian shadow (see below)."""
    import numpy as np
    import torch
    from workloads import Lattice4D, gaussian_block, lattice_csr, point_sources
    from workloads.lattice import GAMMA, LATTICE_MASS, haar_links
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    L = args.grid if args.grid != 128 else 16
    lat = Lattice4D((L,) * 4, LATTICE_MASS, seed=0)
    links = haar_links(lat.dims, lat.seed)
    if args.operator == "csr":
        rp, ci, v = lattice_csr(lat, links)
        A = kr.Operator(lat.n, rp, ci, v)
    else:
        A = kr.Operator.lattice4d(lat.dims, 4.0 + LATTICE_MASS, -0.5, GAMMA, links)
    site = int(np.random.default_rng(12).integers(0, lat.sites))
    rhs = {"point": point_sources(lat.n, 12, site), "gauss": gaussian_block(lat.n, 12, seed=12)}
    # point sources: seeded Gaussian shadows (vector for the economic methods, block for
    # Bl-BiCGStab-rQ); with the default shadows built from the 12 unit vectors of one site the
    # first inner products are exact zeros plus rounding noise
    shadow_vec = torch.from_numpy(np.ascontiguousarray(gaussian_block(lat.n, 1, seed=5)[:, 0])).cuda()
    shadow_blk = torch.from_numpy(gaussian_block(lat.n, 12, seed=5)).cuda()
    out = {"workload": "4D lattice %d^4 x 12 (n=%d), m=%.2f, s=12, to 1e-8, %s operator"
                       % (L, lat.n, LATTICE_MASS, "matrix-free" if args.operator == "lattice" else "CSR"),
           "mass_reading": "diagonal 4 + m with m = %.2f, the spectrum kept in the right half-plane as the paper "
                           "states for Example 4 (kappa about 54 on 4^4); a mass giving kappa = 1e3 puts eigenvalues "
                           "in the left half-plane, where all three methods diverge on 16^4" % LATTICE_MASS,
           "shadow_reading": "point sources (the 12 unit vectors of one site): seeded Gaussian shadows (a vector for "
                             "the economic methods, a 12-column block for Bl-BiCGStab-rQ), since the default shadows "
                             "make the first inner products cancel to rounding noise; Gaussian right-hand sides: the "
                             "paper's defaults (R0, the mean of R0's columns)",
           "results": {}}
    for kind, B in rhs.items():
        Bd = torch.from_numpy(B).cuda()
        for method in ("egl_bicg", "egl_qmr", "bl_bicgstab_rq"):
            sh = None
            if kind == "point":
                sh = shadow_vec if method.startswith("egl") else shadow_blk
            kr.kr_solve(A, method, Bd, torch.zeros_like(Bd), tol=1e-8, maxit=3, shadow=sh)  # workspaces
            X = torch.zeros_like(Bd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf = kr.kr_solve(A, method, Bd, X, tol=1e-8, maxit=3000, shadow=sh)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            out["results"]["%s_%s" % (method, kind)] = {
                "time_to_tol_ms": 1000 * el, "status": inf.status, "iters": inf.iters,
                "relres_true": inf.relres_true, "rhs_iters_per_s": 12 * inf.iters / el}
    print(json.dumps(out))
    A.close()


def spmm_rates(args):
    """Rates of the product fused with an s x s Gram U^H (A V) or a trace tr(U^H A V) (U a streamed
    n x s block) on 3D convection-diffusion (--grid, --s): complex64 on each of its kernels (row
    tiles staged by bulk copies, column pairs, one column per thread) and complex128.  CUDA events
    over 30 launches after 5 warm-up launches, inputs larger than L2.  Algorithmic bytes: the CSR
    arrays once (real off-diagonal storage: 4-byte index and one real value per off-diagonal entry,
    complex diagonal, row pointers), V and U read, Y written.  The same operator as a matrix-free
    7-point stencil (no matrix bytes): complex64 on the plane-marching kernel and on column pairs."""
    import torch
    import paper_1504_04395_gb300 as kr
    from paper_1504_04395_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    op, rp, ci, v, _ = workload(args.grid, args.s)
    A = kr.Operator(op.n, rp, ci, v, device=0)
    n, s, nnz = op.n, args.s, len(ci)
    real_off = A.info()["real_offdiag"]
    hbm_peak, hbm_src = measured_peaks()
    out = {"mode": "spmm_rates", "workload": "3D convection-diffusion %d^3 (n=%d, nnz=%d), s=%d" % (args.grid, n, nnz, s),
           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src, "rates": {}}
    variants = {"tile": (True, True), "pairs": (False, True), "one_column": (False, False)}
    for dt, b, fn in ((torch.complex64, 8, kr.kr_op_apply_reduce_c64), (torch.complex128, 16, kr.kr_op_apply_reduce)):
        g = torch.Generator(device="cuda").manual_seed(s)
        V = torch.randn(n, s, dtype=dt, device="cuda", generator=g)
        U = torch.randn(n, s, dtype=dt, device="cuda", generator=g)
        Y = torch.empty_like(V)
        noff = nnz - n
        mbytes = 8 * (n + 1) + (4 + b // 2) * noff + b * n if real_off else 8 * (n + 1) + (4 + b) * nnz
        byts = mbytes + 3 * b * n * s
        for kind in ("gram", "trace"):
            for vname, (tile, pairs) in (variants.items() if b == 8 else [("fp64", (False, False))]):
                if kind == "gram" and s > 16 and not tile:
                    continue  # the per-thread kernels hold a fused Gram in registers for s <= 16 only
                if b == 8:
                    kr.kr_set_tile_kernels(tile)
                    kr.kr_set_column_pairs(pairs)
                for _ in range(5):
                    fn(A, V, U, kind=kind, Y=Y)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(30):
                    fn(A, V, U, kind=kind, Y=Y)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 30
                gbs = byts / ms / 1e6
                out["rates"]["%s_%s_%s" % ("c64" if b == 8 else "c128", kind, vname)] = {
                    "ms": ms, "bytes": byts, "gbs": gbs, "hbm_frac": gbs / hbm_peak}
        kr.kr_set_tile_kernels(True)
        kr.kr_set_column_pairs(True)
        del V, U, Y
    # the same operator without stored matrix (the 7-point stencil formed from its coefficients):
    # algorithmic bytes are V and U read and Y written
    centre, minus, plus = op.coefficients()
    St = kr.Operator.stencil(op.dims, centre, minus, plus)
    g = torch.Generator(device="cuda").manual_seed(s)
    V = torch.randn(n, s, dtype=torch.complex64, device="cuda", generator=g)
    U = torch.randn(n, s, dtype=torch.complex64, device="cuda", generator=g)
    Y = torch.empty_like(V)
    byts = 3 * 8 * n * s
    for kind in ("gram", "trace"):
        # "plane": the plane-marching kernel (TMA tensor copies of halo'd x-y tiles, 2D/3D grids)
        for vname, (tile, pairs) in (("plane", (True, True)), ("pairs", (False, True))):
            if kind == "gram" and s > 16 and not tile:
                continue
            kr.kr_set_tile_kernels(tile)
            kr.kr_set_column_pairs(pairs)
            for _ in range(5):
                kr.kr_op_apply_reduce_c64(St, V, U, kind=kind, Y=Y)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(30):
                kr.kr_op_apply_reduce_c64(St, V, U, kind=kind, Y=Y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 30
            gbs = byts / ms / 1e6
            out["rates"]["stencil_c64_%s_%s" % (kind, vname)] = {"ms": ms, "bytes": byts, "gbs": gbs,
                                                               "hbm_frac": gbs / hbm_peak}
    kr.kr_set_tile_kernels(True)
    kr.kr_set_column_pairs(True)
    St.close()
    out["device_wait_timeouts"] = kr.kr_take_device_timeouts(reset=True)
    print(json.dumps(out))


def config2_sweep(args):
    """Config 2 across block widths: 3D convection-diffusion --grid^3 (default 128^3), Pe 0.8, shift
    0.05i, s in {1, 4, 8, 16} Gaussian right-hand sides (seed 0), X0 = 0; every method solves to 1e-8
    (maxit --maxit), FP64; per method and s: status, iterations, time to tolerance (CUDA events around
    kr_solve after one untimed solve that allocates the workspaces) and RHS*iterations/s."""
    import torch
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    methods = args.methods.split(",") if args.methods else list(METHODS10)
    stream = torch.cuda.current_stream()
    out = {"mode": "config2_sweep", "tol": args.tol, "maxit": args.maxit, "results": {}}
    op = None
    for s in (1, 4, 8, 16):
        op_, rp, ci, v, B = workload(args.grid, s)
        if op is None:
            op = kr.Operator(op_.n, rp, ci, v)
            out["workload"] = workload_name(args.grid, s, op_.n, len(ci)).replace("s=%d " % s, "")
        Bd = torch.from_numpy(B).cuda()
        Xd = torch.zeros_like(Bd)
        row = {}
        for m in methods:
            kr.kr_solve(op, m, Bd, torch.zeros_like(Bd), tol=args.tol, maxit=2)  # workspaces
            info, ms = solve_timed(kr, torch, op, m, Bd, Xd, args.tol, args.maxit, stream)
            row[m] = {"status": info.status, "iters": info.iters, "relres_true": info.relres_true,
                      "time_to_tol_ms": ms if info.status == "OK" else None, "ms_to_exit": ms,
                      "rhs_iters_per_s": s * info.iters / (ms / 1000.0)}
            if info.status == "BREAKDOWN":
                row[m]["breakdown_iter"] = info.breakdown_iter
        out["results"]["s%d" % s] = row
        del Bd, Xd
    print(json.dumps(out))
    op.close()


def config5(args):
    """Differentiation through the solve (config 5): 3D convection-diffusion 64^3 (n = 262,144)
    whose three cell Peclet numbers (0.3, 0.2, 0.1) are learnable FP64 scalars, shift 0.05i, s = 16
    Gaussian right-hand sides (seed 0), loss ||X - X*||_F^2 with a seeded target X* (seed 1, x0.1).
    One step: forward eGl-BiCG to 1e-8 (Algorithm 4), backward adjoint eGl-BiCG A^H Lambda = dL/dX to
    1e-8, and dL/dA on the stored pattern, through the torch.autograd.Function.  Reported: the
    step's time (median of 5, CUDA-synchronised wall clock), the three phases' CUDA-event times,
    iterations, the gradient against central finite differences of GPU solves at tol 1e-13
    (h = 1e-6), and the oracle's eGl-BiCG seconds per iteration on the same matrix (5 timed
    iterations, one process) scaled by the GPU's forward + adjoint iteration counts (a projection)."""
    import numpy as np
    import torch
    from workloads import ConvDiff, convdiff_csr, gaussian_block
    from workloads.stencil import convdiff_dpe_csr
    pe0, N, s = (0.3, 0.2, 0.1), (args.grid if args.grid != 128 else 64), (args.s if args.s != 8 else 16)
    spec = convdiff_spec(N, s, pe0, 0.05, 0)
    cpu = run_cpu_sample(args, ["egl_bicg"], spec) if not args.no_cpu_baseline else None
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as kr
    from paper_1504_04395_gb300.autograd import krylov_solve
    cd = ConvDiff((N, N, N), (0.0, 0.0, 0.0), 0.05j)
    rp, ci, base = convdiff_csr(cd)
    d = [convdiff_dpe_csr(cd, a).real for a in range(3)]
    n = cd.n
    vals0 = base + sum(pe0[a] * d[a] for a in range(3))
    op = kr.Operator(n, rp, ci, vals0)
    base_t = torch.from_numpy(base).cuda()
    d_t = [torch.from_numpy(x).cuda() for x in d]
    B_t = torch.from_numpy(gaussian_block(n, s, seed=0)).cuda()
    Xs_t = torch.from_numpy(gaussian_block(n, s, seed=1) * 0.1).cuda()

    def step():
        pe_t = torch.tensor(pe0, dtype=torch.float64, device="cuda", requires_grad=True)
        vals = base_t + pe_t[0] * d_t[0] + pe_t[1] * d_t[1] + pe_t[2] * d_t[2]
        X = krylov_solve(vals, B_t, op, "egl_bicg", 1e-8, 4000)
        L = torch.sum(torch.abs(X - Xs_t) ** 2)
        L.backward()
        return float(L.item()), pe_t.grad.cpu().numpy()

    step()
    times = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L, g = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    # the three phases, each bracketed by CUDA events
    kr.kr_op_update_values(op, vals0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    X, fi = kr.kr_solve(op, "egl_bicg", B_t, tol=1e-8, maxit=4000)
    ev[1].record()
    G = (2 * (X - Xs_t)).contiguous()
    Lam, ai = kr.kr_adjoint_solve(op, "egl_bicg", G, tol=1e-8, maxit=4000)
    ev[2].record()
    kr.kr_grad_values(op, Lam, X)
    ev[3].record()
    torch.cuda.synchronize()
    phases = {"forward_ms": ev[0].elapsed_time(ev[1]), "adjoint_ms": ev[1].elapsed_time(ev[2]),
              "grad_values_ms": ev[2].elapsed_time(ev[3])}

    def loss(pe):
        kr.kr_op_update_values(op, base + sum(pe[a] * d[a] for a in range(3)))
        Xp, info = kr.kr_solve(op, "egl_bicg", B_t, tol=1e-13, maxit=4000)
        return float(torch.sum(torch.abs(Xp - Xs_t) ** 2).item()), info.relres_true

    h, fd, fd_res = 1e-6, [], []
    for a in range(3):
        pp, pm = list(pe0), list(pe0)
        pp[a] += h
        pm[a] -= h
        (lp, rp_), (lm, rm_) = loss(pp), loss(pm)
        fd.append((lp - lm) / (2 * h))
        fd_res.append(max(rp_, rm_))
    fd = np.array(fd)
    out = {"mode": "config5",
           "workload": "3D convection-diffusion %d^3 (n=%d), learnable Peclet numbers %s, shift 0.05i, s=%d Gaussian RHS, "
                       "loss ||X - X*||_F^2; forward eGl-BiCG + adjoint eGl-BiCG + gradient on the pattern, tol 1e-8"
                       % (N, n, list(pe0), s),
           "step_ms_median": 1000 * statistics.median(times), "step_ms_all": [1000 * t for t in times],
           "phases": phases, "forward_iters": fi.iters, "adjoint_iters": ai.iters,
           "forward_status": fi.status, "adjoint_status": ai.status, "loss": L,
           "grad_pe": g.tolist(), "fd_grad_pe": fd.tolist(), "fd_solve_relres_max": max(fd_res),
           "grad_rel_err_vs_fd": float(np.max(np.abs(g - fd)) / np.max(np.abs(fd)))}
    if cpu is not None:
        t_it = cpu["per_method"]["egl_bicg"]["s_per_iter"]
        out["oracle"] = {"s_per_iter": t_it, "cpu_model": cpu["cpu_model"], "cores": 1,
                         "projected_step_s": t_it * (fi.iters + ai.iters),
                         "note": "projection: oracle eGl-BiCG seconds per iteration on this matrix (5 timed "
                                 "iterations) x the GPU's forward + adjoint iteration counts; the adjoint's A^H "
                                 "product costs what A's does"}
        out["speedup_vs_oracle_projection"] = out["oracle"]["projected_step_s"] / (out["step_ms_median"] / 1000)
    print(json.dumps(out))
    op.close()


def main():
    args = parse_args()
    if args.cpu_sample_worker:
        cpu_sample_worker(args)
        return
    if args.ilu:
        ilu_mode(args)
        return
    if args.config1:
        config1(args)
        return
    if args.config3:
        config3(args)
        return
    if args.config4:
        config4(args)
        return
    if args.spmm_rates:
        spmm_rates(args)
        return
    if args.config5:
        config5(args)
        return
    if args.config2_sweep:
        config2_sweep(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
