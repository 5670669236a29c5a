#!/usr/bin/env python
"""Throughput of the batched implicit Elder time step on GB300.

Workload: the batched qMC ensemble at 64x64x16 cells (71,825 nodes, 143,650
unknowns per sample), 256 samples of scrambled-Sobol porosity fields
phi = 0.1*(1 + 0.3*(xi1 cos(pi x/600) + xi2 cos(pi y/600) + xi3 sin(2 pi
z/150))/3) with normalised Kozeny-Carman permeability, dt = 1/12 yr, mixed
precision (bfloat16 multigrid matrices, FP32 Krylov operator and vectors
inside FP64 Newton with FP64 residual and inner products).  One bench step =
one implicit Euler step of every sample (elder_step_predicted: Newton from
the quadratic extrapolation of the last states; --predictor 0 uses
elder_step) plus the ensemble moments of that step (elder_moments).
Metric: sample-timesteps/s, higher is better.

Timed window: the K timed steps are steps 1..K of the run from the initial
state (t = 0); the W warm-up steps (autotuning, CUDA-graph capture) run on a
discarded copy of the initial state first.  Beside it the line carries the
whole 60-step run of the configuration from t = 0 (`full_run`) and the FP64
solver over the same steps 1..K with the same Newton start (`fp64_path`).

Under torchrun each rank takes its own 256 samples (weak scaling, no
data-path collective); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one implicit step of several samples, one per
worker process, per bench step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample-timesteps/s at 64x64x16 batched (mixed vs FP64); GMG HBM GB/s vs peak"
UNIT = "sample-timesteps/s"
YEAR = 365.25 * 86400.0
FP64_NOMINAL_GFLOPS = 1250.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--grid", type=int, nargs=3, default=[64, 64, 16])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-workers", type=int, default=0)
    ap.add_argument("--fields", choices=["sobol", "paper3rv"], default="sobol",
                    help="sobol: the cosine porosity field at scrambled-Sobol points; paper3rv: "
                         "the paper's parallelepiped field at Halton points")
    ap.add_argument("--dt-yr", type=float, default=1.0 / 12.0)
    ap.add_argument("--no-gpc", action="store_true", help="skip the gPC kernel timings")
    ap.add_argument("--gpc-only", action="store_true",
                    help="time only the gPC surrogate kernels (projection, exceedance) and exit")
    ap.add_argument("--gpc-samples", type=int, default=1_000_000,
                    help="surrogate sample points per node of the exceedance timing")
    ap.add_argument("--smoother", choices=["jacobi", "zline", "ilu"], default="zline",
                    help="multigrid smoother: point block Jacobi, z-line block Jacobi, or the "
                         "multicolour block ILU(0)")
    ap.add_argument("--predictor", type=int, choices=[0, 1, 2], default=2,
                    help="Newton's starting point: 0 u^n (elder_step), 1 2u^n - u^{n-1}, "
                         "2 3u^n - 3u^{n-1} + u^{n-2} (elder_step_predicted)")
    ap.add_argument("--no-extrapolate", action="store_true", help="the same as --predictor 0")
    ap.add_argument("--graphs", type=int, choices=[0, 1, 2], default=2,
                    help="0: every kernel launched from the host; 1: the BiCGStab iteration "
                         "replayed as a CUDA graph, the host polling convergence flags; 2: the "
                         "whole step one graph with device-driven Newton/Krylov/line-search "
                         "loops (conditional while nodes)")
    ap.add_argument("--no-graphs", action="store_true", help="the same as --graphs 0")
    ap.add_argument("--profile-steps", type=int, default=1,
                    help="steps of the profiled pass (per-kernel-class CUDA events)")
    ap.add_argument("--workload", choices=["qmc", "uneven", "config2", "fingers"], default="qmc",
                    help="qmc: the batched 64x64x16 ensemble (the headline); uneven: 48 samples "
                         "at 128x128x32 plus 16 at 256x256x64, dt = 1/24 yr, one context per grid "
                         "size, samples shared out longest-processing-time first across ranks; "
                         "config2: one sample at 128x128x32 for --run-steps steps with the FP64 "
                         "and the mixed solver, their states compared along the run; "
                         "fingers: the paper's parallelepiped ensemble (3 random variables, "
                         "Halton points, 128x128x32, dt = 0.005 yr, the paper's boundary sets) "
                         "marched 1500 steps to 7.5 yr, with the plume lobes of the mean's 0.5 "
                         "level set counted")
    ap.add_argument("--fingers-samples", type=int, default=200)
    ap.add_argument("--fingers-method", choices=["qmc", "gpc"], default="qmc",
                    help="qmc: the Halton ensemble's sample moments; gpc: the 125 points of "
                         "the 5^3 Gauss-Legendre rule, the moments of the order-4 gPC "
                         "surrogate projected from them (Section 3, Section 5.3)")
    ap.add_argument("--fingers-grid", type=int, nargs=3, default=[128, 128, 32])
    ap.add_argument("--fingers-dt-yr", type=float, default=0.005)
    ap.add_argument("--fingers-steps", type=int, default=1500)
    ap.add_argument("--fingers-snap", type=int, default=300,
                    help="steps between the moment snapshots of the fingers workload")
    ap.add_argument("--fingers-compare", nargs=2, metavar=("A.npz", "B.npz"), default=None,
                    help="compare the fields of two --fingers-out files (e.g. QMC against gPC) "
                         "and exit: mean differences per snapshot, lobe counts, variance level "
                         "sets at 0.05")
    ap.add_argument("--fingers-out", default="",
                    help="npz file for the fingers workload's mean and variance fields")
    ap.add_argument("--run-steps", type=int, default=60,
                    help="steps of the configuration's whole run from t = 0, timed beside the "
                         "K bench steps (0: skip)")
    a = ap.parse_args()
    if a.no_extrapolate:
        a.predictor = 0
    if a.no_graphs:
        a.graphs = 0
    return a


def workload_config(a):
    nx, ny, nz = a.grid
    fields = ("scrambled Sobol (torch SobolEngine seed 0) -> phi (cosine field), Kozeny-Carman K"
              if a.fields == "sobol" else
              "Halton points (bases 2,3,5) -> the paper's parallelepiped porosity field, "
              "Kozeny-Carman K")
    tag = "qmc" if a.fields == "sobol" else "paper3rv-halton"
    return {
        "workload": f"elder3d-box-{nx}x{ny}x{nz}-{tag}{a.samples}",
        "grid_cells": [nx, ny, nz],
        "nodes_per_sample": (nx + 1) * (ny + 1) * (nz + 1),
        "samples_per_gpu": a.samples,
        "dt_yr": a.dt_yr,
        "precision": a.precision,
        "smoother": a.smoother,
        "solver": "inexact Newton (Krylov rtol 1e-2), BiCGStab + V(1,0) multigrid, " +
                  {"zline": "z-line damping 0.95", "jacobi": "point block Jacobi damping 0.5",
                   "ilu": "multicolour block ILU(0), undamped"}[a.smoother],
        "newton_start": ["u^n", "2u^n - u^(n-1)", "3u^n - 3u^(n-1) + u^(n-2)"][a.predictor],
        "fields": fields,
        "l2": "no flush: per-step working set (Jacobians of all levels, vectors) ~10 GB >> 129 MB L2",
        "parallelism": f"samples sharded, dp{a.gpus}",
        "timed_steps": f"1-{a.steps} of the run from t = 0 (warm-up on a discarded copy)",
        "precision_detail": ("FP64 Newton residual, inner products and state; FP32 Krylov vectors "
                             "and level-0 Krylov operator; bfloat16 multigrid matrices"
                             if a.precision == "mixed" else "FP64 throughout"),
    }


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            # a temporary file, removed once read
            fd, self.path = tempfile.mkstemp(prefix="elder_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path:
                self.f.close()
                os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores
# --------------------------------------------------------------------------

def _oracle_one_step(args):
    nx, ny, nz, xi = args
    import numpy as np  # noqa: F401
    import oracle as O
    P = O.Problem(nx, ny, nz)
    phi, K = O.fields_sobol(P, xi)
    p, c = O.initial_state(P)
    t = time.perf_counter()
    p, c, info = O.newton_step(P, phi, K, p, c, YEAR / 12)
    return time.perf_counter() - t, info["status"]


def cpu_baseline(a, workers=None):
    import multiprocessing as mp
    from paper_1906_01632_gb300 import inputs as I
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    workers = workers or a.cpu_workers or min(16, nproc)
    xi = I.sobol_xi(workers)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_one_step, [(a.grid[0], a.grid[1], a.grid[2], xi[i]) for i in range(workers)])
    wall = time.perf_counter() - t0
    return {"value": workers / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} samples x 1 implicit step (first step from t=0) at "
                      f"{a.grid[0]}x{a.grid[1]}x{a.grid[2]}, one sample per process, wall {wall:.1f} s",
            "per_sample_step_s": [round(r[0], 2) for r in res]}


def run_reference(a):
    """The oracle as it stands on the host cores, on the GPU arm's workload:
    the K timed steps are sample-steps (the first implicit step of one Sobol
    sample at the bench grid, the hardest of the run), rounded up to whole
    rounds of one per worker process (one worker per host core, at most 16)
    and timed together on the wall clock; the W warm-up steps run first on
    the same pool at 8x8x2 (process start-up and library load stay outside
    the timed region).  value = sample-steps / wall."""
    import multiprocessing as mp
    from paper_1906_01632_gb300 import inputs as I
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    cfg = workload_config(a)
    # the same workload; the solver keys describe the oracle's own method
    cfg["precision"] = "fp64"
    cfg["smoother"] = "block Jacobi (oracle)"
    cfg["solver"] = ("Newton (tolerance 1e-12) with dense LU up to 1200 unknowns, else BiCGStab + "
                     "damped block-Jacobi V(1,1) multigrid (oracle)")
    cfg["newton_start"] = "u^n"
    nproc = os.cpu_count() or 1
    workers = a.cpu_workers or min(16, nproc)
    K = max(1, a.steps)
    # whole rounds of one sample-step per worker, so that no core idles
    n = workers * (-(-K // workers))
    xi = I.sobol_xi(n)
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_oracle_one_step, [(8, 8, 2, xi[i % n]) for i in range(max(a.warmup, 1) * workers)],
                 chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_oracle_one_step, [(a.grid[0], a.grid[1], a.grid[2], xi[i]) for i in range(n)],
                       chunksize=1)
        wall = time.perf_counter() - t0
    value = n / wall
    sample = (f"{n} sample-steps (the first implicit step of {n} Sobol samples from t = 0) at "
              f"{a.grid[0]}x{a.grid[1]}x{a.grid[2]} on {workers} worker processes, wall {wall:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": K, "warmup": a.warmup, "ms_per_step": 1000.0 * wall / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": sample,
                             "per_sample_step_s": [round(r[0], 2) for r in res]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the CUDA path
# --------------------------------------------------------------------------

def alu_peaks(E):
    """FMA peaks of this GPU measured by the library's FMA-chain probe
    (elder_measure_peak), with the nominal figures as fallback."""
    out = {}
    for kind, nominal in (("fp64", FP64_NOMINAL_GFLOPS), ("fp32", FP32_NOMINAL_GFLOPS)):
        try:
            out[kind] = (E.elder_measure_peak(kind), f"measured {kind.upper()} FMA-chain probe "
                         "(elder_measure_peak)")
        except Exception as ex:  # noqa: BLE001
            out[kind] = (nominal, f"nominal {kind.upper()} ({ex})")
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def ncu_traffic(kernel_class: str, precision: str):
    """DRAM bytes per node and sample of one launch from the committed ncu
    summary (profiles/*.md lines 'traffic_bytes_per_node <class> <precision> <value>')."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for f in sorted(os.listdir(d)):
        if not f.endswith(".md"):
            continue
        for line in open(os.path.join(d, f)):
            parts = line.strip().strip("`").split()
            if len(parts) == 4 and parts[0] == "traffic_bytes_per_node" and parts[1] == kernel_class \
                    and parts[2] == precision:
                return float(parts[3])
    return None


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1906_01632_gb300 import build as B
    B.build()
    from paper_1906_01632_gb300 import elder as E
    from paper_1906_01632_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    nx, ny, nz = a.grid
    S = a.samples
    dt = YEAR * a.dt_yr
    prec = E.ELDER_MIXED if a.precision == "mixed" else E.ELDER_FP64
    smoother = {"zline": E.ELDER_SMOOTH_ZLINE, "jacobi": E.ELDER_SMOOTH_JACOBI,
                "ilu": E.ELDER_SMOOTH_ILU}[a.smoother]
    ctx = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S, precision=prec,
                                                smoother=smoother,
                                                use_graphs=a.graphs))
    N, C = ctx.N, ctx.C
    xi_all = I.sobol_xi(S * world, seed=0) if a.fields == "sobol" else I.halton_xi(S * world)
    xi = torch.tensor(xi_all[rank * S:(rank + 1) * S].ravel(), dtype=torch.float64, device=dev)
    phi, K = ctx.fields(S, 0 if a.fields == "sobol" else 2, xi)
    p, c = ctx.initial_state(S, device=dev)
    stream = torch.cuda.current_stream()

    if a.gpc_only:
        if rank == 0:
            print(json.dumps({"metric": "gPC surrogate kernel timings", "config": {
                "workload": f"gpc-{nx}x{ny}x{nz}", "grid_cells": [nx, ny, nz]},
                "gpc": gpc_timings(E, torch, c.reshape(S, N), stream, a.gpc_samples)}))
        ctx.destroy()
        return

    # history levels (u^{n-1}[, u^{n-2}]) of the extrapolated Newton start,
    # u^n in every level on the first step
    order = a.predictor
    p_init, c_init = p, c

    def fresh():
        """The initial state (t = 0) and its history levels, as new tensors."""
        return (p_init.clone(), c_init.clone(), p_init.repeat(max(order, 1)),
                c_init.repeat(max(order, 1)))

    def bench_step(ctx_, state):
        p_, c_, ph_, ch_ = state
        if order == 0:
            st, info = ctx_.step(S, phi, K, p_, c_, dt)
        else:
            st, info = ctx_.step_predicted(S, phi, K, order, ph_, ch_, p_, c_, dt)
        mom = ctx_.moments(S, c_)
        return st, info, mom

    def timed_run(ctx_, steps, log=None):
        """steps bench steps from t = 0 between CUDA events on the launching
        stream; returns (ms, final state)."""
        state = fresh()
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            st, info, _ = bench_step(ctx_, state)
            if log is not None:
                log.append((st, info))
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return t0.elapsed_time(t1), state

    # warm-up (autotuning, CUDA-graph capture) on a discarded copy of t = 0
    warm = fresh()
    for _ in range(a.warmup):
        bench_step(ctx, warm)
    del warm
    torch.cuda.synchronize()

    # ---- device-timed region: steps 1..K from t = 0 -------------------------
    # (no per-launch events here: they force a host synchronisation per Krylov
    # iteration and bypass the captured CUDA graphs; the per-kernel-class
    # events are taken in a separate profiled pass right after)
    clocks = Clocks(local)
    clocks.start()
    l0 = E.elder_launch_count()
    log = []
    # the ncu launch list is taken with --profile-from-start off: only the
    # timed steps are captured
    torch.cuda.profiler.start()
    ms, state = timed_run(ctx, a.steps, log)
    torch.cuda.profiler.stop()
    launches = E.elder_launch_count() - l0
    clk = clocks.stop()
    fails = sum(int((st != 0).sum()) for st, _ in log)
    retries = sum(1 for _, info in log for x in info if x["fp64_retry"])
    newton = [np.mean([x["newton_iters"] for x in info]) for _, info in log]
    krylov = [np.mean([x["krylov_iters"] for x in info]) for _, info in log]
    p, c, p_hist, c_hist = state
    c_mixed_K = c.clone()

    # ---- profiled pass: CUDA events around every launch of the stencil,
    # residual and assembly kernel classes, on the launching stream ----------
    ctx.profile(True)
    torch.cuda.synchronize()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(a.profile_steps):  # continues the run: steps K+1, ...
        bench_step(ctx, state)
    q1.record(stream)
    torch.cuda.synchronize()
    prof_step_ms = q0.elapsed_time(q1) / max(a.profile_steps, 1)
    ctx.profile(False)
    prof = {E.KERNEL_CLASSES[k]: ctx.profile_read(k) for k in E.KERNEL_CLASSES}
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = S * world * a.steps / (ms / 1000.0)

    # ---- roofline of the dominant kernel class ------------------------------
    top = max(prof, key=lambda k: prof[k]["ms"])
    pk = prof[top]
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    tsize = 4 if a.precision == "mixed" else 8
    per_launch_ms = pk["ms"] / max(pk["launches"], 1)
    bytes_per_launch = pk["bytes"] / max(pk["launches"], 1)
    tr = ncu_traffic(top, a.precision)
    apk = alu_peaks(E)
    alu = apk["fp64"]
    if top == "residual" or (top == "jacobian" and a.precision == "fp64"):
        # FP64-ALU bound (FP64 pipe ~85% busy under ncu): rated against the
        # FP64 FMA peak measured on this GPU
        achieved = (pk["flops"] / 1e9) / (pk["ms"] / 1e3) if pk["ms"] > 0 else None
        bound, peak, unit = "alu", alu[0], "GFLOP/s"
        src = alu[1] + "; flops from the per-node model"
    else:
        achieved = (pk["bytes"] / 1e9) / (pk["ms"] / 1e3) if pk["ms"] > 0 else None
        bound, peak, unit = "hbm", hbm_peak, "GB/s"
        src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
    roofline = {"kernel": top, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak if achieved else None,
                "peak_source": src,
                "traffic": (tr * bytes_per_launch /
                            max(1e-30, E_model_bytes(top, tsize, nx, ny, nz,
                                                     a.smoother != "jacobi",
                                                     ilu=a.smoother == "ilu"))
                            if tr is not None else None),
                "algorithmic_flops_per_launch": pk["flops"] / max(pk["launches"], 1),
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": per_launch_ms,
                "launches": pk["launches"]}
    classes = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share": round(v["ms"] / (prof_step_ms * a.profile_steps), 4)
                   if prof_step_ms else None,
                   "GB/s": round((v["bytes"] / 1e9) / (v["ms"] / 1e3), 1) if v["ms"] > 0 else None,
                   "GFLOP/s": round((v["flops"] / 1e9) / (v["ms"] / 1e3), 1) if v["ms"] > 0 else None}
               for k, v in prof.items()}
    for k, v in classes.items():  # fraction of the class's own bound
        if k == "residual":
            v["bound"], v["frac"] = "fp64 alu", (v["GFLOP/s"] / alu[0] if v["GFLOP/s"] else None)
        else:
            v["bound"], v["frac"] = "hbm", (v["GB/s"] / hbm_peak if v["GB/s"] else None)

    # ---- the configuration's whole run from t = 0 -----------------------------
    full_run = None
    if a.run_steps > 0:
        if a.run_steps == a.steps:
            ms_run = ms
        else:
            ms_run, _ = timed_run(ctx, a.run_steps)
            if world > 1:
                t = torch.tensor([ms_run], dtype=torch.float64, device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ms_run = float(t.item())
        full_run = {"value": S * world * a.run_steps / (ms_run / 1000.0), "unit": UNIT,
                    "steps": f"1-{a.run_steps} from t = 0", "ms": ms_run,
                    "timing": "CUDA events on the launching stream, as value"}

    # ---- end to end through host buffers: steps 1..K from t = 0 ---------------
    e2e = None
    if not a.no_e2e:
        barrier()
        el, _, hc_end = e2e_pipeline(torch, ctx, S, N, C, order, dt, a.steps, p_init, c_init,
                                     phi, K, dev)
        # the same steps through the device-resident run: the same state
        e2e_dc = float((hc_end.to(dev) - c_mixed_K).abs().max())
        if world > 1:
            t = torch.tensor([el], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": S * world * a.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": 8 * S * ((2 + 2 * order) * N + 2 * C),
               "d2h_bytes_per_step": 8 * (S * 2 * N + 3 * N),
               "steps": f"1-{a.steps} from t = 0", "timing": "host wall clock (perf_counter)",
               "copies": "history levels and fields of the next step on a side stream during "
                         "the step; the state in, the result out on the launching stream",
               "max_abs_dc_vs_device_run": e2e_dc}

    # ---- FP64 solver over the same steps 1..K, same Newton start -------------
    fp64 = None
    if not a.no_fp64 and a.precision == "mixed":
        ctx64 = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S,
                                                      precision=E.ELDER_FP64, smoother=smoother))
        warm = fresh()
        bench_step(ctx64, warm)  # warm-up (autotuning, graph capture) on a discarded copy
        del warm
        log64 = []
        ms64, state64 = timed_run(ctx64, a.steps, log64)
        if world > 1:
            t = torch.tensor([ms64], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms64 = float(t.item())
        diff = float((state64[1] - c_mixed_K).abs().max().item())
        fp64 = {"value": S * world * a.steps / (ms64 / 1000.0), "unit": UNIT,
                "steps": f"1-{a.steps} from t = 0", "ms_per_step": ms64 / a.steps,
                "newton_start": workload_config(a)["newton_start"],
                "newton_per_step": float(np.mean([np.mean([x["newton_iters"] for x in info])
                                                  for _, info in log64])),
                "krylov_per_step": float(np.mean([np.mean([x["krylov_iters"] for x in info])
                                                  for _, info in log64])),
                "mixed_vs_fp64_max_abs_c_after_K_steps": diff,
                "mixed_speedup": (S * world * a.steps / (ms / 1000.0)) /
                                 (S * world * a.steps / (ms64 / 1000.0))}
        ctx64.destroy()

    gpc = None
    if rank == 0 and not a.no_gpc and S >= 1:
        gpc = gpc_timings(E, torch, c.reshape(S, N), stream, a.gpc_samples, apk)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32+bf16" if a.precision == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(a), "clocks": clk,
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
                "full_run": full_run, "fp64_path": fp64, "gpc": gpc, "kernel_classes": classes,
                "iterations": {"newton_per_step": float(np.mean(newton)),
                               "krylov_per_step": float(np.mean(krylov)), "failed_samples": fails,
                               "fp64_retries": retries},
                "profiled_pass": {"steps": a.profile_steps, "ms_per_step": prof_step_ms},
                "autotune": {"threads_per_block": ctx.autotune_result()["threads_per_block"],
                             "mg_residual (threads, samples per CTA, ms of candidates)":
                                 ctx.autotune_choice(E.K_MGRES),
                             "zline_sweep (threads, samples per CTA, ms of candidates)":
                                 ctx.autotune_choice(E.K_SMOOTH0)},
                "timing": "value: CUDA events on the launching stream around the K timed steps "
                          "(graphs replayed, no per-launch events); kernel_classes and roofline: "
                          "CUDA events around every launch of each class in a profiled pass of "
                          "the same workload right after the timed steps (graph replay bypassed "
                          "and the host synchronised per Krylov iteration there, so its step time "
                          "is longer)"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.07  # SMs x FP32 lanes x FMA x max SM clock (GHz)


def e2e_pipeline(torch, ctx, S, N, C, order, dt, steps, p_init, c_init, phi, K, dev,
                 arena=True):
    """Steps 1..steps from t = 0 through host buffers, timed on the host wall
    clock: every step copies its inputs (state u^n, the history levels
    u^{n-1}[, u^{n-2}] of the Newton start, phi and K) from pinned host memory
    and reads its result (u^{n+1} and the three moment fields) back.  The host
    keeps the states in a ring of order + 1 pinned buffers (u^m in slot m mod
    (order + 1)).  The history levels and fields of step n+1 do not depend on
    step n's result, so a side stream copies them into the second of two
    device buffer sets while step n runs (after step n's own state copy,
    with which it would share the host link); the state u^n comes in on the
    launching stream right before its step.  Two untimed steps first capture
    the step graphs of both buffer sets.  Returns the elapsed seconds and the
    final state (host)."""
    R = max(order, 0) + 1
    f64 = torch.float64
    sizes = [S * N] * (2 * R) + [S * C, S * C, 3 * N]
    if arena:  # all host buffers as views of one pinned allocation
        pool = torch.empty(sum(sizes), dtype=f64, pin_memory=True)
        bufs = list(torch.split(pool, sizes))
    else:
        bufs = [torch.empty(n, dtype=f64, pin_memory=True) for n in sizes]
    hp, hc = bufs[:R], bufs[R:2 * R]
    hphi, hK, hmom = bufs[2 * R:]
    for q in range(R):
        hp[q].copy_(p_init)
        hc[q].copy_(c_init)
    hphi.copy_(phi)
    hK.copy_(K)
    dp_ = torch.empty(S * N, dtype=f64, device=dev)
    dc_ = torch.empty_like(dp_)
    lv = max(order, 1)
    sets = [{"ph": torch.empty(lv * S * N, dtype=f64, device=dev),
             "ch": torch.empty(lv * S * N, dtype=f64, device=dev),
             "phi": torch.empty(S * C, dtype=f64, device=dev),
             "K": torch.empty(S * C, dtype=f64, device=dev)} for _ in range(2)]
    main = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    landed = torch.cuda.Event()
    state_in = torch.cuda.Event()
    for e in free:
        e.record(main)
    landed.record(main)
    state_in.record(main)

    def prefetch(n, X):
        with torch.cuda.stream(side):
            side.wait_event(free[X])      # the step that used set X is done
            side.wait_event(landed)       # u^n is in its host slot
            # after the current step's state copies: both directions share the
            # host link, so a concurrent prefetch would only delay the step
            side.wait_event(state_in)
            for q in range(order):        # level q holds u^{n-1-q}
                sets[X]["ph"][q * S * N:(q + 1) * S * N].copy_(hp[(n - 1 - q) % R],
                                                               non_blocking=True)
                sets[X]["ch"][q * S * N:(q + 1) * S * N].copy_(hc[(n - 1 - q) % R],
                                                               non_blocking=True)
            sets[X]["phi"].copy_(hphi, non_blocking=True)
            sets[X]["K"].copy_(hK, non_blocking=True)
            ready[X].record(side)

    def run(nsteps):
        for q in range(R):
            hp[q].copy_(p_init)
            hc[q].copy_(c_init)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prefetch(0, 0)
        for n in range(nsteps):
            X = n % 2
            main.wait_event(ready[X])
            dp_.copy_(hp[n % R], non_blocking=True)
            dc_.copy_(hc[n % R], non_blocking=True)
            state_in.record(main)
            if n + 1 < nsteps:
                prefetch(n + 1, 1 - X)
            st_ = sets[X]
            if order == 0:
                ctx.step(S, st_["phi"], st_["K"], dp_, dc_, dt)
            else:
                ctx.step_predicted(S, st_["phi"], st_["K"], order, st_["ph"], st_["ch"], dp_,
                                   dc_, dt)
            free[X].record(main)
            m, v, pe = ctx.moments(S, dc_, stream=main)
            hp[(n + 1) % R].copy_(dp_, non_blocking=True)
            hc[(n + 1) % R].copy_(dc_, non_blocking=True)
            hmom[:N].copy_(m, non_blocking=True)
            hmom[N:2 * N].copy_(v, non_blocking=True)
            hmom[2 * N:].copy_(pe, non_blocking=True)
            landed.record(main)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # untimed: two steps from t = 0, so that the step graphs of both buffer
    # sets are captured before the timed steps (as in the device-timed run)
    run(min(2, steps))
    el = run(steps)
    return el, hp[steps % R], hc[steps % R]


def gpc_timings(E, torch, cfield, stream, Ns=1_000_000, apk=None):
    """Kernel timings of the gPC surrogate (Section 3) on this GPU: FP64
    projection of 125 fields (the 5^3 Gauss-Legendre points, total degree
    <= 4, 35 terms) onto every node, and the FP32 surrogate evaluated
    at Ns (default 10^6) uniform points per node for P(c > 0.5).  The bench's current
    concentration fields stand in for the quadrature-point fields (the
    kernels' cost does not depend on the values)."""
    S, N = cfield.shape
    apk = apk or alu_peaks(E)
    M, p, q = 3, 4, 5
    x, w1 = E.elder_gauss_legendre(q)
    import numpy as np
    g = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)[:, ::-1].copy()
    wq = np.prod(np.stack(np.meshgrid(w1, w1, w1, indexing="ij"), -1).reshape(-1, 3), 1)
    Nq = q ** M
    dev = cfield.device
    beta = torch.tensor(E.elder_gpc_indices(M, p), device=dev)
    T = beta.shape[0]
    theta_q = torch.tensor(g, dtype=torch.float64, device=dev)
    wt = torch.tensor(wq, dtype=torch.float64, device=dev)
    u = cfield[torch.arange(Nq, device=dev) % S].contiguous()
    gen = torch.Generator(device=dev).manual_seed(5)
    theta_s = (torch.rand(Ns, M, generator=gen, dtype=torch.float64, device=dev) * 2 - 1).contiguous()
    coef, mean, var = E.elder_gpc_project(beta, theta_q, wt, u)
    out = E.elder_gpc_exceed(beta, coef, theta_s, 0.5, engine="tensor")
    out32 = E.elder_gpc_exceed(beta, coef, theta_s, 0.5, engine="fp32")
    torch.cuda.synchronize()
    # the two engines' counts differ only for samples inside the FP32 band
    engines_max_count_diff = int(((out - out32).abs() * Ns).round().max().item())
    # tensor-core rate: TF32 dense peak from the measured bf16 GEMM peak and
    # the nominal TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s); the product runs
    # over the stacked inner dimension 112 for 128-node tiles and 128-point
    # chunks
    peaks = measured_peaks()
    tf32_peak = (peaks["bf16_tflops"] * 1e3 if peaks else 1.9e6) * 1.1 / 2.25
    mma_flops = 2.0 * 112 * (-(-N // 128) * 128) * (-(-Ns // 128) * 128)
    res = {}
    for name, fn, flops, unit_peak in (
            ("project", lambda: E.elder_gpc_project(beta, theta_q, wt, u, coef, mean, var),
             2.0 * T * Nq * N, (apk["fp64"][1], apk["fp64"][0])),
            ("exceed", lambda: E.elder_gpc_exceed(beta, coef, theta_s, 0.5, out=out,
                                                  engine="tensor"),
             mma_flops, ("TF32 dense tensor peak: measured bf16 GEMM x 1.1/2.25", tf32_peak)),
            ("exceed_fp32", lambda: E.elder_gpc_exceed(beta, coef, theta_s, 0.5, out=out32,
                                                       engine="fp32"),
             2.0 * T * Ns * N, (apk["fp32"][1], apk["fp32"][0]))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gf = flops / 1e9 / (ms / 1e3)
        res[name] = {"ms": ms, "GFLOP/s": gf, "bound": "tensor" if name == "exceed" else "alu",
                     "peak_GFLOP/s": unit_peak[1], "peak_source": unit_peak[0],
                     "frac": gf / unit_peak[1]}
    res["exceed"]["fp32_equivalent_GFLOP/s"] = 2.0 * T * Ns * N / 1e9 / (res["exceed"]["ms"] / 1e3)
    res["exceed"]["engines_max_count_diff"] = engines_max_count_diff
    res["config"] = {"M": M, "order": p, "terms": T, "quadrature_points": Nq, "nodes": N,
                     "surrogate_samples": Ns,
                     "exceed": "tcgen05 TF32 split product (hi*hi + hi*lo + lo*hi), FLOPs of "
                               "the stacked product (inner dimension 112); exceed_fp32: the "
                               "CUDA-core FP32 engine, FLOPs 2 T per node and point"}
    return res


def E_model_bytes(cls, tsize, nx, ny, nz, line=True, ilu=False):
    """Algorithmic bytes per node of one launch (mirrors the library's model);
    the mixed path stores the multigrid matrices in bfloat16.  With the z-line
    smoother the sweep from x = 0 reads the assembly's line factors (zMi, zC),
    the lower line block, b and writes x; the assembly also forms those
    factors (reading Dinv and both line blocks).  With the ILU smoother
    (ilu=True) the sweep from x = 0 reads the 26 factor blocks, the inverse
    pivot, b and bc twice, writes, reads and rewrites its scratch vector and
    writes x; the assembly also forms the factors (J, Dinv, bc read; 26
    factor blocks and the inverse pivot written)."""
    N = (nx + 1) * (ny + 1) * (nz + 1)
    cpn = nx * ny * nz / N
    mz = 2 if tsize == 4 else 8
    smooth0 = (12 * tsize + 4 * mz + 1) if line else 8 * tsize + 1
    if ilu:
        smooth0 = 104 * mz + 14 * tsize + 2
    return {"smooth": 108 * mz + 10 * tsize + 1,
            "smooth0": smooth0,
            "spmv": 108 * tsize + 6 * tsize + 1, "mg_residual": 108 * mz + 6 * tsize + 1,
            "residual": 49 + 16 * cpn,
            "jacobian": 108 * tsize + 108 * mz + 4 * tsize + 17 + 16 * cpn +
                        ((12 * tsize + 8 * mz + 1) if line else 0) +
                        ((212 * mz + 8 * tsize + 1) if ilu else 0)}[cls]


# --------------------------------------------------------------------------
# the uneven ensemble: two grid sizes in one run
# --------------------------------------------------------------------------

UNEVEN = ((128, 128, 32, 48), (256, 256, 64, 16))


def uneven_plan(world: int, rank: int, sizes=UNEVEN):
    """The samples of the uneven ensemble that ``rank`` owns, per grid size:
    {(nx, ny, nz): [global sample indices]}.  Samples are numbered in the
    order of ``sizes`` and shared out longest-processing-time first with a
    cost proportional to the sample's node count."""
    from paper_1906_01632_gb300.ensemble import lpt_assign
    grids = [(nx, ny, nz) for nx, ny, nz, count in sizes for _ in range(count)]
    costs = [(nx + 1) * (ny + 1) * (nz + 1) for nx, ny, nz in grids]
    mine = lpt_assign(costs, world)[rank]
    plan: dict = {}
    for i in mine:
        plan.setdefault(grids[i], []).append(i)
    return plan


def run_uneven(a):
    """Sample-timesteps/s of the uneven ensemble: 64 scrambled-Sobol samples
    (seed 0), the first 48 at 128x128x32 and the last 16 at 256x256x64,
    dt = 1/24 yr, mixed precision, Newton from the quadratic extrapolation.
    One context per grid size; each bench step advances every grid's batch
    by one implicit step (converged samples masked out within a batch).
    Steps 1..K from t = 0 are timed, after W warm-up steps on discarded
    copies of the initial state."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1906_01632_gb300 import build as B
    B.build()
    from paper_1906_01632_gb300 import elder as E
    from paper_1906_01632_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    total = sum(cnt for *_, cnt in UNEVEN)
    xi_all = I.sobol_xi(total, seed=0)
    dt = YEAR / 24.0
    order = a.predictor
    stream = torch.cuda.current_stream()
    runs = []
    for (nx, ny, nz), ids in sorted(uneven_plan(world, rank).items()):
        S = len(ids)
        ctx = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S,
                                                    precision=E.ELDER_MIXED))
        xi = torch.tensor(xi_all[ids].ravel(), dtype=torch.float64, device=dev)
        phi, K = ctx.fields(S, 0, xi)
        p0, c0 = ctx.initial_state(S, device=dev)
        runs.append({"grid": (nx, ny, nz), "S": S, "ctx": ctx, "phi": phi, "K": K,
                     "p0": p0, "c0": c0, "newton": [], "krylov": [], "fails": 0,
                     "retries": 0})

    def fresh(r):
        return (r["p0"].clone(), r["c0"].clone(), r["p0"].repeat(max(order, 1)),
                r["c0"].repeat(max(order, 1)))

    def step(r, state, log):
        p_, c_, ph_, ch_ = state
        if order == 0:
            st, info = r["ctx"].step(r["S"], r["phi"], r["K"], p_, c_, dt)
        else:
            st, info = r["ctx"].step_predicted(r["S"], r["phi"], r["K"], order, ph_, ch_, p_,
                                               c_, dt)
        if log:
            r["fails"] += int((st != 0).sum())
            r["retries"] += sum(1 for x in info if x["fp64_retry"])
            r["newton"].append(float(np.mean([x["newton_iters"] for x in info])))
            r["krylov"].append(float(np.mean([x["krylov_iters"] for x in info])))

    for r in runs:  # warm-up: autotuning and graph capture on discarded copies
        warm = fresh(r)
        for _ in range(a.warmup):
            step(r, warm, False)
    torch.cuda.synchronize()
    states = [fresh(r) for r in runs]
    clocks = Clocks(local)
    clocks.start()
    l0 = E.elder_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        for r, stt in zip(runs, states):
            step(r, stt, True)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = E.elder_launch_count() - l0
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = total * a.steps / (ms / 1000.0)
    per_grid = {f"{r['grid'][0]}x{r['grid'][1]}x{r['grid'][2]}": {
        "samples": r["S"], "nodes_per_sample": (r["grid"][0] + 1) * (r["grid"][1] + 1) *
        (r["grid"][2] + 1), "newton_per_step": float(np.mean(r["newton"])),
        "krylov_per_step": float(np.mean(r["krylov"])), "failed_samples": r["fails"],
        "fp64_retries": r["retries"], "autotune": r["ctx"].autotune_result()}
        for r in runs}
    if rank == 0:
        line = {"metric": "sample-timesteps/s, uneven ensemble 48 @ 128x128x32 + 16 @ 256x256x64",
                "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64+f32+bf16",
                "data": "synthetic",
                "config": {"workload": "elder3d-box-uneven-48x128x128x32+16x256x256x64-qmc64",
                           "dt_yr": 1.0 / 24.0, "precision": "mixed",
                           "newton_start": ["u^n", "2u^n - u^(n-1)",
                                            "3u^n - 3u^(n-1) + u^(n-2)"][order],
                           "fields": "scrambled Sobol (torch SobolEngine seed 0), first 48 "
                                     "points at 128x128x32, last 16 at 256x256x64",
                           "timed_steps": f"1-{a.steps} of the run from t = 0",
                           "schedule": "one context per grid size, batches stepped in turn "
                                       "on one stream; ranks get samples by LPT on node count",
                           "l2": "no flush: working set ~100 GB >> 129 MB L2",
                           "parallelism": f"samples sharded (LPT), dp{world}"},
                "clocks": clk, "gpu_launches": launches, "per_grid": per_grid,
                "timing": "CUDA events on the launching stream around the K timed steps"}
        print(json.dumps(line), flush=True)
    for r in runs:
        r["ctx"].destroy()
    if world > 1:
        dist.destroy_process_group()


def run_config2(a):
    """The paper's box mesh (128x128x32, 1,098,306 unknowns), one sample with
    phi = 0.1 and K = 4.845e-13, dt = 1/12 yr, --run-steps steps (default
    120) from t = 0 with the FP64 solver and with the mixed solver, each
    timed with CUDA events; along the run, max |c_mixed - c_fp64| and the
    salt masses of both runs.  Newton from the quadratic extrapolation."""
    import numpy as np
    import torch

    from paper_1906_01632_gb300 import build as B
    B.build()
    from paper_1906_01632_gb300 import elder as E

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nx, ny, nz = 128, 128, 32
    steps = a.run_steps or 120
    dt = YEAR / 12
    stream = torch.cuda.current_stream()
    runs = {}
    for name, prec in (("fp64", E.ELDER_FP64), ("mixed", E.ELDER_MIXED)):
        ctx = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=1, precision=prec))
        C = ctx.C
        phi = torch.full((C,), 0.1, dtype=torch.float64, device=dev)
        K = torch.full((C,), 4.845e-13, dtype=torch.float64, device=dev)
        p0, c0 = ctx.initial_state(1, device=dev)
        warm = (p0.clone(), c0.clone(), p0.repeat(2), c0.repeat(2))
        for _ in range(max(a.warmup, 2)):  # tuning and graph capture on a discarded copy
            ctx.step_predicted(1, phi, K, 2, warm[2], warm[3], warm[0], warm[1], dt)
        p, c, ph, ch = p0.clone(), c0.clone(), p0.repeat(2), c0.repeat(2)
        states, info_log, ms = [], [], 0.0
        for n in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, info = ctx.step_predicted(1, phi, K, 2, ph, ch, p, c, dt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            info_log.append(info[0])
            states.append(c.clone())
        runs[name] = {"ms": ms, "states": states, "info": info_log}
        ctx.destroy()
    drift = {}
    for n in (1, 2, 5, 10, 30, 60, steps):
        if n <= steps:
            d = float((runs["mixed"]["states"][n - 1] - runs["fp64"]["states"][n - 1]).abs().max())
            m64 = runs["fp64"]["info"][n - 1]["salt_mass"]
            m32 = runs["mixed"]["info"][n - 1]["salt_mass"]
            drift[str(n)] = {"max_abs_dc": d, "salt_mass_fp64": m64,
                             "salt_mass_rel_diff": abs(m32 - m64) / abs(m64)}
    line = {"metric": "sample-timesteps/s, 128x128x32 single sample, mixed vs FP64 solver",
            "value": steps / (runs["mixed"]["ms"] / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": max(a.warmup, 2), "higher_is_better": True,
            "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": "elder3d-box-128x128x32-single", "dt_yr": 1.0 / 12.0,
                       "fields": "phi = 0.1, K = 4.845e-13 (Table 1)",
                       "newton_start": "3u^n - 3u^(n-1) + u^(n-2)",
                       "timed_steps": f"1-{steps} from t = 0"},
            "fp64_value": steps / (runs["fp64"]["ms"] / 1000.0),
            "newton_per_step": {k: float(np.mean([i["newton_iters"] for i in r["info"]]))
                                for k, r in runs.items()},
            "krylov_per_step": {k: float(np.mean([i["krylov_iters"] for i in r["info"]]))
                                for k, r in runs.items()},
            "failed": {k: sum(1 for i in r["info"] if i["status"]) for k, r in runs.items()},
            "mixed_vs_fp64": drift,
            "timing": "CUDA events around each step on the launching stream"}
    print(json.dumps(line), flush=True)


def plume_lobes(mean, nx, ny, nz, Lx=600.0, Ly=600.0, Lz=150.0, level=0.5, min_nodes=4):
    """Plume lobes of the level set {mean = level} of a node field
    [nz+1][ny+1][nx+1] (x fastest, z up, the top plane k = nz).

    Plane cuts: for every node plane below the top, the 8-connected
    components of {mean > level} with at least min_nodes nodes.  The largest
    such count and the first plane from the top that reaches it are reported
    with the centroids [m] of its lobes, each labelled with the nearest of
    the source square's four corners and its centre.  Column depths: per node
    column the depth below the top of the lowest node above the level; the
    components of {depth >= depth_max / 2} are counted the same way."""
    import numpy as np
    from scipy import ndimage

    m = np.asarray(mean, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    conn = np.ones((3, 3), dtype=bool)
    refs = {"corner(-,-)": (Lx / 4, Ly / 4), "corner(+,-)": (3 * Lx / 4, Ly / 4),
            "corner(-,+)": (Lx / 4, 3 * Ly / 4), "corner(+,+)": (3 * Lx / 4, 3 * Ly / 4),
            "centre": (Lx / 2, Ly / 2)}

    def lobes(mask):
        lab, n = ndimage.label(mask, structure=conn)
        if n == 0:
            return lab, []
        sizes = np.bincount(lab.ravel(), minlength=n + 1)
        return lab, [i for i in range(1, n + 1) if sizes[i] >= min_nodes]

    counts, best = [], {"count": 0, "z_m": None, "lobes": []}
    for k in range(nz - 1, -1, -1):
        lab, keep = lobes(m[k] > level)
        counts.append(len(keep))
        if len(keep) > best["count"]:
            out = []
            for i in keep:
                cy, cx = ndimage.center_of_mass(lab == i)
                x, y = cx * hx, cy * hy
                near = min(refs, key=lambda r: (refs[r][0] - x) ** 2 + (refs[r][1] - y) ** 2)
                out.append({"x_m": round(x, 1), "y_m": round(y, 1), "nearest": near,
                            "nodes": int((lab == i).sum())})
            best = {"count": len(keep), "z_m": round(k * hz, 3), "lobes": out}
    above = m > level
    low = np.where(above.any(0), above.argmax(0), nz + 1)
    depth = np.where(low <= nz, (nz - low) * hz, 0.0)
    dmax = float(depth.max())
    _, ckeep = lobes(depth >= 0.5 * dmax) if dmax > 0 else (None, [])
    return {"plane_counts_top_down": counts, "max_plane_count": best["count"],
            "plane": best, "column_depth_max_m": round(dmax, 3),
            "column_lobes_half_depth": len(ckeep)}


def compare_fingers(path_a, path_b, var_level=0.05):
    """Compares two --fingers-out files of the same grid (Section 5.3 compares
    the QMC and the gPC moments): per common snapshot the largest and mean
    |mean_a - mean_b| and the number of nodes where the decision mean > 0.5
    differs; at the last snapshot the per-plane lobe counts of both means
    (plume_lobes) and the variance level sets {var > var_level}."""
    import numpy as np
    A, B = np.load(path_a), np.load(path_b)
    nx, ny, nz = (int(v) for v in A["grid"])
    assert [int(v) for v in B["grid"]] == [nx, ny, nz]
    snaps = sorted(int(k[5:]) for k in A.files if k.startswith("mean_") and k in B.files)
    out = {"snapshots": {}}
    for t in snaps:
        ma, mb = A[f"mean_{t}"].astype(np.float64), B[f"mean_{t}"].astype(np.float64)
        out["snapshots"][str(t)] = {"max_abs_dmean": float(np.abs(ma - mb).max()),
                                    "mean_abs_dmean": float(np.abs(ma - mb).mean()),
                                    "decision_differs": int(((ma > 0.5) != (mb > 0.5)).sum())}
    t = snaps[-1]
    la = plume_lobes(A[f"mean_{t}"], nx, ny, nz)
    lb = plume_lobes(B[f"mean_{t}"], nx, ny, nz)
    out["plane_counts_top_down"] = {"a": la["plane_counts_top_down"],
                                    "b": lb["plane_counts_top_down"]}
    out["column_depth_max_m"] = {"a": la["column_depth_max_m"], "b": lb["column_depth_max_m"]}
    if "var" in A.files and "var" in B.files:
        va, vb = A["var"] > var_level, B["var"] > var_level
        out["var_level_set"] = {"level": var_level, "a": int(va.sum()), "b": int(vb.sum()),
                                "both": int((va & vb).sum())}
    print(json.dumps(out), flush=True)
    return out


def run_fingers(a):
    """The paper's parallelepiped workload with three random variables
    (Section 5.3, eq. poro-paral3RVS): the porosity field at Halton points,
    Kozeny-Carman K, 128x128x32 cells, dt = 0.005 yr, the paper's boundary
    sets (Section 2.1: c = 1 on the top square, c = 0 on the rest of the top
    and on the bottom, p = 0 on the four top edges), mixed precision, Newton
    from the quadratic extrapolation, marched --fingers-steps steps (1500 =
    7.5 yr) from t = 0 and timed with CUDA events per step.  Every
    --fingers-snap steps the ensemble mean, variance and P(c > 0.5) are
    formed (elder_moments) and the plume lobes of the mean's 0.5 level set
    counted (plume_lobes); Section 5.3 reports five fingers at 7.5 yr, four at
    the corners and one at the centre.  With --fingers-method gpc the samples
    are the 125 points of the 5^3 Gauss-Legendre rule and the moments are the
    order-4 gPC surrogate's (elder_gpc_project; P(c > 0.5) from 10^5 uniform
    points, elder_gpc_exceed), the paper's second method for the same
    figure."""
    import numpy as np
    import torch

    from paper_1906_01632_gb300 import build as B
    B.build()
    from paper_1906_01632_gb300 import elder as E
    from paper_1906_01632_gb300 import inputs as I

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nx, ny, nz = a.fingers_grid
    S, steps, snap = a.fingers_samples, a.fingers_steps, max(1, a.fingers_snap)
    gpc = a.fingers_method == "gpc"
    if gpc:  # the 5^3 tensor Gauss-Legendre rule, total degree <= 4 (35 terms)
        xg, wg = E.elder_gauss_legendre(5)
        theta = np.stack(np.meshgrid(xg, xg, xg, indexing="ij"), -1).reshape(-1, 3)[:, ::-1]
        wq = np.prod(np.stack(np.meshgrid(wg, wg, wg, indexing="ij"), -1).reshape(-1, 3), 1)
        S = theta.shape[0]
        beta = torch.tensor(E.elder_gpc_indices(3, 4), device=dev)
        theta_t = torch.tensor(np.ascontiguousarray(theta), dtype=torch.float64, device=dev)
        wq_t = torch.tensor(wq, dtype=torch.float64, device=dev)
        gen = torch.Generator(device=dev).manual_seed(5)
        theta_s = (torch.rand(100_000, 3, generator=gen, dtype=torch.float64, device=dev) * 2
                   - 1).contiguous()
    dt = YEAR * a.fingers_dt_yr
    stream = torch.cuda.current_stream()
    ctx = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S,
                                                precision=E.ELDER_MIXED, bc_mode=1))
    N = ctx.N
    xi_np = np.ascontiguousarray(theta) if gpc else I.halton_xi(S)
    xi = torch.tensor(xi_np.ravel(), dtype=torch.float64, device=dev)
    phi, K = ctx.fields(S, 2, xi)
    p0, c0 = ctx.initial_state(S, device=dev)
    warm = [p0.clone(), c0.clone(), p0.repeat(2), c0.repeat(2)]
    for _ in range(max(a.warmup, 2)):  # tuning and graph capture on a discarded copy
        ctx.step_predicted(S, phi, K, 2, warm[2], warm[3], warm[0], warm[1], dt)
    del warm
    p, c, ph, ch = p0.clone(), c0.clone(), p0.repeat(2), c0.repeat(2)
    torch.cuda.synchronize()
    ms, newton, krylov, failed, retries = 0.0, 0, 0, 0, 0
    snaps, lob, fields = {}, {}, {}
    t_wall = time.time()
    for n in range(1, steps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = ctx.step_predicted(S, phi, K, 2, ph, ch, p, c, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        newton += sum(i["newton_iters"] for i in info)
        krylov += sum(i["krylov_iters"] for i in info)
        failed += int((st != 0).sum())
        retries += sum(1 for i in info if i["fp64_retry"])
        if n % snap == 0 or n == steps:
            if gpc:  # moments of the surrogate (eqs. PCEcoef, var), P from 10^5 points
                coef, mean, var = E.elder_gpc_project(beta, theta_t, wq_t, c.view(S, N))
                pexc = E.elder_gpc_exceed(beta, coef, theta_s, 0.5)
            else:
                mean, var, pexc = ctx.moments(S, c)
            mh = mean.cpu().numpy()
            lob[str(n)] = plume_lobes(mh, nx, ny, nz)
            snaps[f"mean_{n}"] = mh.astype(np.float32)
            if n == steps:
                fields = {"var": var.cpu().numpy().astype(np.float32),
                          "pexc": pexc.cpu().numpy().astype(np.float32)}
            print(f"fingers: step {n} ({n * a.fingers_dt_yr:.2f} yr), "
                  f"{S * n / (ms / 1000.0):.1f} sample-timesteps/s so far, lobes "
                  f"{json.dumps(lob[str(n)]['plane'])}, wall {time.time() - t_wall:.0f} s",
                  file=sys.stderr, flush=True)
            if a.fingers_out:  # written at every snapshot, so a cut-off run keeps its fields
                np.savez_compressed(a.fingers_out, xi=xi_np, grid=np.array([nx, ny, nz]),
                                    dt_yr=np.array(a.fingers_dt_yr), **snaps, **fields)
    ctx.destroy()
    line = {"metric": f"sample-timesteps/s, the paper's parallelepiped ensemble (3 random "
                      f"variables) at {nx}x{ny}x{nz}",
            "value": S * steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": max(a.warmup, 2), "higher_is_better": True, "dtype": "f64+f32+bf16",
            "data": "synthetic",
            "config": {"workload": (f"elder3d-box-{nx}x{ny}x{nz}-paper3rv-"
                                    + (f"gauss-legendre{S}-gpc4" if gpc else f"halton{S}")),
                       "dt_yr": a.fingers_dt_yr, "bc": "paper variant (bc_mode 1)",
                       "fields": ("5^3 Gauss-Legendre points; mean, variance and P(c > 0.5) "
                                  "of the order-4 gPC surrogate" if gpc else
                                  "Halton points (bases 2,3,5, first point skipped)") +
                                 " -> the paper's parallelepiped porosity field, Kozeny-Carman K",
                       "newton_start": "3u^n - 3u^(n-1) + u^(n-2)",
                       "timed_steps": f"1-{steps} from t = 0"},
            "iterations": {"newton_per_step": newton / (S * steps),
                           "krylov_per_step": krylov / (S * steps),
                           "failed_sample_steps": failed, "fp64_retries": retries},
            "lobes": lob,
            "timing": "CUDA events around each step on the launching stream"}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "uneven":
        run_uneven(a)
    elif a.workload == "config2":
        run_config2(a)
    elif a.fingers_compare:
        compare_fingers(*a.fingers_compare)
    elif a.workload == "fingers":
        run_fingers(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
