#!/usr/bin/env python
"""Benchmark: PID (ns per DOF per RK stage) of the DGSEM Navier-Stokes LSERK4(5)
step on GB300 (Krais et al., FLEXI, Sec. 5.6: PID = wall * #cores / (#DOF *
#steps * #stages), with #cores -> #GPUs).

Workload: Taylor-Green vortex (Re = 1600, Ma = 0.1) on a periodic 16^3 mesh,
N = 7 Gauss nodes (2,097,152 DOF), HLLC flux, BR1 lifting, fixed dt from CFL
0.9; one bench step = one LSERK4(5) time step (5 RK stages) in FP64.  Inputs
are resident in HBM and larger than L2.  Extra keys report the FP32 forms
(PID and error against FP64 after the timed steps) and the adjoint/forward
cost ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torchrun): every rank runs an independent replica (the library
computes on one GPU; no data-path collective); value is whole-job.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PID ns/DOF/RK-stage at N=7 on 1 GB300: FP64 vs FP32/TC (err vs FP64); adjoint/fwd"
UNIT = "ns/DOF/RK-stage"
WORKLOAD = dict(workload="taylor-green vortex, periodic 16^3 hex, N=7 Gauss, HLLC, BR1, LSERK4(5), CFL 0.9",
                elements=4096, N=7, dof=2097152, re=1600, mach=0.1, step="one LSERK4(5) step = 5 RK stages",
                l2="inputs larger than L2 (working set > 129 MB)")
NSTAGES = 5


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM bytes (read + write) per launch of the lifting/volume kernel (k_lift_vol_mb) from the ncu captures
# summarised in profiles/, keyed by form and by a hash of the kernel sources at
# capture time; reported only while the sources are unchanged (else null).
KERNEL_SOURCES = ["paper_1910_02858_gb300/csrc/k_dg.cuh", "paper_1910_02858_gb300/csrc/dg_common.cuh",
                  "paper_1910_02858_gb300/csrc/k_tc.cuh", "paper_1910_02858_gb300/csrc/k_adj.cuh"]
NCU_TRAFFIC = {("fp64", "41f95f6d2cdf1e15"): 574419200, ("fp32", "41f95f6d2cdf1e15"): 266935296}


def kernel_source_hash(texts=None) -> str:
    """Hash of the kernel sources without comments and blank lines (what the
    compiler sees), so that an ncu figure stays attached to unchanged kernels."""
    import hashlib
    import re

    h = hashlib.sha256()
    for i, f in enumerate(KERNEL_SOURCES):
        if texts is None:
            with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
                t = fh.read()
        else:
            t = texts[i]
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in t.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


# GB300 FP64 FMA peak derived from unit counts and clocks: 152 SMs x 2 DFMA/clk
# (4 FP64 flop/clk/SM, consistent with the nominal 1.25 TFLOP/s) x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# FP32 FMA peak from the same unit counts: 128 FP32 lanes x 2 flop/clk per SM
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Slowest rank's time (the job is as slow as its slowest replica)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_pid(seconds: float, steps: int, dof_per_rank: int, world: int) -> float:
    """PID of the whole job in ns per DOF per RK stage: wall / (all ranks' DOF * steps * stages)."""
    return seconds * 1e9 / (steps * NSTAGES * dof_per_rank * world)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def algorithmic_per_dof(n: int, word: int):
    """Per DOF and RK stage: minimum-traffic bytes of the three-kernel schedule and
    the flops of the dominant kernel (lifting + volume integral), FMA = 2 flops."""
    f = 3.0 / n
    bytes_stage = (46.0 + 117.0 * f) * word
    bytes_liftvol = (20.0 + 48.0 * f) * word
    flops_liftvol = (2 * 45 * n          # lifting D_hat sweeps (3 directions x 15 components)
                     + 2 * 90            # LG lifting surface terms, 6 faces x 15 components
                     + 45 + 15 + 10      # contravariant products Ja W, 1/J scaling, primitives
                     + 2 * 90            # LG prolongation of the 15 gradients to 6 faces
                     + 3 * 30            # pointwise fluxes F^c - F^v, 3 directions
                     + 2 * 45            # contravariant transform sum_d Ja^l_d F^d
                     + 2 * 15 * n)       # volume D_hat sweeps (3 directions x 5 variables)
    return bytes_stage, bytes_liftvol, flops_liftvol


def host_cpu():
    """Core count and CPU model of the host (the oracle runs on these cores)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "model": model}


def time_oracle_stages(warmup: int, stages: int, threads=None):
    """The FP64 oracle as it stands, on the host cores: full LSERK4(5) stages
    (right-hand side + low-storage update) of the 16^3, N = 7 Taylor-Green
    workload, after untimed warm-up stages.  Returns (PID, threads used, seconds)."""
    import torch

    import workloads as wl
    from oracle.dgsem import DGSEM, HLLC, RK_A, RK_B, Params

    if threads is not None:
        torch.set_num_threads(threads)
    mesh = wl.box_mesh((16, 16, 16), Ngeo=1)
    dg = DGSEM(Params(N=7, node_type=0, riemann=HLLC), mesh.coords, mesh.conn)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(7, 0)))
    dU = torch.zeros_like(U)
    dof = dg.K * dg.n ** 3

    def stage(U, dU, k):
        Ut = dg.rhs(U)
        dU = RK_A[k % 5] * dU + 1e-4 * Ut
        return U + RK_B[k % 5] * dU, dU

    for k in range(warmup):
        U, dU = stage(U, dU, k)
    t0 = time.perf_counter()
    for k in range(stages):
        U, dU = stage(U, dU, k)
    el = time.perf_counter() - t0
    return el / (stages * dof) * 1e9, torch.get_num_threads(), el


CPU_BASELINE_STAGES = (5, 20)  # warm-up and timed stages, all host cores
CPU_BASELINE_STAGES_1T = (1, 3)  # the same on one host thread


def run_cpu_baseline():
    """CPU baseline of the native arm: the reference arm's own measurement (the
    oracle on the host cores), run in fresh processes before any GPU work, so that
    both arms time the same code in the same conditions; plus the one-thread figure."""
    def arm(warmup, steps, threads=None):
        cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
               "--warmup", str(warmup)]
        if threads is not None:
            cmd += ["--threads", str(threads)]
        env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
        for ln in out.stdout.splitlines()[::-1]:
            if ln.startswith("{"):
                return json.loads(ln)
        raise RuntimeError(f"oracle timing failed: {out.stderr[-500:]}")

    full = arm(*CPU_BASELINE_STAGES)
    one = arm(*CPU_BASELINE_STAGES_1T, threads=1)
    w, k = CPU_BASELINE_STAGES
    return {"value": full["value"], "unit": UNIT, "cores": full["cpu_baseline"]["cores"], "kind": "oracle",
            "sample": f"{k} RK stages (full RHS + low-storage update) of the 16^3 N=7 TGV workload after {w} "
                      "warm-up stages, FP64 torch CPU, fresh process before any GPU work (the reference arm's code)",
            "value_1_thread": one["value"],
            "sample_1_thread": f"{CPU_BASELINE_STAGES_1T[1]} RK stages after {CPU_BASELINE_STAGES_1T[0]} warm-up, "
                               "one host thread",
            "host": host_cpu()}


def reference_arm(args):
    """--impl reference: the oracle timed as the reference arm on the host cores
    (one bench step = one RK stage of the workload, a bounded sample of it)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    pid, cores, el = time_oracle_stages(args.warmup, args.steps, args.threads)
    line = {"metric": METRIC, "value": pid, "unit": UNIT, "impl": "reference", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, step="one RK stage (RHS + update) of the oracle"),
            "cpu_baseline": {"value": pid, "unit": UNIT, "kind": "oracle", "cores": cores,
                             "sample": f"{args.steps} RK stages of the 16^3 N=7 TGV workload after "
                                       f"{args.warmup} warm-up stages", "host": host_cpu()},
            "e2e": {"value": pid, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(s, U, dU, dt, nsteps, F, torch, dev, t0=0.0):
    """Event-timed LSERK4(5) steps on the library's stream with per-launch profiling
    off (the product's launch stream), then the same number of steps again with the
    library's per-launch events on, for the per-kernel times.  Returns (ms of the
    clean steps, per-kernel times of the profiled pass)."""
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(nsteps):
        s.step(U, dU, t0 + k * dt, dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    F.flexi_kernel_times(s.ctx, reset=True)
    F.flexi_profile(s.ctx, True)
    for k in range(nsteps):
        s.step(U, dU, t0 + (nsteps + k) * dt, dt)
    torch.cuda.synchronize(dev)
    kt = F.flexi_kernel_times(s.ctx, reset=True)
    F.flexi_profile(s.ctx, False)
    return ms, kt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32 and adjoint extra measurements")
    ap.add_argument("--form", default="fp64", choices=["fp64", "fp32", "tf32x3", "bf16x3"],
                    help="arithmetic form of the timed workload (default: the FP64 headline)")
    ap.add_argument("--threads", type=int, default=None, help="host threads of the reference arm (default: all)")
    ap.add_argument("--nelem", type=int, default=16,
                    help="elements per direction of the timed Taylor-Green mesh (16: the headline workload; "
                         "smaller meshes for profiler captures)")
    ap.add_argument("--case", default=None, choices=["c1"],
                    help="time only the small C1 case (4^3 elements, N = 3 Gauss-Lobatto, Roe, FP64): "
                         "--warmup steps, then --steps steps replayed from the CUDA graph; one JSON line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)
    world, rank, local = dist_env()
    cpu_line = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        # before any GPU work in this process: the oracle in fresh processes
        try:
            cpu_line = run_cpu_baseline()
        except Exception as exc:  # pragma: no cover
            cpu_line = {"value": None, "error": repr(exc)}

    import numpy as np
    import torch

    import workloads as wl
    from paper_1910_02858_gb300 import Solver, SolverConfig
    from paper_1910_02858_gb300 import build as B
    from paper_1910_02858_gb300 import flexi as F

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    F.lib()
    if args.case == "c1":
        print(json.dumps(c1_case(args, dev, F, wl, Solver, SolverConfig, torch)))
        return 0

    N = 7
    mesh = wl.box_mesh((args.nelem,) * 3, Ngeo=1)
    x = mesh.node_coords(N, 0)
    U0 = wl.taylor_green(x)
    workload = WORKLOAD if args.nelem == 16 else dict(
        WORKLOAD, workload=WORKLOAD["workload"].replace("16^3", f"{args.nelem}^3"), elements=mesh.K,
        dof=mesh.K * (N + 1) ** 3, l2="small profiling case")
    prec = {"fp64": F.FP64, "fp32": F.FP32, "tf32x3": F.FP32_TF32, "bf16x3": F.FP32_BF16}[args.form]
    cfg = SolverConfig(N=N, riemann=F.RIEMANN_HLLC, precision=prec)
    s = Solver(cfg, mesh.coords, mesh.conn, device=dev)
    dof = s.query(F.Q_DOF)
    U = torch.tensor(U0, device=dev, dtype=s.dtype)
    dU = torch.zeros_like(U)
    dt = s.reduce(U)["dt_max"]
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    # count kernel launches per step (profiled, untimed)
    F.flexi_profile(s.ctx, True)
    s.step(U.clone(), dU.clone(), 0.0, dt)
    launches_per_step = sum(c for _, c in F.flexi_kernel_times(s.ctx, reset=True).values())
    F.flexi_profile(s.ctx, False)

    t = 0.0
    for _ in range(args.warmup):
        s.step(U, dU, t, dt)
        t += dt
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed region: the product's launch stream, no per-launch events
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            s.step(U, dU, t, dt)
            t += dt
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    # per-kernel times: the same number of steps again, with the library's per-launch
    # CUDA events (on the launching stream), timed on their own
    F.flexi_kernel_times(s.ctx, reset=True)
    F.flexi_profile(s.ctx, True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        s.step(U, dU, t, dt)
        t += dt
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    ms_profiled = pe0.elapsed_time(pe1)
    ktimes = F.flexi_kernel_times(s.ctx, reset=True)
    F.flexi_profile(s.ctx, False)
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    pid = whole_job_pid(ms_total * 1e-3, args.steps, dof, world)

    # roofline of the dominant kernel (lifting + volume): FP64 form ALU-bound (FP64 pipe),
    # FP32 forms HBM-bound
    n = N + 1
    word = 8 if args.form == "fp64" else 4
    bytes_stage, bytes_lv, flops_lv = algorithmic_per_dof(n, word)
    lv_ms, lv_cnt = ktimes["lift_vol"]
    lv_avg_s = lv_ms / max(lv_cnt, 1) * 1e-3
    share = lv_ms / max(sum(v[0] for v in ktimes.values()), 1e-9)
    traffic = NCU_TRAFFIC.get((args.form, kernel_source_hash()))
    if args.form == "fp64":
        achieved_tflops = flops_lv * dof / lv_avg_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": "k_lift_vol_mb<double,8>",
                    "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2070 MHz (nominal 1.25 TFLOP/s)",
                    "kernel_share": share}
    else:
        hbm = peaks().get("hbm_gbs", 6800.0)
        achieved = bytes_lv * dof / lv_avg_s / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": traffic,
                    # k_lift_vol_mb: the instance with a minimum of resident CTAs per SM
                    "kernel": "k_lift_vol_mb<float,8>" if args.form == "fp32" else f"k_lift_vol<float,8,{args.form}>",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks() else "fallback 6.8 TB/s",
                    "kernel_share": share}
    step_bytes_gbs = bytes_stage * dof * NSTAGES / (ms_step * 1e-3) / 1e9
    # whole-step roofline: the slower of the step's algorithmic bytes over the measured HBM
    # bandwidth and its algorithmic flops at the form's FMA peak (the library's own counts)
    bps = s.query(F.Q_BYTES_PER_STAGE) / dof
    fps = s.query(F.Q_FLOPS_PER_STAGE) / dof
    fpk = FP64_PEAK_TFLOPS if args.form == "fp64" else FP32_PEAK_TFLOPS
    t_mem, t_alu = bps / peaks().get("hbm_gbs", 6800.0), fps / (fpk * 1e3)  # ns per DOF and stage
    step_roofline = {"bound": "alu" if t_alu > t_mem else "hbm", "floor_ns": max(t_mem, t_alu),
                     "achieved_ns": pid * world, "frac": max(t_mem, t_alu) / (pid * world),
                     "bytes_per_dof": bps, "flops_per_dof": fps, "alu_peak_tflops": fpk,
                     "alu_peak_source": "derived from unit counts at 2070 MHz"}
    kernels = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else 0.0, "launches": v[1]} for k, v in ktimes.items() if v[1]}

    # end to end through the public API with host buffers (H2D + step + D2H per step)
    Uh = torch.tensor(U0, dtype=s.dtype).pin_memory()
    F.flexi_rk_run_host(s.ctx, Uh, 1, 0.0, dt, stream)
    barrier()
    t0 = time.perf_counter()
    for k in range(max(3, args.steps // 2)):
        F.flexi_rk_run_host(s.ctx, Uh, 1, k * dt, dt, stream)
    e2e_s = time.perf_counter() - t0
    e2e_steps = max(3, args.steps // 2)
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_pid = whole_job_pid(e2e_s, e2e_steps, dof, world)
    ubytes = U.numel() * U.element_size()

    line = {"metric": METRIC, "value": pid, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f32", "data": "synthetic",
            "config": dict(workload, dt=dt, form=args.form),
            "clocks": clk.summary(), "gpu_launches": launches_per_step * args.steps,
            "e2e": {"value": e2e_pid, "unit": UNIT, "h2d_bytes_per_step": ubytes, "d2h_bytes_per_step": ubytes},
            "roofline": roofline, "dof_updates_per_s": dof * world / (pid * 1e-9 * dof * world) if pid else None,
            "step_algorithmic_hbm_gbs": step_bytes_gbs, "step_roofline": step_roofline, "kernels": kernels}

    line["profiled_pass"] = {"steps": args.steps, "ms_per_step": ms_profiled / args.steps,
                             "note": "per-kernel times and the roofline's launch duration come from this pass "
                                     "(library CUDA events around every launch); value is timed without them"}
    if rank == 0 and not args.no_extras:
        line["extras"] = extras(args, s, U0, mesh, dt, dev, F, wl, Solver, SolverConfig, torch, np)
    s.close()
    if cpu_line is not None:
        line["cpu_baseline"] = cpu_line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def rel_err_per_var(U, Uref):
    """Relative L2 error per conserved variable; the momentum components are
    normalised by the norm of the whole momentum vector (the Taylor-Green
    w-momentum starts at zero)."""
    d = (U.double() - Uref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = Uref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    rm = r[1:4].norm()
    r = r.clone()
    r[1:4] = rm
    return (d / r).tolist()


def extras(args, s64, U0, mesh, dt, dev, F, wl, Solver, SolverConfig, torch, np):
    """FP32 forms on the same workload (PID and error vs FP64 after the same
    number of steps) and the adjoint/forward cost ratio."""
    out = {}
    nsteps = 20
    U64 = torch.tensor(U0, device=dev)
    s64.run(U64, nsteps, dt)
    for name, prec in (("fp32", F.FP32), ("fp32_tf32x3", F.FP32_TF32), ("fp32_bf16x3", F.FP32_BF16)):
        try:
            s = Solver(SolverConfig(N=7, riemann=F.RIEMANN_HLLC, precision=prec), mesh.coords, mesh.conn, device=dev)
        except Exception as exc:
            out[name] = {"error": str(exc)}
            continue
        try:
            U = torch.tensor(U0, device=dev, dtype=torch.float32)
            dU = torch.zeros_like(U)
            for _ in range(3):
                s.step(U, dU, 0.0, dt)
            U = torch.tensor(U0, device=dev, dtype=torch.float32)
            dU.zero_()
            ms, kt = timed_steps(s, U, dU, dt, nsteps, F, torch, dev)
            # the error against FP64 is taken after the first nsteps steps (as the FP64 run)
            U = torch.tensor(U0, device=dev, dtype=torch.float32)
            s.run(U, nsteps, dt)
            dof = s.query(F.Q_DOF)
            n = 8
            bytes_stage = (46.0 + 117.0 * 3.0 / n) * 4 * dof
            lv = kt["lift_vol"][0] / max(kt["lift_vol"][1], 1)
            pid32 = ms * 1e6 / (nsteps * NSTAGES * dof)
            floor = max(s.query(F.Q_BYTES_PER_STAGE) / dof / peaks().get("hbm_gbs", 6800.0),
                        s.query(F.Q_FLOPS_PER_STAGE) / dof / (FP32_PEAK_TFLOPS * 1e3))
            out[name] = {"pid": pid32, "step_roofline_frac": floor / pid32, "steps": nsteps,
                         "rel_l2_err_vs_fp64": rel_err_per_var(U, U64),
                         "step_algorithmic_hbm_gbs": bytes_stage * NSTAGES * nsteps / (ms * 1e-3) / 1e9,
                         "lift_vol_ms_per_launch": lv,
                         "lift_vol_hbm_gbs": (20.0 + 48.0 * 3.0 / n) * 4 * dof / (lv * 1e-3) / 1e9}
        except Exception as exc:
            out[name] = {"error": str(exc)}
        finally:
            s.close()
    try:
        out["lobatto"] = lobatto_pid(mesh, dt, dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["lobatto"] = {"error": repr(exc)}
    try:
        out["c4_curved_24^3_N7"] = c4_curved_pid(dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["c4_curved_24^3_N7"] = {"error": repr(exc)}
    try:
        out["c3_32^3_N5"] = c3_forms_pid(dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["c3_32^3_N5"] = {"error": repr(exc)}
    try:
        out["memory_kib_per_dof"] = memory_per_dof(dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["memory_kib_per_dof"] = {"error": repr(exc)}
    try:
        out["small_cases"] = small_cases_pid(dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["small_cases"] = {"error": repr(exc)}
    try:
        out["mortar"] = mortar_pid(dt, dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["mortar"] = {"error": repr(exc)}
    try:
        out["adjoint"] = adjoint_ratio(dev, F, wl, Solver, SolverConfig, torch)
    except Exception as exc:
        out["adjoint"] = {"error": repr(exc)}
    return out


def lobatto_pid(mesh, dt, dev, F, wl, Solver, SolverConfig, torch):
    """The same 16^3, N = 7 Taylor-Green step on Gauss-Lobatto nodes (prolongation
    is a copy, face terms touch only face nodes), FP64 and FP32, with the standard
    and with the split-form (kinetic-energy-preserving) volume integral."""
    res = {}
    x = mesh.node_coords(7, 1)
    for name, prec, split in (("fp64", F.FP64, F.SPLIT_STANDARD), ("fp32", F.FP32, F.SPLIT_STANDARD),
                              ("fp64_split_kep", F.FP64, F.SPLIT_KEP), ("fp32_split_kep", F.FP32, F.SPLIT_KEP),
                              ("fp64_split_ec", F.FP64, F.SPLIT_EC), ("fp32_split_ec", F.FP32, F.SPLIT_EC)):
        s = Solver(SolverConfig(N=7, node_type=F.NODES_LOBATTO, riemann=F.RIEMANN_HLLC, precision=prec,
                                split_form=split), mesh.coords, mesh.conn, device=dev)
        try:
            U = torch.tensor(wl.taylor_green(x), device=dev, dtype=s.dtype)
            dU = torch.zeros_like(U)
            for _ in range(3):
                s.step(U, dU, 0.0, dt)
            ms, kt = timed_steps(s, U, dU, dt, 10, F, torch, dev)
            res[name] = {"pid": ms * 1e6 / (10 * NSTAGES * s.query(F.Q_DOF)), "steps": 10,
                         "lift_vol_ms_per_launch": kt["lift_vol"][0] / max(kt["lift_vol"][1], 1)}
        finally:
            s.close()
    return res


def c4_curved_pid(dev, F, wl, Solver, SolverConfig, torch):
    """The curved-mesh workload: [-1, 1]^3, 24^3 elements mapped by
    x_i = xi_i + 0.1 prod_j sin(pi xi_j), N = Ngeo = 7 Gauss, curl-form metrics,
    HLLC, BR1, Dirichlet (exact-state) boundaries on all six sides (7,077,888 DOF).
    (a) free stream rho = 1, u = (0.3, 0.2, 0.1), p = 1/gamma (operator independent
    of t: the exact state is constant); (b) the manufactured solution with its
    source term (time-dependent boundary state and source).  FP64 and FP32: PID,
    whole-step roofline fraction, the lifting/volume kernel's time and share, and
    for (a) the largest deviation from the free stream after the steps."""
    mesh = wl.box_mesh((24, 24, 24), lo=(-1.0,) * 3, hi=(1.0,) * 3, Ngeo=7, mapping="sine", periodic=(False,) * 3)
    N, nsteps = 7, 10
    x = mesh.node_coords(N, 0)
    res = {}
    for case, U0, bc, src in (("freestream", wl.freestream(x), F.EXACT_FREESTREAM, False),
                              ("manufactured", wl.manufactured(x, 0.0), F.EXACT_MANUFACTURED, True)):
        for name, prec in (("fp64", F.FP64), ("fp32", F.FP32)):
            s = Solver(SolverConfig(N=N, Ngeo=N, riemann=F.RIEMANN_HLLC, precision=prec, bc_exact=bc, source=src),
                       mesh.coords, mesh.conn, device=dev)
            try:
                U = torch.tensor(U0, device=dev, dtype=s.dtype)
                dt = s.reduce(U)["dt_max"]
                dU = torch.zeros_like(U)
                for k in range(3):
                    s.step(U, dU, k * dt, dt)
                U = torch.tensor(U0, device=dev, dtype=s.dtype)
                dU.zero_()
                ms, kt = timed_steps(s, U, dU, dt, nsteps, F, torch, dev)
                dof = s.query(F.Q_DOF)
                pid = ms * 1e6 / (nsteps * NSTAGES * dof)
                fpk = FP64_PEAK_TFLOPS if prec == F.FP64 else FP32_PEAK_TFLOPS
                floor = max(s.query(F.Q_BYTES_PER_STAGE) / dof / peaks().get("hbm_gbs", 6800.0),
                            s.query(F.Q_FLOPS_PER_STAGE) / dof / (fpk * 1e3))
                tot = sum(v[0] for v in kt.values())
                lv = kt["lift_vol"][0] / max(kt["lift_vol"][1], 1)
                row = {"dof": dof, "dt": dt, "steps": nsteps, "pid": pid, "step_roofline_frac": floor / pid,
                       "floor_ns": floor, "lift_vol_ms_per_launch": lv,
                       "lift_vol_share": kt["lift_vol"][0] / tot if tot > 0 else None}
                if prec == F.FP64:
                    row["lift_vol_alu_frac"] = (algorithmic_per_dof(N + 1, 8)[2] * dof / (lv * 1e-3) / 1e12
                                                / FP64_PEAK_TFLOPS)
                else:
                    row["lift_vol_hbm_frac"] = (algorithmic_per_dof(N + 1, 4)[1] * dof / (lv * 1e-3) / 1e9
                                                / peaks().get("hbm_gbs", 6800.0))
                if case == "freestream":
                    # 2 * nsteps steps were taken from U0 (timed + profiled pass)
                    U0d = torch.tensor(U0, device=dev, dtype=s.dtype)
                    row["freestream_max_rel_dev"] = float(((U - U0d).abs().amax(dim=(0, 2, 3, 4))
                                                           / U0d.abs().amax(dim=(0, 2, 3, 4))).max())
                res[f"{case}_{name}"] = row
            finally:
                s.close()
    return res


def c3_forms_pid(dev, F, wl, Solver, SolverConfig, torch):
    """The precision form's own workload: Taylor-Green 32^3, N = 5 Gauss (7.08 M DOF),
    HLLC, in FP64 and the three FP32 forms: PID, whole-step roofline fraction and the
    relative L2 error against FP64 after 20 steps (momentum against the momentum-vector
    norm)."""
    mesh = wl.box_mesh((32, 32, 32), Ngeo=1)
    N, nsteps = 5, 20
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    res, ref = {}, None
    for name, prec in (("fp64", F.FP64), ("fp32", F.FP32), ("fp32_tf32x3", F.FP32_TF32), ("fp32_bf16x3", F.FP32_BF16)):
        s = Solver(SolverConfig(N=N, riemann=F.RIEMANN_HLLC, precision=prec), mesh.coords, mesh.conn, device=dev)
        try:
            U = torch.tensor(U0, device=dev, dtype=s.dtype)
            dt = 0.5 * s.reduce(U)["dt_max"] if ref is None else res["fp64"]["dt"]
            dU = torch.zeros_like(U)
            for _ in range(3):
                s.step(U, dU, 0.0, dt)
            U = torch.tensor(U0, device=dev, dtype=s.dtype)
            dU.zero_()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(nsteps):
                s.step(U, dU, k * dt, dt)
            e1.record()
            torch.cuda.synchronize(dev)
            dof = s.query(F.Q_DOF)
            pid = e0.elapsed_time(e1) * 1e6 / (nsteps * NSTAGES * dof)
            fpk = FP64_PEAK_TFLOPS if prec == F.FP64 else FP32_PEAK_TFLOPS
            floor = max(s.query(F.Q_BYTES_PER_STAGE) / dof / peaks().get("hbm_gbs", 6800.0),
                        s.query(F.Q_FLOPS_PER_STAGE) / dof / (fpk * 1e3))
            res[name] = {"pid": pid, "step_roofline_frac": floor / pid, "steps": nsteps, "dt": dt}
            red = s.reduce(U, s.rhs(U))
            if ref is None:
                ref, ref_red = U.double(), red
            else:
                res[name]["rel_l2_err_vs_fp64"] = rel_err_per_var(U, ref)
                res[name]["ke_rel_err"] = abs(red["kinetic_energy"] - ref_red["kinetic_energy"]) / ref_red["kinetic_energy"]
                res[name]["dkedt_rel_err"] = abs(red["dkedt"] - ref_red["dkedt"]) / abs(ref_red["dkedt"])
        finally:
            s.close()
    return res


def memory_per_dof(dev, F, wl, Solver, SolverConfig, torch):
    """Device bytes the library holds per DOF (FP64, Gauss, periodic, about 1 M DOF),
    without and with the adjoint's scratch, plus the caller's U and dU (2 x 5 words),
    for N = 1..7; the paper measures 1.47, 1.08, 0.906, 0.805, 0.74, 0.693, 0.659 KiB per
    DOF on its CPUs (Table memoryReq)."""
    res = {}
    for N in range(1, 8):
        nel = max(2, round((1.0e6 ** (1.0 / 3.0)) / (N + 1)))
        mesh = wl.box_mesh((nel,) * 3, Ngeo=1)
        row = {"elements": int(mesh.K)}
        for adj in (False, True):
            s = Solver(SolverConfig(N=N, riemann=F.RIEMANN_ROE, adjoint=adj), mesh.coords, mesh.conn, device=dev)
            try:
                dof = s.query(F.Q_DOF)
                row["kib_adjoint" if adj else "kib"] = (s.query(F.Q_DEVICE_BYTES) + 2 * 5 * 8 * dof) / dof / 1024
            finally:
                s.close()
        res[f"N{N}"] = row
    return res


def small_cases_pid(dev, F, wl, Solver, SolverConfig, torch):
    """Launch-bound sizes: C1 (4^3, N = 3 LGL, Roe, dt = 1e-3) and the adjoint
    workload's forward (8^3, N = 5, smoothed Roe): PID with every step launched
    (flexi_rk_step) and with the CUDA-graph replay of flexi_rk_run."""
    res = {}
    for label, nel, N, nt, riem in (("c1_4^3_N3_lgl", 4, 3, 1, F.RIEMANN_ROE), ("c5_8^3_N5", 8, 5, 0,
                                                                               F.RIEMANN_ROE_SMOOTH)):
        mesh = wl.box_mesh((nel,) * 3, Ngeo=1)
        s = Solver(SolverConfig(N=N, node_type=nt, riemann=riem), mesh.coords, mesh.conn, device=dev)
        try:
            U = torch.tensor(wl.taylor_green(mesh.node_coords(N, nt)), device=dev)
            dof = s.query(F.Q_DOF)
            out = {}
            for mode, graph in (("launches", False), ("graph", True)):
                s.run(U, 20, 1e-4, graph=graph)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.run(U, 200, 1e-4, graph=graph)
                e1.record()
                torch.cuda.synchronize(dev)
                out[mode] = e0.elapsed_time(e1) * 1e6 / (200 * NSTAGES * dof)
            F.flexi_kernel_times(s.ctx, reset=True)
            F.flexi_profile(s.ctx, True)
            s.run(U, 20, 1e-4, graph=False)
            torch.cuda.synchronize(dev)
            kt = F.flexi_kernel_times(s.ctx, reset=True)
            F.flexi_profile(s.ctx, False)
            res[label] = {"dof": dof, "pid_launches": out["launches"], "pid_graph": out["graph"],
                          "us_per_launch": {k: v[0] / v[1] * 1e3 for k, v in kt.items() if v[1]}}
        finally:
            s.close()
    return res


def c1_case(args, dev, F, wl, Solver, SolverConfig, torch):
    """C1 alone (Taylor-Green, 4^3 periodic elements, N = 3 Gauss-Lobatto, Roe, FP64,
    dt = 1e-4): args.warmup steps, then args.steps steps of flexi_rk_run (CUDA-graph
    replay), event-timed on the launching stream; PID in ns per DOF and RK stage."""
    mesh = wl.box_mesh((4,) * 3, Ngeo=1)
    s = Solver(SolverConfig(N=3, node_type=1, riemann=F.RIEMANN_ROE), mesh.coords, mesh.conn, device=dev)
    try:
        U = torch.tensor(wl.taylor_green(mesh.node_coords(3, 1)), device=dev)
        dof = s.query(F.Q_DOF)
        s.run(U, args.warmup, 1e-4)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.run(U, args.steps, 1e-4)
        e1.record()
        torch.cuda.synchronize(dev)
        pid = e0.elapsed_time(e1) * 1e6 / (args.steps * NSTAGES * dof)
        return {"case": "c1_4^3_N3_lgl_roe_fp64", "dof": dof, "steps": args.steps, "warmup": args.warmup,
                "pid_graph": pid, "unit": "ns/DOF/RK-stage"}
    finally:
        s.close()


def mortar_pid(dt, dev, F, wl, Solver, SolverConfig, torch):
    """Taylor-Green step (N = 7 Gauss, HLLC, FP64) on a non-conforming periodic
    [0, 2 pi]^3 mesh: left half 4 x 8 x 8 elements, right half refined 2:1 in
    every direction (8 x 16 x 16), type-3 mortars at both interfaces (128 big
    sides); PID and the share of the mortar kernels."""
    import math

    m = wl.mortar_box_mesh(nx=4, ny=8, nz=8, refine=(2, 2, 2), lo=(0.0,) * 3, hi=(2 * math.pi,) * 3)
    s = Solver(SolverConfig(N=7, riemann=F.RIEMANN_HLLC, precision=F.FP64), m.coords, m.conn, device=dev,
               mortars=m.mortars)
    try:
        U = torch.tensor(wl.taylor_green(m.node_coords(7, 0)), device=dev)
        dU = torch.zeros_like(U)
        dtm = 0.5 * dt  # the fine half has half the element width
        for _ in range(3):
            s.step(U, dU, 0.0, dtm)
        ms, kt = timed_steps(s, U, dU, dtm, 10, F, torch, dev)
        tot = sum(v[0] for v in kt.values())
        return {"elements": m.K, "mortars": int(len(m.mortars)), "pid": ms * 1e6 / (10 * NSTAGES * s.query(F.Q_DOF)),
                "steps": 10, "mortar_kernel_share": kt["other"][0] / tot if tot > 0 else None}
    finally:
        s.close()


def adjoint_ratio(dev, F, wl, Solver, SolverConfig, torch):
    """Cost of dJ/dU0 (checkpointed forward + recompute + reverse sweep) over the
    cost of the plain forward run, on the adjoint workload: Taylor-Green Re = 400,
    8^3, N = 5, Roe with smoothed |lambda|, 40 steps of dt = 1e-3, checkpoints
    every 20 steps; the per-step ratio at N = 7, 16^3; and the same workload on
    Gauss-Lobatto nodes with the split-form volume integral (kinetic-energy-preserving
    and entropy-conservative two-point fluxes)."""
    from paper_1910_02858_gb300.adjoint import final_state

    res = {}
    for label, nel, N, nsteps, nt, split in (("c5_8^3_N5_40steps", 8, 5, 40, 0, F.SPLIT_STANDARD),
                                             ("16^3_N7_10steps", 16, 7, 10, 0, F.SPLIT_STANDARD),
                                             ("c5_lgl_split_kep", 8, 5, 40, 1, F.SPLIT_KEP),
                                             ("c5_lgl_split_ec", 8, 5, 40, 1, F.SPLIT_EC)):
        mesh = wl.box_mesh((nel,) * 3, Ngeo=1)
        s = Solver(SolverConfig(N=N, node_type=nt, riemann=F.RIEMANN_ROE_SMOOTH, mu=1 / 400.0, adjoint=True,
                                split_form=split), mesh.coords, mesh.conn, device=dev)
        U0 = torch.tensor(wl.taylor_green(mesh.node_coords(N, nt)), device=dev)
        dt = 1e-3
        lam = torch.randn_like(U0)

        def fwd():
            U = U0.clone()
            s.run(U, nsteps, dt)
            return U

        def grad():
            U0g = U0.clone().requires_grad_(True)
            UT = final_state(U0g, s, nsteps, dt, 0.0, 20)
            UT.backward(lam)
            return U0g.grad

        for f in (fwd, grad):
            f()
        times = {}
        for name, f in (("forward", fwd), ("gradient", grad)):
            reps = []
            for _ in range(3):  # median of three: the gradient includes host-side autograd work
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                f()
                torch.cuda.synchronize(dev)
                reps.append(time.perf_counter() - t0)
            times[name] = sorted(reps)[1]
        res[label] = {"forward_ms": times["forward"] * 1e3, "gradient_ms": times["gradient"] * 1e3,
                      "ratio": times["gradient"] / times["forward"]}
        s.close()
    res["c5_fp32_vs_fp64"] = adjoint_fp32_error(dev, F, wl, Solver, SolverConfig, torch, final_state)
    return res


def adjoint_fp32_error(dev, F, wl, Solver, SolverConfig, torch, final_state):
    """C5 forward and gradient in the FP32 form against FP64: relative L2 of the
    final state (momentum against the momentum-vector norm), of J and of dJ/dU0."""
    import math

    import numpy as np

    N, nsteps, dt = 5, 40, 1e-3
    mesh = wl.box_mesh((8, 8, 8), Ngeo=1)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    # J = sum_nodes w_i w_j w_k J_e |m|^2 / (2 rho): Gauss weights (numpy), affine elements of width 2 pi / 8
    w = np.polynomial.legendre.leggauss(N + 1)[1]
    w3 = np.einsum("k,j,i->kji", w, w, w) * (math.pi / 8) ** 3
    out = {}
    for name, prec, dtype in (("fp64", F.FP64, torch.float64), ("fp32", F.FP32, torch.float32)):
        s = Solver(SolverConfig(N=N, riemann=F.RIEMANN_ROE_SMOOTH, mu=1 / 400.0, precision=prec, adjoint=True),
                   mesh.coords, mesh.conn, device=dev)
        try:
            wJ = torch.tensor(w3, device=dev, dtype=dtype)
            U0d = torch.tensor(U0, device=dev, dtype=dtype, requires_grad=True)
            UT = final_state(U0d, s, nsteps, dt, 0.0, 20)
            J = (wJ * 0.5 * (UT[:, 1] ** 2 + UT[:, 2] ** 2 + UT[:, 3] ** 2) / UT[:, 0]).sum()
            J.backward()
            out[name] = (UT.detach().double(), U0d.grad.detach().double(), J.detach().item())
        finally:
            s.close()
    (U64, g64, J64), (U32, g32, J32) = out["fp64"], out["fp32"]
    d = (U32 - U64).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = U64.transpose(0, 1).reshape(5, -1).norm(dim=1)
    r[1:4] = U64[:, 1:4].norm()
    return {"state_rel_l2": (d / r).tolist(), "J_rel": abs(J32 - J64) / abs(J64),
            "grad_rel_l2": float((g32 - g64).norm() / g64.norm())}


if __name__ == "__main__":
    sys.exit(main())
