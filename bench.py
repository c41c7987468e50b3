#!/usr/bin/env python
"""Throughput benchmark of the CDBM hot path on GB300.

Workload: the Taylor-Green vortex on a periodic 4096 x 4096 grid (Sec. 3.5 setup
scaled up: L = 0.05, U0 = 0.01, tau = 1e-4, dt = 5e-6, I = 3, velocity set
(0.2, 0.2, 2, 2) / (0, 5, 0, 2.6)), double precision.  One bench step is one
Runge-Kutta time step over the whole grid (two fused stage kernels).  The state is
2.15 GB per buffer, far above the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank advances its own
independent vortex (weak scaling, no data-path collective); the barrier and the
max-over-ranks time use torch.distributed.

--impl reference times the CPU oracle (test infrastructure) on a bounded sample
of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s and HBM GB/s vs FP64 plain on same GB300 at stated L2 error"
UNIT = "cell-updates/s"

# FP64 work of the fused (row-marching) stage kernels per cell.  Instructions: ncu
# sm__inst_executed_pipe_fp64 per warp of 32 cells (stage 1: 246, stage 2: 262).
# Flops, counted from the kernel source with an FMA as two flops: stage 1: 367,
# stage 2: 399 (each x difference computed once per cell and shared through the row
# buffer; the halo recomputation of the block-edge threads is not counted).  Bytes
# per cell-step: stage 1 reads f^n and writes f1 (128 + 128 B); stage 2 reads f1 and
# f^n and writes f^n+1 (384 B).
FP64_INSTR_PER_CELL_STEP = 508
FP64_FLOPS_PER_CELL_STEP = 766
BYTES_PER_CELL_STEP = 640
FP64_LANES_PER_CLK_PER_SM = 2       # 1.25 TFLOP/s nominal FP64 / (2 flops x 152 SMs x 2.07 GHz)
BYTES_PER_CELL_STEP_FP32 = 320      # the same buffers in single precision
# Adjoint backward sweep per cell-step (FP64): the segment recompute (one forward
# step, 640 B, its stage-1 state written to the kept segment) and the two adjoint
# stage kernels (stage 2: read the stage-1 state and the cotangent, write one, 384 B;
# stage 1: read the state, two cotangents, write one, 512 B).
BYTES_PER_CELL_STEP_ADJ_BWD = 640 + 384 + 512

# DRAM traffic of one stage launch (mean of the two stages) from one ncu capture of
# the stage kernels; valid only while the code of the kernel sources (comments
# stripped) hashes to TRAFFIC_SHA.
# Captured at 1024^2 (134 MB per plane set, above L2) and scaled by 16 cells-fold.
TRAFFIC_SHA = "9985129ad1d51c36"
TRAFFIC_BYTES_PER_LAUNCH = 5.092e9


STAGE_SOURCES = ("cdbm_device.cuh", "cdbm_kernels.cu", "cdbm_internal.h")


def _code_only(text):
    """C/C++ source without comments and blank lines (string literals in these
    files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_sha():
    """Hash of the code (comments stripped) of the sources that define the stage kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_16818_gb300", "csrc")
    for name in STAGE_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            h.update(name.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["cdbm", "reference"], default="cdbm")
    p.add_argument("--n", type=int, default=4096, help="grid size (n x n)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-aux", action="store_true", help="skip timing the on-demand kernels (init, macros, Delta*, sums)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true", help="skip the FP32-bulk and ensemble runs")
    p.add_argument("--ens-steps", type=int, default=200, help="timed steps of the tube ensemble")
    p.add_argument("--no-ensemble", action="store_true", help="skip the tube ensemble runs")
    p.add_argument("--no-configs", action="store_true", help="skip the per-configuration wall times")
    p.add_argument("--cpu-configs", action="store_true",
                   help="also time the oracle on each configuration (1 thread and all cores)")
    p.add_argument("--adj-steps", type=int, default=4000, help="steps of the adjoint run (0: skip it)")
    p.add_argument("--adj-every", type=int, default=200, help="checkpoint interval of the adjoint run")
    p.add_argument("--adj-n", type=int, default=1024, help="grid size of the adjoint run")
    p.add_argument("--full-steps", type=int, default=2000,
                   help="steps of the full-length vortex runs in all four precisions (0: skip them)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(n):
    from paper_2502_16818_gb300 import workloads as W
    return W.taylor_green(n=n, I=3.0)


def arm_config(a, w, world):
    """The config of the bench line, the same for both arms."""
    plane_set_bytes = 16 * 8 * w.nx * w.ny
    return {"workload": "taylor_green_%dx%d_fp64" % (a.n, a.n), "nx": w.nx, "ny": w.ny,
            "I": w.I, "tau": w.tau, "dt": w.dt, "vset": [w.vg, w.eg], "precision": "fp64",
            "rk": "tvd2",
            "l2": "state %.3g GB per buffer vs 129 MB L2, no flush" % (plane_set_bytes / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


def cpu_sample(w, side):
    """A side x side block of the workload's initial fields (zero-gradient edges)."""
    import oracle
    sub = [a[:side, :side] for a in (w.rho, w.ux, w.uy, w.T)]
    m = oracle.Model(nx=side, ny=side, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg,
                     eg=w.eg, bc_x=1, bc_y=1, threads=os.cpu_count() or 1)
    return m, sub


def cpu_baseline(w, side=2048, steps=8):
    """The oracle (as it stands) on the host cores: `steps` steps on a side^2 sample."""
    import oracle
    m, sub = cpu_sample(w, side)
    f = oracle.init(m, *sub)
    t0 = time.perf_counter()
    oracle.step(m, f, steps)
    dt = time.perf_counter() - t0
    return {"value": side * side * steps / dt, "unit": UNIT, "cores": m.threads, "kind": "oracle",
            "sample": "%dx%d block of the %d^2 Taylor-Green initial state, %d RK2 steps, "
                      "zero-gradient edges, %.1f s wall" % (side, side, w.nx, steps, dt)}


def cpu_configs():
    """The oracle (as it stands) on each configuration, on 1 thread and on all host
    cores, each run bounded to about 10 s (2e6 cell-updates on one thread, 2e7 on
    all cores): Sod, Lax, the sound wave 512^2 and a 1024^2 block of the 4096^2
    vortex; cell-updates/s."""
    import oracle
    from paper_2502_16818_gb300 import workloads as W
    tgv = W.taylor_green(n=4096, I=3.0)
    block = [x[:1024, :1024] for x in (tgv.rho, tgv.ux, tgv.uy, tgv.T)]
    runs = [("sod_500_I0", W.sod(nx=500, I=0.0), None, 10000), ("lax_2000_I0", W.lax(nx=2000, I=0.0), None, 10000)]
    runs += [("sound_512_I%d" % I, W.sound(n=512, I=float(I)), None, 10) for I in (0, 1, 3)]
    runs += [("taylor_green_4096_block1024", tgv, block, 4)]
    res = {}
    for name, w, fields, steps in runs:
        row = {}
        for threads in (1, os.cpu_count() or 1):
            nx, ny = (1024, 1024) if fields else (w.nx, w.ny)
            bc = (1, 1) if fields else (w.bc_x, w.bc_y)
            m = oracle.Model(nx=nx, ny=ny, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg, eg=w.eg,
                             bc_x=bc[0], bc_y=bc[1], threads=threads)
            f = oracle.init(m, *(fields or (w.rho, w.ux, w.uy, w.T)))
            cap = 2e7 if threads > 1 else 2e6          # about 10 s of oracle work per run
            n = max(1, min(steps, int(cap // (nx * ny))))
            t0 = time.perf_counter()
            oracle.step(m, f, n)
            dt = time.perf_counter() - t0
            row["threads_%d" % threads] = {"value": nx * ny * n / dt, "unit": UNIT, "steps": n, "s": dt}
        res[name] = row
    return res


def run_reference(a, rank, world):
    if rank != 0:
        return
    w = workload(a.n)
    import oracle
    side = min(512, w.nx)
    m, sub = cpu_sample(w, side)
    f = oracle.init(m, *sub)
    for _ in range(a.warmup):
        f = oracle.step(m, f, 1)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        f = oracle.step(m, f, 1)
    dt = time.perf_counter() - t0
    value = side * side * a.steps / dt
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": arm_config(a, w, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": m.threads, "kind": "oracle",
                         "sample": "%dx%d block of the %d^2 Taylor-Green initial state, one RK2 step "
                                   "per bench step" % (side, side, a.n)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def tgv_amplitude(w, ux):
    """Projection of u_x onto sin(kx) cos(ky) (the Taylor-Green mode)."""
    import torch
    k = w.extra["k"]
    x = (torch.arange(w.nx, dtype=torch.float64, device=ux.device) + 0.5) * w.dx
    return float((ux * torch.cos(k * x)[:, None] * torch.sin(k * x)[None, :]).sum())


def time_tgv(w, precision, steps, warmup, torch, Solver):
    """A solver for the vortex on its own stream, initialised and warmed up; returns
    (solver, stream, Taylor-Green amplitude of u_x after the warm-up)."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = Solver.from_workload(w, stream=stream, precision=precision)
        fields = [torch.from_numpy(x).to("cuda") for x in (w.rho, w.ux, w.uy, w.T)]
        s.init(*fields)
        s.step(warmup)
    s.sync()
    a0 = tgv_amplitude(w, s.macros()[1])
    torch.cuda.synchronize()
    return s, stream, a0


def fp64_peak(torch, cdbm, stream, local_rank=0, launches=40):
    """Measured FP64 FMA rate of this GPU (TFLOP/s): the library's probe kernel, 8
    independent chains of dependent FMAs per thread, 152 x 8 blocks of 256 threads,
    each launch timed with CUDA events on `stream` (about 16 ms each; best and
    median of `launches`), SM clocks sampled meanwhile."""
    blocks, threads, iters = 152 * 8, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    sampler = ClockSampler(local_rank)
    sampler.start()
    rates = []
    for _ in range(launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = cdbm.cdbm_diag_fp64_fma(out.data_ptr(), blocks, threads, iters, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        rates.append(flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    clocks = sampler.stop()
    return {"tflops": max(rates), "tflops_median": statistics.median(rates),
            "kernel": "fp64_fma_kernel (cdbm_diag_fp64_fma)", "launch": [blocks, threads, iters],
            "flops_per_launch": flops, "launches": launches, "clocks": clocks}


def run_cdbm(a, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2502_16818_gb300 import (CDBM_FP32_BULK, CDBM_FP32_DEV, CDBM_FP32_DF64, CDBM_FP64, Solver, cdbm,
                                        replicas)

    torch.cuda.set_device(local_rank)
    w = workload(a.n)
    cells = w.nx * w.ny
    s, stream, amp0 = time_tgv(w, CDBM_FP64, a.steps, a.warmup, torch, Solver)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(a.steps)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    s.sync()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_max = replicas.max_over_ranks(ms, device="cuda")
    value = replicas.job_throughput(cells * a.steps, world, ms_max * 1e-3)
    rho64, ux64, uy64, T64 = s.macros()
    amp1 = tgv_amplitude(w, ux64)
    t_run = a.steps * w.dt
    nu = float(T64.mean()) * w.tau
    decay = {"measured": -np.log(amp1 / amp0) / t_run, "navier_stokes": 2 * nu * w.extra["k"] ** 2,
             "window": "the timed steps only, right after the equilibrium initial state, while the viscous "
                       "stress still builds up (about 5 tau); config3_full fits the configured horizon"}

    # roofline of the dominant kernels (the two fused stage kernels, ~100% of the step)
    launch_ms = ms / (2 * a.steps)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_instr = FP64_LANES_PER_CLK_PER_SM * 152 * sm_mhz * 1e6
    achieved_tflops = FP64_FLOPS_PER_CELL_STEP / 2 * cells / (launch_ms * 1e-3) / 1e12
    peak_tflops = 2 * FP64_LANES_PER_CLK_PER_SM * 152 * 2070e6 / 1e12
    instr_rate = FP64_INSTR_PER_CELL_STEP / 2 * cells / (launch_ms * 1e-3)
    hbm_gbs = BYTES_PER_CELL_STEP * cells * a.steps / (ms * 1e-3) / 1e9
    # the capture scales with the cells only while a plane set exceeds the L2
    plane_set_bytes = 16 * 8 * cells
    traffic = None
    if TRAFFIC_SHA == kernel_sha() and plane_set_bytes >= 1024 * 1024 * 128:
        traffic = TRAFFIC_BYTES_PER_LAUNCH * cells / 4096 ** 2
    # the end-to-end run right after the timed region, before the probe's FP64 load
    e2e_res = None if a.no_e2e else e2e(a, w, stream, cdbm, s, torch, local_rank)
    probe = fp64_peak(torch, cdbm, stream, local_rank)
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                "kernel": "stage_march_kernel (RK stages 1 and 2, mean per launch)",
                "peak_source": "FP64 pipe: 2 lanes/clk/SM x 152 SMs x 2070 MHz x 2 flops (recipe nominal 1.25 TFLOP/s)",
                "peak_measured": probe["tflops"], "frac_of_measured_peak": achieved_tflops / probe["tflops"],
                "peak_measured_source": "%s, %d x %d threads x 8 chains x %d FMAs, best of %d, this run"
                                        % (probe["kernel"], probe["launch"][0], probe["launch"][1],
                                           probe["launch"][2], probe["launches"]),
                "peak_measured_median": probe["tflops_median"], "peak_measured_clocks": probe["clocks"],
                "fp64_pipe_frac": instr_rate / peak_instr,
                "hbm_gbs": hbm_gbs, "hbm_frac_of_measured": hbm_gbs / measured_hbm()}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(a, w, world),
        "gpu_launches": 2 * a.steps,
        "clocks": clocks,
        "roofline": roofline,
        "decay_rate": decay,
    }

    if not a.no_aux:
        out["aux_kernels"] = aux_kernels(s, w, stream, torch, cdbm, 8, True)
    if e2e_res is not None:
        out["e2e"] = e2e_res
    s.close()

    if not a.no_variants and rank == 0:
        out["fp32_bulk"] = fp32_variant(a, w, torch, Solver, CDBM_FP32_BULK, (rho64, ux64, uy64, T64), value, amp0,
                                        "f in single precision as deviation from a reference "
                                        "equilibrium; sums, moment shift and equilibrium product in double")
        out["fp32_df64"] = fp32_variant(a, w, torch, Solver, CDBM_FP32_DF64, (rho64, ux64, uy64, T64), value, amp0,
                                        "as fp32_bulk, with sums, moment shift and equilibrium product in "
                                        "double-float arithmetic on the FP32 pipe")
        out["fp32_dev"] = fp32_variant(a, w, torch, Solver, CDBM_FP32_DEV, (rho64, ux64, uy64, T64), value, amp0,
                                       "all in single precision: the state as its deviation from the reference "
                                       "equilibrium and the equilibrium formed from the deviations of the moments "
                                       "(not the FP64 moment shift and product of fp32_bulk)")
        if a.full_steps > 0:
            out["config3_full"] = full_length_vortex(a, w, torch, Solver)
        if not a.no_ensemble:
            out["ensemble"] = ensemble(a, torch)
        if a.adj_steps > 0:
            out["adjoint"] = adjoint(a, torch)
        if not a.no_configs:
            out["configs"] = configs(a, torch)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, side=min(2048, w.nx))
        if a.cpu_configs:
            out["cpu_baseline"]["configs"] = cpu_configs()
    if rank == 0:
        print(json.dumps(out), flush=True)


def field_errors(got, ref, gamma, torch):
    """Per-field errors of (rho, ux, uy, T) against a reference run: relative L2 and
    max-norm of rho and T, velocity max-norm over max(|u|, c_s)."""
    rho, ux, uy, T = got
    r_rho, r_ux, r_uy, r_T = ref
    cs = float(torch.sqrt(gamma * r_T.mean()))
    us = max(float(r_ux.abs().max()), float(r_uy.abs().max()), cs)
    return {"rho_l2": float(torch.linalg.norm(rho - r_rho) / torch.linalg.norm(r_rho)),
            "rho_max": float((rho - r_rho).abs().max() / r_rho.abs().max()),
            "T_l2": float(torch.linalg.norm(T - r_T) / torch.linalg.norm(r_T)),
            "T_max": float((T - r_T).abs().max() / r_T.abs().max()),
            "u_max_over_scale": max(float((ux - r_ux).abs().max()), float((uy - r_uy).abs().max())) / us}


def fp32_variant(a, w, torch, Solver, precision, ref64, value64, amp0, note):
    """A single-precision state on the same vortex and steps: throughput, speed-up over
    the FP64 plain path, per-field errors against the FP64 run, decay rate."""
    from paper_2502_16818_gb300 import workloads as W
    rho64 = ref64[0]
    import numpy as np
    s, stream, _ = time_tgv(w, precision, a.steps, a.warmup, torch, Solver)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(a.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s.sync()
    rho, ux, uy, T = s.macros()
    from paper_2502_16818_gb300 import cdbm
    aux = None if a.no_aux else aux_kernels(s, w, stream, torch, cdbm, 4, False)
    s.close()
    l2 = float(torch.linalg.norm(rho - rho64) / torch.linalg.norm(rho64))
    errs = field_errors((rho, ux, uy, T), ref64, W.gamma_of(w.I), torch)
    val = w.nx * w.ny * a.steps / (ms * 1e-3)
    amp1 = tgv_amplitude(w, ux)
    return {"value": val, "unit": UNIT, "ms_per_step": ms / a.steps, "speedup_vs_fp64": val / value64,
            "l2_density_error_vs_fp64": l2, "field_errors_vs_fp64": errs, "steps_compared": a.steps + a.warmup,
            "decay_rate_measured": float(-np.log(amp1 / amp0) / (a.steps * w.dt)),
            "hbm_gbs": BYTES_PER_CELL_STEP_FP32 * w.nx * w.ny * a.steps / (ms * 1e-3) / 1e9,
            "hbm_frac_of_measured": BYTES_PER_CELL_STEP_FP32 * w.nx * w.ny * a.steps / (ms * 1e-3) / 1e9
                                    / measured_hbm(), "aux_kernels": aux, "note": note}


def full_length_vortex(a, w, torch, Solver):
    """The vortex run for its configured length (2000 steps, t = 0.01) in FP64,
    FP32_BULK, FP32_DF64 and FP32_DEV, whatever --steps is: each run timed as a whole, the
    Taylor-Green amplitude sampled every 100 steps, the decay rate fitted (least
    squares on log amplitude) over the last 1000 steps against the Navier-Stokes
    rate 2 nu k^2 with nu = T tau (Eqs. 22-23), and the per-field errors of the
    single-precision runs against the FP64 run at the last step."""
    import numpy as np
    from paper_2502_16818_gb300 import CDBM_FP32_BULK, CDBM_FP32_DEV, CDBM_FP32_DF64, CDBM_FP64, workloads as W
    steps = a.full_steps
    every = 100 if steps % 100 == 0 else steps
    k = w.extra["k"]
    x = (torch.arange(w.nx, dtype=torch.float64, device="cuda") + 0.5) * w.dx
    mode = torch.cos(k * x)[:, None] * torch.sin(k * x)[None, :]
    res = {"steps": steps, "t_end": steps * w.dt, "sample_every": every}
    finals = {}
    for label, prec in (("fp64", CDBM_FP64), ("fp32_bulk", CDBM_FP32_BULK), ("fp32_df64", CDBM_FP32_DF64),
                        ("fp32_dev", CDBM_FP32_DEV)):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = Solver.from_workload(w, stream=st, precision=prec)
            s.init(*(torch.from_numpy(v).to("cuda") for v in (w.rho, w.ux, w.uy, w.T)))
        s.sync()
        amps, ms = [], 0.0
        for _ in range(steps // every):
            with torch.cuda.stream(st):
                amps.append(float((s.macros()[1] * mode).sum()))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.step(every)
            e1.record(st)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        with torch.cuda.stream(st):
            fin = s.macros()
            amps.append(float((fin[1] * mode).sum()))
        s.sync()
        s.close()
        torch.cuda.synchronize()
        t = np.arange(len(amps)) * every * w.dt
        tail = t >= t[-1] - 0.5 * steps * w.dt - 1e-12
        rate = float(-np.polyfit(t[tail], np.log(np.abs(amps))[tail], 1)[0])
        nu = float(fin[3].mean()) * w.tau
        row = {"value": w.nx * w.ny * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
               "decay_rate_last_half": rate, "navier_stokes_2nuk2": 2 * nu * k * k,
               "decay_rate_rel_err": rate / (2 * nu * k * k) - 1.0}
        if label == "fp64":
            finals = fin
        else:
            row["field_errors_vs_fp64"] = field_errors(fin, finals, W.gamma_of(w.I), torch)
            row["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / row["ms_per_step"]
        res[label] = row
        del fin
    return res


def ensemble(a, torch):
    """1024 shock tubes, Nx ~ U{200..4000} (seed 0), one persistent autotuned launch
    per call, FP64, FP32-bulk, FP32 with the df64 equilibrium and FP32 with the
    single-precision deviation equilibrium; against a per-tube
    loop of the single-grid FP64 solver over the same tubes."""
    from paper_2502_16818_gb300 import BatchSolver, Solver, workloads as W
    specs = W.ensemble_draw(1024, seed=0)
    tubes = [W.ensemble_tube(sp, steps=1000) for sp in specs]
    res = {"tubes": len(tubes), "cells": int(sum(w.nx for w in tubes)), "steps": a.ens_steps}
    for name, prec in (("fp64_batched", 0), ("fp32_bulk_batched", 1), ("fp32_df64_batched", 2),
                       ("fp32_dev_batched", 3)):
        st = torch.cuda.Stream()
        b = BatchSolver(tubes, precision=prec, stream=st)
        b.init(tubes)
        tile = b.autotune(5)
        b.step(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.step(a.ens_steps)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        b.sync()
        b.close()
        per = BYTES_PER_CELL_STEP if prec == 0 else BYTES_PER_CELL_STEP_FP32
        gbs = per * res["cells"] * a.ens_steps / (ms * 1e-3) / 1e9
        res[name] = {"value": res["cells"] * a.ens_steps / (ms * 1e-3), "unit": UNIT, "tile": tile,
                     "gpu_launches": 1, "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / measured_hbm(),
                     "bytes_per_cell_step": per}
    # per-tube loop: one single-grid FP64 solver per tube, stepped one after another
    st = torch.cuda.Stream()
    solvers = []
    for w in tubes:
        s = Solver.from_workload(w, stream=st)
        s.init(w.rho, w.ux, w.uy, w.T)
        solvers.append(s)
    loop_steps = 32
    for s in solvers:
        s.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for s in solvers:
        s.step(loop_steps)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    for s in solvers:
        s.sync()
        s.close()
    res["fp64_per_tube_loop"] = {"value": res["cells"] * loop_steps / (ms * 1e-3), "unit": UNIT,
                                 "steps": loop_steps, "gpu_launches": 2 * loop_steps * len(tubes)}
    res["batched_fp32_vs_fp64_plain_loop"] = res["fp32_bulk_batched"]["value"] / res["fp64_per_tube_loop"]["value"]
    res["batched_df64_vs_fp64_plain_loop"] = res["fp32_df64_batched"]["value"] / res["fp64_per_tube_loop"]["value"]
    return res


def configs(a, torch):
    """Wall time of the paper-scale configurations on the GPU (CUDA events around the
    whole run, state resident): Sod (500 cells, 10^4 steps), Lax (2000 cells, 10^4
    steps) and the 512^2 sound wave for I = 0, 1, 3 (2000 steps), in FP64 and with
    the single-precision state and the df64 or the single-precision deviation
    equilibrium."""
    from paper_2502_16818_gb300 import CDBM_FP32_DEV, CDBM_FP32_DF64, CDBM_FP64, Solver, workloads as W
    runs = [("sod_500_I0", W.sod(nx=500, I=0.0), 10000), ("lax_2000_I0", W.lax(nx=2000, I=0.0), 10000)]
    runs += [("sound_512_I%d" % I, W.sound(n=512, I=float(I)), 2000) for I in (0, 1, 3)]
    res = {}
    for name, w, steps in runs:
        row = {"cells": w.nx * w.ny, "steps": steps}
        for label, prec in (("fp64", CDBM_FP64), ("fp32_df64", CDBM_FP32_DF64), ("fp32_dev", CDBM_FP32_DEV)):
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                s = Solver.from_workload(w, stream=st, precision=prec)
                s.init(*(torch.from_numpy(x).to("cuda") for x in (w.rho, w.ux, w.uy, w.T)))
                s.step(64)
                s.init(*(torch.from_numpy(x).to("cuda") for x in (w.rho, w.ux, w.uy, w.T)))
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.step(steps)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            s.sync()
            s.close()
            per = BYTES_PER_CELL_STEP if prec == CDBM_FP64 else BYTES_PER_CELL_STEP_FP32
            gbs = per * row["cells"] * steps / (ms * 1e-3) / 1e9
            row[label] = {"run_ms": ms, "value": row["cells"] * steps / (ms * 1e-3), "unit": UNIT,
                          "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / measured_hbm()}
        res[name] = row
    return res


def adjoint(a, torch):
    """Gradient of L = sum (rho_T - rho_target)^2 with respect to the initial rho, T
    (and u) fields and tau on the periodic sound-mode case: forward run storing a
    checkpoint every `every` steps, then the reverse sweep (segment recomputation
    and the adjoint stage kernels), with the frozen limiter linearisation (the exact
    one grows without bound over this horizon).  Throughput counts the forward
    cell-updates over the time of forward plus backward."""
    from paper_2502_16818_gb300 import Solver, cdbm, workloads as W
    w = W.sound_modes(n=a.adj_n, seed=0, kmax=8, steps=a.adj_steps)
    target = torch.from_numpy(W.sound_modes(n=a.adj_n, seed=1, kmax=8).rho).to("cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = Solver.from_workload(w, stream=st)
        s.init(*(torch.from_numpy(x).to("cuda") for x in (w.rho, w.ux, w.uy, w.T)))
        cdbm.cdbm_adjoint_set_limiter(s.ctx, cdbm.CDBM_ADJ_LIMITER_FROZEN)
        grads = [torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        fbar = torch.empty((16, w.ny, w.nx), dtype=torch.float64, device="cuda")
    s.sync()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t0 = time.perf_counter()
    ev[0].record(st)
    cdbm.cdbm_adjoint_forward(s.ctx, a.adj_steps, a.adj_every)
    ev[1].record(st)
    with torch.cuda.stream(st):
        rho = s.macros()[0]
        grho = 2.0 * (rho - target)
        loss = float(((rho - target) ** 2).sum())
    cdbm.cdbm_macros_vjp(s.ctx, grho.data_ptr(), 0, 0, 0, fbar.data_ptr())
    gtau = cdbm.cdbm_adjoint_backward(s.ctx, fbar.data_ptr(), *(g.data_ptr() for g in grads))
    ev[2].record(st)
    ev[2].synchronize()
    wall = time.perf_counter() - t0
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    s.close()
    cells = w.nx * w.ny
    fwd_gbs = (BYTES_PER_CELL_STEP * a.adj_steps + 128 * (a.adj_steps // a.adj_every)) * cells / (fwd_ms * 1e-3) / 1e9
    bwd_gbs = BYTES_PER_CELL_STEP_ADJ_BWD * a.adj_steps * cells / (bwd_ms * 1e-3) / 1e9
    return {"value": cells * a.adj_steps / ((fwd_ms + bwd_ms) * 1e-3), "unit": UNIT,
            "workload": "sound_modes_%dx%d_kmax8_fp64" % (w.nx, w.ny), "steps": a.adj_steps,
            "checkpoint_every": a.adj_every, "limiter": "frozen", "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "backward_over_forward": bwd_ms / fwd_ms, "wall_s": wall, "loss": loss, "dL_dtau": gtau,
            "grad_rho_l2": float(torch.linalg.norm(grads[0])), "grad_T_l2": float(torch.linalg.norm(grads[3])),
            "checkpoint_bytes": 128 * cells * (a.adj_steps // a.adj_every + 1),
            "forward_hbm_gbs": fwd_gbs, "forward_hbm_frac_of_measured": fwd_gbs / measured_hbm(),
            "backward_hbm_gbs": bwd_gbs, "backward_hbm_frac_of_measured": bwd_gbs / measured_hbm(),
            "bytes_per_cell_step": {"forward": BYTES_PER_CELL_STEP, "backward": BYTES_PER_CELL_STEP_ADJ_BWD}}


def aux_kernels(s, w, stream, torch, cdbm, state_bytes, with_init, reps=10):
    """The on-demand kernels on the resident vortex state, each call timed with CUDA
    events on the solver's stream (mean of `reps` after one untimed call), with the
    HBM GB/s of its algorithmic bytes per cell: init from device fields (reads rho,
    u, T: 32 B; writes the 16 planes), macros (reads the planes, writes rho, u, T:
    32 B), Delta* (reads the planes, writes 12 doubles: 96 B; it rebuilds the
    central moments of every cell from its raw moments) and the conserved sums
    (reads the planes; a synchronous call that returns 4
    doubles).  Delta*, macros and the sums are bound by the FP64 pipe at these
    byte counts (167, 51 and 22 FP64 instructions per cell on the FP64 state).  state_bytes:
    bytes per stored value (8 for FP64, 4 for the single-precision states)."""
    cells = w.nx * w.ny
    planes = 16 * state_bytes
    with torch.cuda.stream(stream):
        fields = [torch.from_numpy(x).to("cuda") for x in (w.rho, w.ux, w.uy, w.T)]
        outs = [torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        tne = torch.empty((12, w.ny, w.nx), dtype=torch.float64, device="cuda")
    stream.synchronize()
    calls = [("macros_kernel", planes + 32, lambda: cdbm.cdbm_macros(s.ctx, *(o.data_ptr() for o in outs))),
             ("tne_kernel (Delta*)", planes + 96, lambda: cdbm.cdbm_tne(s.ctx, tne.data_ptr())),
             ("sums_partial_kernel + sums_final_kernel (conserved sums)", planes,
              lambda: cdbm.cdbm_conserved_sums(s.ctx))]
    if with_init:
        calls.insert(0, ("init_kernel", 32 + planes, lambda: cdbm.cdbm_init(s.ctx, *(f.data_ptr() for f in fields))))
    res = {}
    for name, per_cell, call in calls:
        call()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = per_cell * cells / (ms * 1e-3) / 1e9
        res[name.split(" ")[0]] = {"kernel": name, "ms": ms, "bytes_per_cell": per_cell, "hbm_gbs": gbs,
                                   "hbm_frac_of_measured": gbs / measured_hbm()}
    return res


def e2e(a, w, stream, cdbm, s, torch, local_rank=0):
    """Same metric through the C ABI with host buffers: pinned host fields are
    uploaded by cdbm_init, K steps run, and cdbm_macros downloads rho, u, T to
    pinned host memory, all inside the timed region (clocks sampled meanwhile)."""
    host_in = [torch.from_numpy(x).pin_memory() for x in (w.rho, w.ux, w.uy, w.T)]
    host_out = [torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    cells = w.nx * w.ny
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    cdbm.cdbm_init(s.ctx, *(h.data_ptr() for h in host_in))
    cdbm.cdbm_step(s.ctx, a.steps)
    cdbm.cdbm_macros(s.ctx, *(h.data_ptr() for h in host_out))
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    ms = max(e0.elapsed_time(e1), wall * 1e3)
    cdbm.cdbm_sync(s.ctx)
    nbytes = 4 * 8 * cells
    return {"value": cells * a.steps / (ms * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": nbytes / a.steps, "d2h_bytes_per_step": nbytes / a.steps,
            "job": "upload rho,u,T -> cdbm_init -> %d steps -> cdbm_macros to host" % a.steps, "clocks": clocks}


def measured_hbm():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        return 6793.1     # the driver's measurement of this machine's GB300 copy bandwidth


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_cdbm(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
