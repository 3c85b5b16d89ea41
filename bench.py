"""Benchmark: FAS cycles of the preconditioned AW3 smoother on the 256x64 thin-layer RANS
C-grid workload (M = 0.5, Re = 1e7, wall spacing 1e-5, 4-level W-cycle, Baldwin-Lomax).

One step = one FAS cycle over the whole grid (all steps of the method's hot path).  Prints
one JSON line.  Metric: Mcell-iterations/s (fine cells x cycles / s), plus the wall time to a
6-order residual drop for the FP64 and the mixed-precision preconditioner.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision fp64|mixed]

Multi-GPU: the exact method does not shard (the SGS sweep is one global wavefront), so N GPUs
run N independent replicas of the same case; value = all ranks' cell-iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth.cgrid import make_cgrid  # noqa: E402

WORKLOAD = dict(name="rans_256x64_thin_layer_bl", ni=256, nj=64, n_wake=32, wall_spacing=1e-5,
                mach=0.5, alpha_deg=0.0, re=1e7, nlevels=4, gamma_cycle=2, scheme="AW3", eta=0.8,
                d_cut=0.5, cfl=100.0, cfl_ramp=20.0, ramp_cycles=2, viscous=1, turb=1)
METRIC = "Mcell-iter/s"
L2_FLUSH_BYTES = 256 << 20
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak from unit counts and clock: 152 SMs x 4 FP64 flop/clk (2 DFMA) x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# algorithmic FP64 flops per cell and launch, counted from the kernels (FMA = 2)
FLOPS_PER_CELL = {"sgs": 230.0, "residual": 310.0, "face_blocks": 380.0, "diag_blocks": 100.0}
# DRAM bytes per cell of one FP64 strip-sweep launch (dram__bytes_read.sum + write, cold caches):
# 11.6 MB for the 16,384 cells of the finest 256x64 level (profiles/sweep_strips_fp64_dram_rans_256x64.md);
# the traffic is the transfer blocks and vectors of each cell, so it scales with the cells
SWEEP_DRAM_BYTES_PER_CELL = 11.6e6 / 16384


def level_visits(nlevels, gamma):
    """Smoothing visits per cycle of each level (index 0 = coarsest) for a V (1) / W (2) cycle."""
    v = [0] * nlevels
    def rec(l):
        v[l] += 1
        if l > 0:
            for _ in range(gamma):
                rec(l - 1)
    rec(nlevels - 1)
    return v


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the slowest rank's time); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ncell, steps, world, tot_ms):
    """Mcell-iter/s of the whole job: every rank's cells and cycles over the slowest rank's time."""
    return world * ncell * steps / (tot_ms / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[3 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_grid():
    w = WORKLOAD
    return make_cgrid(w["ni"], w["nj"], n_wake=w["n_wake"], wall_spacing=w["wall_spacing"])


def gpu_params(P, precision):
    w = WORKLOAD
    return P.default_params(scheme=w["scheme"], nlevels=w["nlevels"], gamma_cycle=w["gamma_cycle"],
                            viscous=w["viscous"], turb=w["turb"],
                            sensor=1, mach=w["mach"], alpha_deg=w["alpha_deg"], re=w["re"], eta=w["eta"],
                            d_cut=w["d_cut"], cfl=w["cfl"], cfl_ramp=w["cfl_ramp"], ramp_cycles=w["ramp_cycles"],
                            precision=precision)


def oracle_solver():
    import oracle as O
    w = WORKLOAD
    p = O.make_params(w["scheme"], nlevels=w["nlevels"], gamma_cycle=w["gamma_cycle"], viscous=w["viscous"],
                      turb=w["turb"], sensor=1,
                      mach=w["mach"], alpha_deg=w["alpha_deg"], re=w["re"], eta=w["eta"], d_cut=w["d_cut"],
                      cfl=w["cfl"], cfl_ramp=w["cfl_ramp"], ramp_cycles=w["ramp_cycles"])
    return O.Oracle(workload_grid(), p)


def cpu_oracle_sample(budget_s=12.0, max_cycles=400, min_cycles=3):
    """Time the oracle (as it stands, one host thread) on consecutive cycles of the workload."""
    o = oracle_solver()
    ncell = WORKLOAD["ni"] * WORKLOAD["nj"]
    t0 = time.perf_counter()
    k = 0
    while k < max_cycles and (k < min_cycles or time.perf_counter() - t0 < budget_s):
        o.fas_cycle(k)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": ncell * k / dt / 1e6, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{k} FAS cycles of the 256x64 RANS workload from the free stream, single thread, "
                      f"{dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    ncell = WORKLOAD["ni"] * WORKLOAD["nj"]
    o = oracle_solver()
    for k in range(args.warmup):
        o.fas_cycle(k)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        o.fas_cycle(args.warmup + k)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ncell * args.steps / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD["name"], "cells": ncell, "levels": WORKLOAD["nlevels"],
                                             "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed FAS cycles after {args.warmup} warm-up cycles, "
                                       "single host thread"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_cycles(s, stream, flush, steps, k0):
    """Device time of `steps` FAS cycles (CUDA events on the solver's stream), L2 flushed
    between cycles outside the timed intervals.  Returns per-cycle ms."""
    import torch
    ms = []
    for k in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.fas_cycle(k0 + k)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def measure_c3(P, stream, flush, steps, warmup):
    """W-cycle device time on the 512 x 128 C-grid of the pitching case (thin-layer RANS with
    Baldwin-Lomax, M 0.8, Re 1e6, 4 levels), FP64 and mixed precision, from the free stream."""
    from synth.cases import config_c3
    c = config_c3()
    g = c.grid()
    out = {"cells": g.ni * g.nj}
    for prec in ("fp64", "mixed"):
        p = P.default_params(scheme="AW3", nlevels=4, gamma_cycle=2, viscous=1, turb=1, sensor=1, mach=c.mach,
                             alpha_deg=0.0, re=c.reynolds, eta=0.8, d_cut=0.5, cfl=100.0, cfl_ramp=20.0,
                             ramp_cycles=2, precision=prec)
        s = P.Solver(g, p, stream=stream.cuda_stream)
        for k in range(warmup):
            s.fas_cycle(k)
        ms = time_cycles(s, stream, flush, steps, warmup)
        out[prec] = {"ms_per_cycle": sum(ms) / len(ms), "value": g.ni * g.nj * len(ms) / (sum(ms) / 1e3) / 1e6,
                     "unit": METRIC}
        s.close()
    return out


def measure_adjoint(s, g, n_bumps=16):
    """Discrete adjoint of the steady RANS workload at its 6-order state (eddy viscosity
    frozen): Jacobian assembly, the GMRES adjoint solve for C_D, and the shape gradient of C_D
    for 16 Hicks-Henne bumps, each timed on the host around synchronous library calls."""
    from synth.shape import bump_fields
    V = bump_fields(g, n_bumps)
    t0 = time.perf_counter()
    s.adjoint_jacobian(1e-6)
    t_jac = time.perf_counter() - t0
    t0 = time.perf_counter()
    lam, code, it, rr = s.adjoint_solve(1, tol=1e-8, max_iters=1000, restart=250)
    t_sol = time.perf_counter() - t0
    t0 = time.perf_counter()
    grad = s.adjoint_shape_gradient(1, lam, V)
    t_grad = time.perf_counter() - t0
    t0 = time.perf_counter()
    gx, gy = s.adjoint_vertex_gradient(1, lam)
    t_vert = time.perf_counter() - t0
    via = np.array([np.sum(gy * V[k]) for k in range(n_bumps)])
    cl, cd = s.force_coefficients()
    return {"objective": "C_D", "cl": cl, "cd": cd, "jacobian_s": t_jac, "solve_s": t_sol,
            "gmres_iterations": it, "relative_residual": rr, "status": int(code), "shape_gradient_s": t_grad,
            "vertex_gradient_s": t_vert,
            "vertex_vs_shape_gradient": float(np.abs(via - grad).max() / max(np.abs(grad).max(), 1e-300)),
            "n_params": n_bumps, "grad_norm": float(np.linalg.norm(grad)),
            "note": "steady state after the 6-order drop; eddy viscosity frozen; flexible GMRES(250), tol 1e-8, "
                    "preconditioned by the transposed linearised W-cycle"}


def measure_c5(P, stream=None, n_bumps=16):
    """The 1024x256 RANS sensitivity case (wall spacing 1e-5, M 0.75, Re 6.5e6, alpha 0, 5-level
    W-cycles of AW3, mixed precision): time to a 6-order drop from the free stream, then the
    C_D adjoint (eddy viscosity frozen) to a 6-order drop and the shape gradient for 16
    Hicks-Henne bumps; host-timed around the synchronous library calls."""
    from synth.shape import bump_fields
    g = make_cgrid(1024, 256, n_wake=128, wall_spacing=1e-5)
    p = P.default_params(scheme="AW3", nlevels=5, gamma_cycle=2, viscous=1, turb=1, sensor=1, mach=0.75,
                         alpha_deg=0.0, re=6.5e6, eta=0.8, d_cut=0.5, cfl=100.0, cfl_ramp=20.0, ramp_cycles=2,
                         precision="mixed")
    s = P.Solver(g, p, stream=stream.cuda_stream if stream is not None else None)
    t0 = time.perf_counter()
    code, nc, hist = s.solve(1e-6, 3000)
    t_primal = time.perf_counter() - t0
    out = {"workload": "rans_1024x256_c5", "cells": g.ni * g.nj, "levels": 5, "precision": "mixed",
           "primal_status": int(code), "primal_cycles": nc, "primal_s": t_primal,
           "primal_drop": float(hist[-1] / hist[0]) if len(hist) else None}
    if code != 0:
        s.close()
        return out
    V = bump_fields(g, n_bumps)
    t0 = time.perf_counter()
    s.adjoint_jacobian(1e-6)
    out["jacobian_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    lam, acode, it, rr = s.adjoint_solve(1, tol=1e-6, max_iters=1500, restart=250)
    out.update(adjoint_status=int(acode), gmres_iterations=it, relative_residual=rr,
               adjoint_s=time.perf_counter() - t0)
    t0 = time.perf_counter()
    grad = s.adjoint_shape_gradient(1, lam, V)
    t_grad = time.perf_counter() - t0
    t0 = time.perf_counter()
    gx, gy = s.adjoint_vertex_gradient(1, lam)
    t_vert = time.perf_counter() - t0
    via = np.array([np.sum(gy * V[k]) for k in range(n_bumps)])
    half = n_bumps // 2
    out.update(shape_gradient_s=t_grad, vertex_gradient_s=t_vert, n_params=n_bumps, cd=s.force_coefficients()[1],
               grad=[float(x) for x in grad],
               vertex_vs_shape_gradient=float(np.abs(via - grad).max() / max(np.abs(grad).max(), 1e-300)),
               upper_lower_antisymmetry=float(np.abs(grad[:half] + grad[half:2 * half]).max()
                                              / max(np.abs(grad).max(), 1e-300)))
    s.close()
    return out


def measure_c5_unsteady(P, n_bumps=16):
    """The unsteady part of the sensitivity case: the pitching motion of the 512x128 RANS case
    (M 0.8, Re 1e6, alpha = 2 deg sin(2kt), k = 0.2, 64 steps per period) over two periods (128
    levels), each level to a 3-order pseudo-time drop, every level stored; time-averaged C_D
    and its shape gradient for 16 bumps with the steady start's own adjoint (eddy viscosity
    frozen per level), mixed precision.  Host-timed around the synchronous library calls."""
    from synth.cases import config_c3
    from synth.shape import bump_fields
    from paper_1710_04875_gb300.adjoint import pitching_gradient
    c = config_c3()
    g = c.grid()
    p = P.default_params(scheme="AW3", nlevels=4, gamma_cycle=2, viscous=1, turb=1, sensor=1, mach=c.mach,
                         alpha_deg=0.0, re=c.reynolds, eta=0.8, d_cut=0.5, cfl=100.0, cfl_ramp=20.0, ramp_cycles=2,
                         precision="mixed")
    s = P.Solver(g, p)
    t0 = time.perf_counter()
    code, nc, hist = s.solve(1e-6, 2000)
    t_steady = time.perf_counter() - t0
    omega = 0.4
    dt = 2.0 * np.pi / omega / 64
    t0 = time.perf_counter()
    J, grad, info = pitching_gradient(s, bump_fields(g, n_bumps), np.radians(2.0), omega, dt, 128, which=1,
                                      snapshots=None, drop=1e-3, max_cycles=400, tol=1e-6, max_iters=1500,
                                      restart=250)
    t = time.perf_counter() - t0
    s.close()
    return {"workload": "rans_512x128_pitching_2_periods", "cells": g.ni * g.nj, "time_levels": 128,
            "precision": "mixed", "steady_start_status": int(code), "steady_start_cycles": nc,
            "steady_start_s": t_steady, "J": J, "seconds": t, "seconds_per_time_level": t / 128,
            "grad": [float(x) for x in grad], **info}


def adjoint_profile(P, iters=30):
    """One adjoint GMRES(250) solve of C_D with a fixed count of iterations on the workload grid
    (FP64, thin-layer RANS, frozen eddy viscosity) at a smoothly perturbed free stream, so that
    a kernel-filtered ncu launch list of this process shows the adjoint's kernels only."""
    g = workload_grid()
    s = P.Solver(g, gpu_params(P, "fp64"))
    u = s.get_state()
    jj, ii = np.meshgrid(np.arange(g.nj), np.arange(g.ni), indexing="ij")
    u = u * (1.0 + 0.02 * np.sin(2 * np.pi * ii / g.ni) * np.cos(np.pi * jj / g.nj))[None]
    s.set_state(np.ascontiguousarray(u))
    s.adjoint_jacobian(1e-6)
    t0 = time.perf_counter()
    lam, code, it, rr = s.adjoint_solve(1, tol=1e-14, max_iters=iters, restart=250)
    t = time.perf_counter() - t0
    s.close()
    return {"adjoint_profile": WORKLOAD["name"], "gmres_iterations": it, "seconds": t,
            "ms_per_iteration": 1e3 * t / max(it, 1), "relative_residual": rr}


def measure_unsteady_adjoint(P, stream, nsteps=128, snapshots=8, n_bumps=16):
    """Unsteady adjoint of the pitching motion (alpha = 2 deg sin(2kt), k = 0.2, 64 steps per
    period) over two periods, with binomial checkpointing of the reverse sweep: time-averaged
    C_D and its gradient for 16 Hicks-Henne bumps, on a 128 x 32 Euler C-grid (M 0.6, two-level
    V-cycles; three levels stall on this case), from the steady solution; timed on the host
    around the synchronous library calls."""
    from synth.shape import bump_fields
    from paper_1710_04875_gb300.adjoint import pitching_gradient
    g = make_cgrid(128, 32, wall_spacing=2e-3)
    p = P.default_params(scheme="AW3", nlevels=2, gamma_cycle=1, mach=0.6, alpha_deg=0.0, cfl=1e4,
                         precision="mixed")
    s = P.Solver(g, p, stream=stream.cuda_stream)
    code, nc, hist = s.solve(1e-10, 1500)
    omega = 0.4
    dt = 2.0 * np.pi / omega / 64
    t0 = time.perf_counter()
    J, grad, info = pitching_gradient(s, bump_fields(g, n_bumps), np.radians(2.0), omega, dt, nsteps, which=1,
                                      snapshots=snapshots, drop=1e-8, max_cycles=500, tol=1e-8, max_iters=600,
                                      restart=250)
    t = time.perf_counter() - t0
    s.close()
    return {"workload": "euler_128x32_pitching_2_periods", "precision": "mixed (FP32 preconditioners)",
            "cells": g.ni * g.nj, "time_levels": nsteps,
            "stored_levels": snapshots, "objective": "time-averaged C_D", "J": J, "n_params": n_bumps,
            "grad_norm": float(np.linalg.norm(grad)), "seconds": t, "seconds_per_time_level": t / nsteps,
            "steady_start_status": int(code), "steady_start_cycles": nc,
            "steady_start_drop": float(hist[-1] / hist[0]) if len(hist) else None, **info,
            "store_all_forward_steps": nsteps,
            "note": "per-level pseudo-time drop 1e-8, adjoint GMRES(250) to 1e-8; gradient includes the "
                    "steady adjoint of the initial state"}


def measure_batched(P, stream, flush, steps, warmup, precision="mixed"):
    """64 uneven Euler cases (128x32 .. 512x128 cells, seeded M, alpha, thickness) advanced
    together, one captured CUDA graph per cycle; sweep variants chosen by the autotuner."""
    import torch
    from synth.cases import config_c4_cases
    cases = config_c4_cases()
    grids, params = [], []
    for c in cases:
        grids.append(c.grid())
        params.append(P.default_params(scheme="AW3", nlevels=c.levels, mach=c.mach, alpha_deg=c.alpha_deg,
                                       cfl=100.0, precision=precision))
    cells = sum(g.ni * g.nj for g in grids)
    b = P.fasw.Batch(grids, params, stream=stream.cuda_stream)
    choice = b.autotune()
    for k in range(warmup):
        b.cycle(k)
    ms = []
    for k in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.cycle(warmup + k)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    value = cells * steps / (sum(ms) / 1e3) / 1e6
    b.close()
    b = P.fasw.Batch(grids, params, stream=stream.cuda_stream)
    b.autotune()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    code, cyc, drops, ncy = b.solve(1e-6, 300)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    b.close()
    return {"cases": len(grids), "cells": cells, "precision": precision, "value": value, "unit": METRIC,
            "ms_per_cycle": sum(ms) / steps,
            "sweep_choice": {"staged8": choice.count(7), "staged4": choice.count(6), "staged": choice.count(5),
                             "cta": choice.count(2)},
            "time_to_6_orders": {"seconds": dt, "cycles_run": ncy, "status": int(code),
                                 "cases_converged": int((cyc > 0).sum()), "cases_diverged": int((cyc == -2).sum()),
                                 "median_cycles": float(np.median(cyc[cyc > 0])) if (cyc > 0).any() else None}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-unsteady-adjoint", action="store_true")
    ap.add_argument("--c5", action="store_true",
                    help="only the 1024x256 RANS shape-sensitivity case (steady solve, adjoint, 16 bump gradients)")
    ap.add_argument("--c5-unsteady", action="store_true",
                    help="only the two-period unsteady adjoint of the pitching 512x128 RANS case (minutes)")
    ap.add_argument("--adjoint-profile", action="store_true",
                    help="only one 30-iteration adjoint GMRES solve on the workload grid (for ncu launch lists)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1710_04875_gb300 as P

    if args.adjoint_profile:
        print(json.dumps(adjoint_profile(P)), flush=True)
        return
    if args.c5:
        print(json.dumps(measure_c5(P)), flush=True)
        return
    if args.c5_unsteady:
        print(json.dumps(measure_c5_unsteady(P)), flush=True)
        return

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()          # non-default stream: cycles are replayed as CUDA graphs
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    g = workload_grid()
    ncell = g.ni * g.nj
    s = P.Solver(g, gpu_params(P, args.precision), stream=stream.cuda_stream)

    # warm-up cycles (untimed) from the free stream
    for k in range(args.warmup):
        s.fas_cycle(k)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = s.launch_count()
    with ClockSampler(local) as clk:
        ms = time_cycles(s, stream, flush, args.steps, args.warmup)
    launches = (s.launch_count() - l0) // max(args.steps, 1) * args.steps
    torch.cuda.synchronize()
    tot_ms = max_over_ranks(float(sum(ms)), dist, "cuda")
    if dist:
        dist.barrier()
    value = whole_job_value(ncell, args.steps, world, tot_ms)

    # same measurement with the mixed-precision preconditioner (FP32 blocks / sweeps)
    sm = P.Solver(g, gpu_params(P, "mixed" if args.precision == "fp64" else "fp64"), stream=stream.cuda_stream)
    for k in range(args.warmup):
        sm.fas_cycle(k)
    ms_other = time_cycles(sm, stream, flush, args.steps, args.warmup)
    other_value = world * ncell * args.steps / (sum(ms_other) / 1e3) / 1e6
    sm.close()

    # the 512x128 pitching-airfoil grid (M 0.8, Re 1e6): W-cycle throughput of both precisions
    c3 = measure_c3(P, stream, flush, min(args.steps, 10), args.warmup)

    # per-kernel device time over a second pass of the same number of cycles
    s.profile(True)
    for k in range(args.steps):
        flush.zero_()
        s.fas_cycle(args.warmup + args.steps + k)
    kt = {name: s.kernel_time(i) for i, name in enumerate(P.fasw.KERNEL_CLASSES)}
    s.profile(False)

    # e2e through the public API with host buffers: per cycle, H2D of the state from pinned
    # memory, one cycle, D2H of the new state and the residual norm
    u_host = torch.from_numpy(s.get_state()).pin_memory()
    u_out = torch.empty_like(u_host).pin_memory()
    e2e_steps = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        s.set_state(u_host.numpy())
        s.fas_cycle(10**6)
        s.get_state(out=u_out.numpy())
    e2e_s = time.perf_counter() - t0
    e2e_value = world * ncell * e2e_steps / e2e_s / 1e6
    state_bytes = 4 * ncell * 8

    # time to a 6-order drop from the free stream, FP64 and mixed preconditioner; then the
    # pitching motion (alpha = 2 deg sin(2kt), k = 0.2, 64 steps per period): an implicit-Euler
    # start step and one BDF2 step, each to an 11-order drop in pseudo time
    drops, unsteady = {}, {}
    states6, states11, final6, final11 = {}, {}, {}, {}
    adjoint = None
    omega = 0.4
    dt_phys = 2.0 * np.pi / omega / 64
    amp = np.radians(2.0)
    for prec in ("fp64", "mixed"):
        sd = P.Solver(g, gpu_params(P, prec), stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, nc, hist = sd.solve(1e-6, 600)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        drops[prec] = {"seconds": dt if code == 0 else None, "cycles": nc, "status": int(code),
                       "final_drop": float(hist[-1] / hist[0]) if len(hist) else None}
        states6[prec] = sd.get_state()
        final6[prec] = float(hist[-1]) if len(hist) else None
        if not args.no_adjoint:
            adjoint = adjoint or {}
            adjoint[prec] = measure_adjoint(sd, g)
        steps = []
        for step in (1, 2):
            tt = step * dt_phys
            sd.set_motion(-amp * np.sin(omega * tt), -amp * omega * np.cos(omega * tt))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2, n2, h2 = sd.dual_time_step(dt_phys, 1e-11, 1000)
            torch.cuda.synchronize()
            steps.append({"kind": "implicit Euler" if step == 1 else "BDF2", "seconds": time.perf_counter() - t0,
                          "cycles": n2, "status": int(c2),
                          "final_drop": float(h2[-1] / h2[0]) if len(h2) else None})
        unsteady[prec] = steps
        states11[prec] = sd.get_state()
        final11[prec] = float(h2[-1]) if len(h2) else None
        sd.close()

    def gap(st):
        return float(np.linalg.norm(st["mixed"] - st["fp64"]) / np.linalg.norm(st["fp64"]))
    precision_gap = {"state_6_orders": gap(states6), "state_11_orders_second_pitching_step": gap(states11),
                     "final_residual_6_orders": final6, "final_residual_11_orders": final11,
                     "note": "||u_mixed - u_fp64|| / ||u_fp64|| after the same number of cycles, and the RMS "
                             "density residual at the stop of each precision"}
    batched = None if args.no_batched else measure_batched(P, stream, flush, args.steps, args.warmup)
    unsteady_adjoint = None if (args.no_adjoint or args.no_unsteady_adjoint) else measure_unsteady_adjoint(P, stream)
    c5 = None if args.no_adjoint else measure_c5(P, stream)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel class: algorithmic FP64 flops per cell of each class
    # (counted from the kernels) x cells processed per launch / average launch time
    dom = max(kt, key=lambda k: kt[k][1])
    n_l, ms_l = kt[dom]
    avg_ms = ms_l / max(n_l, 1)
    visits = level_visits(WORKLOAD["nlevels"], WORKLOAD["gamma_cycle"])
    cells = [ncell // (4 ** (WORKLOAD["nlevels"] - 1 - l)) for l in range(WORKLOAD["nlevels"])]
    per_cycle_cells = {
        "sgs": sum(3 * visits[l] * cells[l] for l in range(len(cells))),
        "residual": sum(3 * visits[l] * cells[l] for l in range(len(cells)))
        + sum(visits[l] * cells[l] for l in range(1, len(cells)))
        + sum(visits[l] * cells[l] for l in range(0, len(cells) - 1)),
        "face_blocks": sum(visits[l] * cells[l] for l in range(len(cells))),
        "diag_blocks": sum(visits[l] * cells[l] for l in range(len(cells))),
    }
    if dom in FLOPS_PER_CELL:
        cells_per_launch = per_cycle_cells[dom] / (n_l / (2 * args.steps) * 2)
        achieved = FLOPS_PER_CELL[dom] * cells_per_launch / (avg_ms / 1e3) / 1e12
        traffic = SWEEP_DRAM_BYTES_PER_CELL * cells_per_launch if dom == "sgs" else None
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "traffic_source": "ncu dram bytes of a finest-level launch (708 B/cell), scaled by cells" if traffic else None,
                "avg_launch_ms": avg_ms,
                "launches_per_cycle": n_l / args.steps, "cells_per_launch": cells_per_launch,
                "flops_per_cell": FLOPS_PER_CELL[dom],
                "peak_source": "FP64 from unit counts and clock (152 SMs x 4 flop/clk x 2.07 GHz)"}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "avg_launch_ms": avg_ms}
    share = {k: round(v[1] / max(sum(x[1] for x in kt.values()), 1e-12), 4) for k, v in kt.items()}
    cpu = None if args.no_cpu_baseline else cpu_oracle_sample()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "cells": ncell, "levels": WORKLOAD["nlevels"],
                       "cycle": "W", "scheme": "AW3", "precision": args.precision, "cfl": WORKLOAD["cfl"],
                       "l2": "flushed (256 MiB write) between timed cycles", "parallelism": "replicas"},
            "other_precision": {"precision": "mixed" if args.precision == "fp64" else "fp64",
                                "value": other_value, "ms_per_step": sum(ms_other) / args.steps},
            "time_to_6_orders": drops, "time_to_11_orders_per_time_step": unsteady, "precision_gap": precision_gap,
            "batched_64_cases": batched, "c3_512x128": c3, "adjoint": adjoint,
            "unsteady_adjoint": unsteady_adjoint, "c5_1024x256": c5, "kernel_share": share,
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes + 8},
            "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
