"""Benchmark: FAS W-cycles of the preconditioned AW3 smoother on the 1024x256 thin-layer RANS
C-grid (M = 0.75, Re = 6.5e6, wall spacing 1e-5, 5 levels, Baldwin-Lomax), the largest
configuration that runs on one GPU.

One step = one FAS cycle over the whole grid (every step of the method's hot path).  Prints
one JSON line.  Metric: Mcell-iterations/s (fine cells x cycles / s), beside the wall time to a
6-order residual drop for the FP64 and the mixed-precision preconditioner and the HBM roofline
of the dominant kernel.  Extras (rank 0, one GPU): the 256x64 and 512x128 workloads, pitching
steps to 11 orders, the batched cases, the adjoints and the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision fp64|mixed]
                  [--quick]

Multi-GPU: the exact method does not shard (the SGS sweep is one global wavefront), so N GPUs
run N independent replicas of the same case; value = all ranks' cell-iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth.cgrid import make_cgrid  # noqa: E402

_RANS = dict(scheme="AW3", eta=0.8, d_cut=0.5, cfl=100.0, cfl_ramp=20.0, ramp_cycles=2, viscous=1, turb=1,
             gamma_cycle=2, alpha_deg=0.0)
HEADLINE = dict(name="rans_1024x256_thin_layer_bl", ni=1024, nj=256, n_wake=128, wall_spacing=1e-5, mach=0.75,
                re=6.5e6, nlevels=5, **_RANS)
C2 = dict(name="rans_256x64_thin_layer_bl", ni=256, nj=64, n_wake=32, wall_spacing=1e-5, mach=0.5, re=1e7,
          nlevels=4, **_RANS)
C3 = dict(name="rans_512x128_thin_layer_bl", ni=512, nj=128, n_wake=64, wall_spacing=1e-5, mach=0.8, re=1e6,
          nlevels=4, **_RANS)
WORKLOAD = HEADLINE
METRIC = "Mcell-iter/s"
L2_FLUSH_BYTES = 256 << 20
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
# Algorithmic DRAM bytes per cell of one launch of each kernel class (the compulsory traffic:
# every input read once, every output written once), by preconditioner precision.  The "sgs"
# class is one preconditioner application of a stage with its update; on the headline workload
# every level runs the warp-strip sweep in both precisions.
#   FP64 (two FP32 warp-strip sweeps and one FP64 defect correction):
#     D^-1 r: D^-1 (16 doubles) and r (4 doubles) read, the FP32 right-hand side written (4 floats)  176 B
#     each sweep: forward blocks G_W G_S and backward blocks H_E H_N (64 floats), its right-hand
#       side read, y written and read back, z written (4 x 4 floats)                            2 x 320 B
#     defect: z read (4 floats), H_E H_N (32 doubles) read, t written (4 doubles); D^-1 G_W G_S
#       (48 doubles), r and t (8 doubles) read, the defect written (4 floats)                  304 + 464 B
#     update: z and dz read (8 floats), u^(0) read and u written (8 doubles)                      96 B
#   mixed (one warp-strip sweep): D^-1 (16 floats) and r read, right-hand side written, the
#     sweep, z and u^(0) read, u written: 112 + 320 + 80                                            512 B
#   residual: ghosted u (4), p, q, 1/rho, radii (2), dt*, volume, mu_t, face vectors (4) read,
#     the stage right-hand side and the F^v carry written and the carry read (12)                 232 B
BYTES_PER_CELL = {"fp64": {"sgs": 1680.0, "residual": 232.0}, "mixed": {"sgs": 512.0, "residual": 232.0}}
# DRAM traffic per cell of one launch of the dominant kernel, from an ncu capture of a finest-level
# launch (dram__bytes_read.sum + dram__bytes_write.sum over the cells of that launch); None where
# no capture of the current kernel exists.
# FP64: 395.1 MB read + 1.2 MB written by one finest-level application on the 262,144 cells of
# the 1024x256 grid (rhs, two sweep pairs, the defect kernels, the update), captured by ncu with
# dram__bytes_read.sum and dram__bytes_write.sum.
DRAM_BYTES_PER_CELL = {"fp64": {"sgs": 396.25e6 / 262144}, "mixed": {"sgs": None}}


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


def grid_of(w):
    return make_cgrid(w["ni"], w["nj"], n_wake=w["n_wake"], wall_spacing=w["wall_spacing"])


def workload_grid():
    return grid_of(WORKLOAD)


def params_of(P, w, precision, **over):
    kw = dict(scheme=w["scheme"], nlevels=w["nlevels"], gamma_cycle=w["gamma_cycle"], viscous=w["viscous"],
              turb=w["turb"], sensor=1, mach=w["mach"], alpha_deg=w["alpha_deg"], re=w["re"], eta=w["eta"],
              d_cut=w["d_cut"], cfl=w["cfl"], cfl_ramp=w["cfl_ramp"], ramp_cycles=w["ramp_cycles"],
              precision=precision)
    kw.update(over)
    return P.default_params(**kw)


def gpu_params(P, precision):
    return params_of(P, WORKLOAD, precision)


def oracle_of(w, variant="timing", grid=None):
    import oracle as O
    p = O.make_params(w["scheme"], nlevels=w["nlevels"], gamma_cycle=w["gamma_cycle"], viscous=w["viscous"],
                      turb=w["turb"], sensor=1, mach=w["mach"], alpha_deg=w["alpha_deg"], re=w["re"], eta=w["eta"],
                      d_cut=w["d_cut"], cfl=w["cfl"], cfl_ramp=w["cfl_ramp"], ramp_cycles=w["ramp_cycles"])
    return O.Oracle(grid if grid is not None else grid_of(w), p, variant=variant)


def oracle_solver():
    return oracle_of(WORKLOAD)


def host_cpu():
    """CPU model and logical core count of this host."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model, "machine": platform.machine(), "nproc": os.cpu_count()}


def cpu_oracle_sample(budget_s=15.0, max_cycles=200, min_cycles=3):
    """Time the oracle (its -O3 timing build, as it stands, one host thread) on consecutive
    cycles of the headline workload from the free stream."""
    o = oracle_solver()
    ncell = WORKLOAD["ni"] * WORKLOAD["nj"]
    t0 = time.perf_counter()
    k = 0
    while k < max_cycles and (k < min_cycles or time.perf_counter() - t0 < budget_s):
        o.fas_cycle(k)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": ncell * k / dt / 1e6, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{k} FAS W-cycles of the {WORKLOAD['name']} workload from the free stream, one host "
                      f"thread, oracle timing build (-O3), {dt:.1f} s", "host": host_cpu()}


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
                                             "cycle": "W", "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed FAS W-cycles after {args.warmup} warm-up cycles, one "
                                       "host thread, oracle timing build (-O3)", "host": host_cpu()},
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


def measure_wcycles(P, w, stream, flush, steps, warmup):
    """W-cycle device time of a workload in both precisions, from the free stream."""
    g = grid_of(w)
    out = {"workload": w["name"], "cells": g.ni * g.nj}
    for prec in ("fp64", "mixed"):
        s = P.Solver(g, params_of(P, w, prec), stream=stream.cuda_stream)
        for k in range(warmup):
            s.fas_cycle(k)
        ms = time_cycles(s, stream, flush, steps, warmup)
        out[prec] = {"ms_per_cycle": sum(ms) / len(ms), "value": g.ni * g.nj * len(ms) / (sum(ms) / 1e3) / 1e6,
                     "unit": METRIC}
        s.close()
    return out


def solve_timed(s, drop, max_cycles):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    code, nc, hist = s.solve(drop, max_cycles)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"seconds": dt, "cycles": nc, "status": int(code),
            "final_drop": float(hist[-1] / hist[0]) if len(hist) else None,
            "rate": float((hist[-1] / hist[0]) ** (1.0 / max(nc - 1, 1))) if len(hist) > 1 else None}


def measure_smoothers_c2(P, stream, max_cycles=1000):
    """The 256x64 RANS workload from the free stream to a 6-order drop with AW3 (robust W
    method, c* = 100) and with preconditioned ARK3J at c* = 1 (the value at which section 6.2
    finds it at its stability limit), both FP64; a run that stops early records its status."""
    g = grid_of(C2)
    out = {"workload": C2["name"]}
    for name, over in (("AW3", {}), ("ARK3J", dict(scheme="ARK3J", cfl=1.0, cfl_ramp=1.0))):
        s = P.Solver(g, params_of(P, C2, "fp64", **over), stream=stream.cuda_stream)
        out[name] = solve_timed(s, 1e-6, max_cycles)
        out[name]["cfl"] = over.get("cfl", C2["cfl"])
        s.close()
    return out


def measure_pitching_c3(P, stream, nsteps=4, max_cycles=600):
    """The pitching 512x128 RANS case (alpha = 2 deg sin(2kt), k = 0.2, 64 steps per period):
    a steady start converged 6 orders (mixed precision), then the first nsteps physical steps
    (implicit Euler, then BDF2), each converged 11 orders in pseudo time, once with the FP64 and
    once with the mixed preconditioner from the same start; cycles and seconds per step and the
    state gap between the two precisions after the last step."""
    import torch
    g = grid_of(C3)
    s0 = P.Solver(g, params_of(P, C3, "mixed"), stream=stream.cuda_stream)
    start = solve_timed(s0, 1e-6, 2000)
    u0 = s0.get_state()
    s0.close()
    omega = 0.4
    dt = 2.0 * np.pi / omega / 64
    amp = np.radians(2.0)
    out = {"workload": C3["name"], "steady_start": start, "dt": dt, "steps": {}}
    final = {}
    for prec in ("fp64", "mixed"):
        s = P.Solver(g, params_of(P, C3, prec), stream=stream.cuda_stream)
        s.set_state(u0)
        rows = []
        for step in range(1, nsteps + 1):
            t = step * dt
            s.set_motion(-amp * np.sin(omega * t), -amp * omega * np.cos(omega * t))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            code, nc, h = s.dual_time_step(dt, 1e-11, max_cycles)
            torch.cuda.synchronize()
            rows.append({"kind": "implicit Euler" if step == 1 else "BDF2", "seconds": time.perf_counter() - t0,
                         "cycles": nc, "status": int(code), "final_drop": float(h[-1] / h[0]) if len(h) else None,
                         "final_residual": float(h[-1]) if len(h) else None})
        out["steps"][prec] = rows
        final[prec] = s.get_state()
        s.close()
    out["state_gap_after_last_step"] = float(np.linalg.norm(final["mixed"] - final["fp64"])
                                             / np.linalg.norm(final["fp64"]))
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


def measure_c5(P, stream=None, n_bumps=16, check_bumps=()):
    """The 1024x256 RANS sensitivity case (wall spacing 1e-5, M 0.75, Re 6.5e6, alpha 0, 5-level
    W-cycles of AW3, mixed precision): time to a 6-order drop from the free stream, then the
    C_D adjoint (eddy viscosity frozen) to a 6-order drop and the shape gradient for 16
    Hicks-Henne bumps; host-timed around the synchronous library calls.  check_bumps: bumps whose
    gradient is checked against central differences (h = 1e-6) of complete solves with the eddy
    viscosity frozen at the converged state's (the derivative the adjoint computes), after a
    further solve and adjoint at that frozen eddy viscosity."""
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
    if check_bumps:
        out["frozen_mut_check"] = _c5_check(P, s, g, p, V[list(check_bumps)], list(check_bumps))
    s.close()
    return out


def _c5_check(P, s, g, p, V, ids, h=1e-6):
    from synth.shape import deformed
    t0 = time.perf_counter()
    mut = s.get_mut()
    s.freeze_mut(mut)
    code, nc, hist = s.solve(1e-5, 4000)
    res = {"bumps": ids, "h": h, "refine_status": int(code), "refine_cycles": nc}
    u = s.get_state()
    s.adjoint_jacobian(1e-6)
    lam, acode, it, rr = s.adjoint_solve(1, tol=1e-10, max_iters=3000, restart=250)
    grad = s.adjoint_shape_gradient(1, lam, V)
    res.update(adjoint_status=int(acode), adjoint_relres=rr, grad=[float(x) for x in grad])
    fd, stat = [], []
    for k in range(V.shape[0]):
        cd = []
        for sgn in (1.0, -1.0):
            e = np.zeros(V.shape[0])
            e[k] = sgn * h
            sd = P.Solver(deformed(g, e, V), p)
            sd.set_state(u)
            sd.freeze_mut(mut)
            c2, n2, h2 = sd.solve(1e-6, 4000)
            stat.append((int(c2), n2))
            cd.append(sd.force_coefficients()[1])
            sd.close()
        fd.append((cd[0] - cd[1]) / (2 * h))
    res.update(fd=fd, fd_solves=stat, rel_diff=[abs(a - b) / max(abs(b), 1e-300) for a, b in zip(grad, fd)],
               seconds=time.perf_counter() - t0)
    return res


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
    g = grid_of(C2)
    s = P.Solver(g, params_of(P, C2, "fp64"))
    u = s.get_state()
    jj, ii = np.meshgrid(np.arange(g.nj), np.arange(g.ni), indexing="ij")
    u = u * (1.0 + 0.02 * np.sin(2 * np.pi * ii / g.ni) * np.cos(np.pi * jj / g.nj))[None]
    s.set_state(np.ascontiguousarray(u))
    s.adjoint_jacobian(1e-6)
    t0 = time.perf_counter()
    lam, code, it, rr = s.adjoint_solve(1, tol=1e-14, max_iters=iters, restart=250)
    t = time.perf_counter() - t0
    s.close()
    return {"adjoint_profile": C2["name"], "gmres_iterations": it, "seconds": t,
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


def measure_schemes_c2(P, stream, max_cycles=1500):
    """The 3- and 5-stage W methods of Table "RK smoothers" (AW3, AW5J, AW51, AW52) on the
    256x64 RANS workload from the free stream to a 6-order drop (mixed precision)."""
    g = grid_of(C2)
    out = {"workload": C2["name"], "precision": "mixed"}
    for scheme in ("AW3", "AW5J", "AW51", "AW52"):
        s = P.Solver(g, params_of(P, C2, "mixed", scheme=scheme), stream=stream.cuda_stream)
        out[scheme] = solve_timed(s, 1e-6, max_cycles)
        s.close()
    return out


def measure_preconditioners_c1(P, stream, exact_iters=40, max_cycles=400):
    """The 128x32 Euler case (M 0.8, alpha 1.25 deg, 3-level V, AW3 robust: d 0.5, c* 1e4): the
    paper's SGS preconditioner against the exact one ((D+L+U)^-1, reached by exact_iters block
    Gauss-Seidel corrections), with the JST residual and with the first-order flux-vector-split
    residual whose linearization the blocks are; FP64, to a 6-order drop."""
    g = make_cgrid(128, 32)
    out = {"workload": "euler_128x32", "exact_iterations": exact_iters}
    for flux in ("jst", "fvs"):
        for prec in ("sgs", "exact"):
            p = P.default_params(scheme="AW3", nlevels=3, gamma_cycle=1, mach=0.8, alpha_deg=1.25, cfl=1e4,
                                 flux=flux)
            s = P.Solver(g, p, stream=stream.cuda_stream)
            if prec == "exact":
                s.set_exact_preconditioner(exact_iters)
            out[f"{flux}_{prec}"] = solve_timed(s, 1e-6, max_cycles)
            s.close()
    return out


def measure_mesh_independence(P, stream, max_cycles=1500):
    """Convergence rates of AW3 on three synthetic C-grids of one family (cells 256x32, 384x48,
    512x64: the sizes of the paper's mesh-independence table), thin-layer RANS at M 0.796,
    Re 1e6, 3-level W-cycles (coarsest grids 64x8, 96x12, 128x16), mixed precision: the steady
    solve from the free stream to a 6-order drop, then the first pitching step (implicit Euler,
    k = 0.202, amplitude 1.01 deg, 36 steps per period) to an 11-order drop.  Rates are the
    average per-cycle reduction (final / first) ^ (1 / cycles)."""
    import torch
    omega = 2 * 0.202
    dt = 2.0 * np.pi / omega / 36
    amp = np.radians(1.01)
    out = {"flow": "M 0.796, Re 1e6, thin layer + Baldwin-Lomax, AW3, d 0.5, eta 0.8, c* 100, 3-level W"}
    for ni, nj in ((256, 32), (384, 48), (512, 64)):
        w = dict(C2, name=f"rans_{ni}x{nj}", ni=ni, nj=nj, n_wake=ni // 8, mach=0.796, re=1e6, nlevels=3)
        g = grid_of(w)
        s = P.Solver(g, params_of(P, w, "mixed"), stream=stream.cuda_stream)
        steady = solve_timed(s, 1e-6, max_cycles)
        s.set_motion(-amp * np.sin(omega * dt), -amp * omega * np.cos(omega * dt))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, nc, h = s.dual_time_step(dt, 1e-11, max_cycles)
        torch.cuda.synchronize()
        first = {"seconds": time.perf_counter() - t0, "cycles": nc, "status": int(code),
                 "final_drop": float(h[-1] / h[0]) if len(h) else None,
                 "rate": float((h[-1] / h[0]) ** (1.0 / max(nc - 1, 1))) if len(h) > 1 else None}
        out[f"{ni}x{nj}"] = {"steady": steady, "first_pitching_step": first}
        s.close()
    return out


def _c4_inputs(P, precision):
    from synth.cases import config_c4_cases
    cases = config_c4_cases()
    grids = [c.grid() for c in cases]
    params = [P.default_params(scheme="AW3", nlevels=c.levels, mach=c.mach, alpha_deg=c.alpha_deg, cfl=100.0,
                               precision=precision) for c in cases]
    return cases, grids, params


def batched_cycle(P, stream, flush, steps=10, warmup=3):
    """The 64 batched cases in mixed precision, tuned as in the benchmark: the device time of a
    cycle (steps cycles after warmup, L2 flushed before each), then one more cycle inside the NVTX
    range "batched_cycle" (the range an ncu capture of the cycle's DRAM traffic filters on)."""
    import torch
    cases, grids, params = _c4_inputs(P, "mixed")
    b = P.fasw.Batch(grids, params, stream=stream.cuda_stream)
    tuned = b.autotune(with_tiles=True)
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
    flush.zero_()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batched_cycle")
    b.cycle(warmup + steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    n0 = b.launch_count()
    b.cycle(warmup + steps + 1)
    torch.cuda.synchronize()
    launches = b.launch_count() - n0
    b.close()
    cells = sum(g.ni * g.nj for g in grids)
    return {"workload": "euler_64_batched_cases", "cells": cells, "precision": "mixed", "ms_per_cycle": sum(ms) / steps,
            "value": cells * steps / (sum(ms) / 1e3) / 1e6, "unit": METRIC, "launches_per_cycle": launches,
            "sweep_choice": [int(k) for k, _ in tuned], "tile_choice": [int(t) for _, t in tuned]}


def measure_batched(P, stream, flush, steps, warmup, sequential=True):
    """The 64 uneven Euler cases (128x32 .. 512x128 cells, seeded M, alpha, thickness):
    (i) mixed precision batched (one captured CUDA graph per cycle, sweep variants from the
    autotuner): cycle throughput and time until every case has dropped 6 orders; (ii) the same
    batched in FP64; (iii) the plain FP64 path, one case after another, each to 6 orders."""
    import torch
    out = {}
    for prec in ("mixed", "fp64"):
        cases, grids, params = _c4_inputs(P, prec)
        cells = sum(g.ni * g.nj for g in grids)
        b = P.fasw.Batch(grids, params, stream=stream.cuda_stream)
        tuned = b.autotune(with_tiles=True)
        choice = [k for k, _ in tuned]
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
        b.close()
        b = P.fasw.Batch(grids, params, stream=stream.cuda_stream)
        b.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, cyc, drops, ncy = b.solve(1e-6, 400)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        b.close()
        out["batched_" + prec] = {
            "cases": len(grids), "cells": cells, "value": cells * steps / (sum(ms) / 1e3) / 1e6, "unit": METRIC,
            "ms_per_cycle": sum(ms) / steps,
            "sweep_choice": {"staged8": choice.count(7), "staged4": choice.count(6), "staged": choice.count(5),
                             "cta": choice.count(2), "warp": choice.count(9), "warp8": choice.count(10)},
            "residual_tile_choice": {str(t): sum(1 for _, x in tuned if x == t) for t in (0, 1, 2, 4, 8)},
            "time_to_6_orders": {"seconds": dt, "cycles_run": ncy, "status": int(code),
                                 "cases_converged": int((cyc > 0).sum()), "cases_diverged": int((cyc == -2).sum()),
                                 "median_cycles": float(np.median(cyc[cyc > 0])) if (cyc > 0).any() else None}}
    if sequential:
        cases, grids, params = _c4_inputs(P, "fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, cyc_total = 0, 0
        for g, p in zip(grids, params):
            s = P.Solver(g, p, stream=stream.cuda_stream)
            code, nc, hist = s.solve(1e-6, 400)
            conv += int(code == 0)
            cyc_total += nc
            s.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["sequential_fp64"] = {"cases": len(grids), "seconds": dt, "cases_converged": conv,
                                  "cycles_total": cyc_total,
                                  "note": "one context per case, created, solved to 6 orders and destroyed in turn"}
    return out


def oracle_all_cores_c4(budget_cycles=2):
    """The oracle (timing build, as it stands) over all host cores: one case per thread (ctypes
    releases the interpreter lock during each call), each case running `budget_cycles` cycles
    from the free stream; the throughput over the whole host."""
    import oracle as O
    from synth.cases import config_c4_cases
    cases = config_c4_cases()
    ncores = os.cpu_count() or 1
    solvers = []
    for c in cases:
        p = O.make_params("AW3", nlevels=c.levels, mach=c.mach, alpha_deg=c.alpha_deg, cfl=100.0)
        solvers.append((c.ni * c.nj, O.Oracle(c.grid(), p, variant="timing")))
    todo = list(range(len(solvers)))
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                if not todo:
                    return
                k = todo.pop()
            for cyc in range(budget_cycles):
                solvers[k][1].fas_cycle(cyc)

    t0 = time.perf_counter()
    threads = [threading.Thread(target=worker) for _ in range(ncores)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    dt = time.perf_counter() - t0
    cells = sum(n for n, _ in solvers)
    return {"value": cells * budget_cycles / dt / 1e6, "unit": METRIC, "cores": ncores, "kind": "oracle",
            "sample": f"{budget_cycles} cycles of each of the 64 batched cases from the free stream, one case per "
                      f"thread on {ncores} threads, oracle timing build, {dt:.1f} s", "host": host_cpu()}


def hbm_peak():
    try:
        pk = json.load(open(MEASURED_PEAKS))
        return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def roofline(kt, steps, precision, w):
    """HBM roofline of the dominant kernel class: its algorithmic bytes per launch (bytes per cell
    x the cells one launch processes on average over the cycle) / its average launch time."""
    dom = max(kt, key=lambda k: kt[k][1])
    n_l, ms_l = kt[dom]
    avg_ms = ms_l / max(n_l, 1)
    nl, gam = w["nlevels"], w["gamma_cycle"]
    visits = level_visits(nl, gam)
    ncell = w["ni"] * w["nj"]
    cells = [ncell // (4 ** (nl - 1 - l)) for l in range(nl)]
    stages = 3
    per_cycle = {
        "sgs": sum(stages * visits[l] * cells[l] for l in range(nl)),
        "residual": sum(stages * visits[l] * cells[l] for l in range(nl))
        + sum(visits[l] * cells[l] for l in range(1, nl)) + sum(visits[l] * cells[l] for l in range(0, nl - 1)),
    }
    peak, src = hbm_peak()
    bpc = BYTES_PER_CELL[precision].get(dom)
    if bpc is None or dom not in per_cycle:
        return {"kernel": dom, "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "avg_launch_ms": avg_ms, "peak_source": src}
    cells_per_launch = per_cycle[dom] / (n_l / steps)
    achieved = bpc * cells_per_launch / (avg_ms / 1e3) / 1e9
    dram = DRAM_BYTES_PER_CELL[precision].get(dom)
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": dram * cells_per_launch if dram else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per cell of a captured launch, "
                              "times the cells of the average launch" if dram else None,
            "avg_launch_ms": avg_ms, "launches_per_cycle": n_l / steps, "cells_per_launch": cells_per_launch,
            "bytes_per_cell": bpc, "peak_source": src,
            "note": "the SGS sweep is a recurrence along i+j: its time is set by the per-step latency of the "
                    "wavefront, not by HBM bandwidth; the fraction states how far from the memory bound it runs"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--quick", action="store_true", help="the headline line only (no extras)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-sequential", action="store_true", help="skip the one-case-at-a-time FP64 batch leg")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-unsteady-adjoint", action="store_true")
    ap.add_argument("--pitch-steps", type=int, default=4, help="physical steps of the 512x128 pitching case")
    ap.add_argument("--c5", action="store_true",
                    help="only the 1024x256 RANS shape-sensitivity case (steady solve, adjoint, 16 bump gradients, "
                         "two of them against differences of frozen-eddy-viscosity solves)")
    ap.add_argument("--c5-unsteady", action="store_true",
                    help="only the two-period unsteady adjoint of the pitching 512x128 RANS case (minutes)")
    ap.add_argument("--c3-period", action="store_true",
                    help="only the full 64-step period of the 512x128 pitching case, FP64 and mixed (minutes)")
    ap.add_argument("--mesh-independence", action="store_true",
                    help="only the convergence rates on the 256x32 / 384x48 / 512x64 grid family")
    ap.add_argument("--batched-cycle", action="store_true",
                    help="only the 64 batched cases (mixed): cycle time, then one cycle in the NVTX range "
                         "'batched_cycle' (for an ncu DRAM capture)")
    ap.add_argument("--adjoint-profile", action="store_true",
                    help="only one 30-iteration adjoint GMRES solve on the 256x64 grid (for ncu launch lists)")
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
        print(json.dumps(measure_c5(P, check_bumps=(2, 11))), flush=True)
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
    if args.c3_period:
        print(json.dumps(measure_pitching_c3(P, stream, nsteps=64)), flush=True)
        return
    if args.mesh_independence:
        print(json.dumps(measure_mesh_independence(P, stream)), flush=True)
        return
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    if args.batched_cycle:
        print(json.dumps(batched_cycle(P, stream, flush)), flush=True)
        return
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

    # per-kernel-class device time over a second pass of the same number of cycles
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
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        s.set_state(u_host.numpy())
        s.fas_cycle(10**6)
        s.get_state(out=u_out.numpy())
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = world * ncell * args.steps / e2e_s / 1e6
    state_bytes = 4 * ncell * 8
    s.close()

    extras = {}
    if not args.quick and rank == 0 and world == 1:
        # the other precision on the same workload
        so = P.Solver(g, gpu_params(P, "mixed" if args.precision == "fp64" else "fp64"), stream=stream.cuda_stream)
        for k in range(args.warmup):
            so.fas_cycle(k)
        ms_other = time_cycles(so, stream, flush, args.steps, args.warmup)
        so.close()
        extras["other_precision"] = {"precision": "mixed" if args.precision == "fp64" else "fp64",
                                     "value": ncell * args.steps / (sum(ms_other) / 1e3) / 1e6,
                                     "ms_per_step": sum(ms_other) / args.steps}
        # time to a 6-order drop from the free stream, FP64 and mixed preconditioner
        drops, states = {}, {}
        for prec in ("fp64", "mixed"):
            sd = P.Solver(g, gpu_params(P, prec), stream=stream.cuda_stream)
            drops[prec] = solve_timed(sd, 1e-6, 1500)
            states[prec] = sd.get_state()
            sd.close()
        extras["time_to_6_orders"] = drops
        extras["precision_gap_6_orders"] = float(np.linalg.norm(states["mixed"] - states["fp64"])
                                                 / np.linalg.norm(states["fp64"]))
        extras["c2_256x64"] = measure_wcycles(P, C2, stream, flush, args.steps, args.warmup)
        extras["c2_256x64"]["smoothers_to_6_orders"] = measure_smoothers_c2(P, stream)
        extras["c2_256x64"]["schemes_to_6_orders"] = measure_schemes_c2(P, stream)
        extras["c1_preconditioners"] = measure_preconditioners_c1(P, stream)
        extras["c3_512x128"] = measure_wcycles(P, C3, stream, flush, min(args.steps, 10), args.warmup)
        if args.pitch_steps > 0:
            extras["c3_512x128"]["pitching"] = measure_pitching_c3(P, stream, nsteps=args.pitch_steps)
        if not args.no_batched:
            extras["batched_64_cases"] = measure_batched(P, stream, flush, args.steps, args.warmup,
                                                         sequential=not args.no_sequential)
            if not args.no_cpu_baseline:
                extras["batched_64_cases"]["oracle_all_cores"] = oracle_all_cores_c4()
        if not args.no_adjoint:
            adj = {}
            for prec in ("fp64", "mixed"):
                sa = P.Solver(grid_of(C2), params_of(P, C2, prec), stream=stream.cuda_stream)
                sa.solve(1e-6, 1000)
                adj[prec] = measure_adjoint(sa, grid_of(C2))
                sa.close()
            extras["adjoint_256x64"] = adj
            if not args.no_unsteady_adjoint:
                extras["unsteady_adjoint"] = measure_unsteady_adjoint(P, stream)
            extras["c5_1024x256_sensitivity"] = measure_c5(P, stream)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    share = {k: round(v[1] / max(sum(x[1] for x in kt.values()), 1e-12), 4) for k, v in kt.items()}
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_oracle_sample()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "cells": ncell, "levels": WORKLOAD["nlevels"],
                       "cycle": "W", "scheme": "AW3", "precision": args.precision, "cfl": WORKLOAD["cfl"],
                       "l2": "inputs larger than L2 (about 0.5 GB resident); L2 also flushed (256 MiB write) "
                             "between timed cycles", "parallelism": "replicas"},
            **extras, "kernel_share": share,
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes + 8},
            "gpu_launches": int(launches), "clocks": clk.summary(),
            "roofline": roofline(kt, args.steps, args.precision, WORKLOAD), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
