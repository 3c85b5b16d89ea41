"""Shape sensitivities through the discrete adjoint, as a torch.autograd.Function.

``ShapeForces.apply(p, ctx)`` returns the lift and drag coefficients of the steady solution on
the grid deformed by the shape parameters p (a float64 tensor), and its backward pass gives
dC/dp from the CUDA library's adjoint solves (``fasw_adjoint_*``).  The geometry is supplied by
the caller: a function ``grid_of(p)`` that returns the deformed C-grid and the vertex fields
dX/dp (y-displacements per unit parameter), so this module carries no shape parameterization.
All numerics run in the library; this file only sequences calls and marshals arrays.
"""
from __future__ import annotations

import numpy as np
import torch

from .fasw import Solver


class AdjointContext:
    """Primal and adjoint settings shared by the forward and backward passes."""

    def __init__(self, grid_of, fields, params, drop=1e-12, max_cycles=2000, h_rel=1e-6, h_x=1e-6,
                 tol=1e-10, max_iters=1500, restart=250, cfl=0.0, warm_state=None):
        self.grid_of = grid_of
        self.fields = np.ascontiguousarray(fields, dtype=np.float64)
        self.params = params
        self.drop, self.max_cycles = drop, max_cycles
        self.h_rel, self.h_x = h_rel, h_x
        self.tol, self.max_iters, self.restart, self.cfl = tol, max_iters, restart, cfl
        self.warm_state = warm_state
        self.solver = None
        self.info = {}


class ShapeForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p: torch.Tensor, actx: AdjointContext):
        grid = actx.grid_of(p.detach().cpu().numpy())
        s = Solver(grid, actx.params)
        if actx.warm_state is not None:
            s.set_state(actx.warm_state)
        code, nc, hist = s.solve(actx.drop, actx.max_cycles)
        actx.info["primal"] = (int(code), int(nc), float(hist[-1] / hist[0]) if len(hist) else None)
        if actx.solver is not None:
            actx.solver.close()
        actx.solver = s
        cl, cd = s.force_coefficients()
        ctx.actx = actx
        return torch.tensor([cl, cd], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        a = ctx.actx
        s = a.solver
        s.adjoint_jacobian(a.h_rel)
        grads = []
        for which in (0, 1):
            lam, code, it, rr = s.adjoint_solve(which, tol=a.tol, max_iters=a.max_iters, restart=a.restart, cfl=a.cfl)
            a.info[("adjoint", which)] = (int(code), it, rr)
            grads.append(s.adjoint_shape_gradient(which, lam, a.fields, a.h_x))
        g = torch.tensor(np.stack(grads), dtype=torch.float64)  # (2, nparam)
        return gout.to(torch.float64) @ g, None


def pitching_gradient(solver: Solver, fields, amp, omega, dt, nsteps, which=1, xc=0.25, yc=0.0, snapshots=None,
                      drop=1e-10, max_cycles=500, h_rel=1e-6, h_x=1e-6, tol=1e-10, max_iters=400, restart=250,
                      cfl=0.0):
    """Time-averaged C_L (which 0) or C_D (1) over nsteps dual-time steps of the pitching motion
    alpha + amp sin(omega t), started from the steady solution that `solver` holds on the grid at
    rest, and its total derivative with respect to the amplitudes of the y-displacement fields:
    the unsteady adjoint (initial state held fixed) plus the initial state's own dependence on
    the shape, through one steady adjoint solve with right-hand side dJ/du^0.
    Returns (J, gradient, info)."""
    J, grad, g0, code, stats = solver.unsteady_adjoint(
        amp, omega, dt, nsteps, fields, which=which, xc=xc, yc=yc, drop=drop, max_cycles=max_cycles,
        snapshots=snapshots, h_rel=h_rel, h_x=h_x, tol=tol, max_iters=max_iters, restart=restart, cfl=cfl)
    solver.adjoint_jacobian(h_rel)
    nu, code0, it0, rr0 = solver.adjoint_solve(which, g=g0, tol=tol, max_iters=max_iters, restart=restart, cfl=cfl)
    # -nu . dR/dX V: the shape gradient of the steady adjoint nu without an explicit objective part
    V = np.ascontiguousarray(fields, dtype=np.float64)
    steady = solver.adjoint_shape_gradient(-1, nu, V, h_x)
    info = dict(stats, unsteady_status=int(code), steady_status=int(code0), steady_iterations=it0,
                steady_relative_residual=rr0)
    return J, grad + steady, info


class PitchingContext:
    """Settings of the pitching objective: motion alpha + amp sin(omega t) for nsteps dual-time
    steps of size dt from the steady state, objective `which` (0 C_L, 1 C_D) averaged over the
    steps, shape from grid_of(p) / fields as for ShapeForces."""

    def __init__(self, grid_of, fields, params, amp, omega, dt, nsteps, which=1, xc=0.25, yc=0.0, snapshots=None,
                 steady_drop=1e-12, steady_cycles=3000, drop=1e-10, max_cycles=500, tol=1e-10, max_iters=600,
                 restart=250):
        self.grid_of = grid_of
        self.fields = np.ascontiguousarray(fields, dtype=np.float64)
        self.params = params
        self.amp, self.omega, self.dt, self.nsteps = amp, omega, dt, nsteps
        self.which, self.xc, self.yc, self.snapshots = which, xc, yc, snapshots
        self.steady_drop, self.steady_cycles = steady_drop, steady_cycles
        self.drop, self.max_cycles = drop, max_cycles
        self.tol, self.max_iters, self.restart = tol, max_iters, restart
        self.info = {}


def _steady_solver(actx, p):
    s = Solver(actx.grid_of(p.detach().cpu().numpy()), actx.params)
    code, nc, hist = s.solve(actx.steady_drop, actx.steady_cycles)
    actx.info["steady"] = (int(code), int(nc))
    return s


class PitchingForces(torch.autograd.Function):
    """Time-averaged lift or drag of the pitching motion as a function of the shape parameters
    p; the forward pass runs the steady start and the dual-time steps, the backward pass the
    unsteady adjoint (fasw_unsteady_adjoint) and the steady start's own adjoint."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, actx: PitchingContext):
        s = _steady_solver(actx, p)
        J, code, cycles = s.pitching_objective(actx.amp, actx.omega, actx.dt, actx.nsteps, which=actx.which,
                                               xc=actx.xc, yc=actx.yc, drop=actx.drop, max_cycles=actx.max_cycles)
        actx.info["forward"] = (int(code), int(cycles))
        s.close()
        ctx.actx = actx
        ctx.save_for_backward(p)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        a = ctx.actx
        (p,) = ctx.saved_tensors
        s = _steady_solver(a, p)
        J, grad, info = pitching_gradient(s, a.fields, a.amp, a.omega, a.dt, a.nsteps, which=a.which, xc=a.xc,
                                          yc=a.yc, snapshots=a.snapshots, drop=a.drop, max_cycles=a.max_cycles,
                                          tol=a.tol, max_iters=a.max_iters, restart=a.restart)
        s.close()
        a.info["adjoint"] = info
        a.info["J_backward"] = J
        return gout.to(torch.float64) * torch.tensor(grad, dtype=torch.float64), None
