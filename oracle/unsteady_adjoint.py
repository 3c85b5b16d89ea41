"""Oracle discrete adjoint of dual time stepping on a rigidly pitching grid (test
infrastructure only).

Primal (section 6): at time level n = 1..N the grid is rotated to phi(t_n) and the physical
step solves F^n(u^n) = R(u^n; X^n, Xdot^n) / vol + a_n u^n + b_n u^(n-1) + c_n u^(n-2) = 0 in
pseudo time, with implicit Euler for the first step (a, b, c) = (1, -1, 0) / dt and BDF2 after
(a, b, c) = (3/2, -2, 1/2) / dt.  Objective: the time average J = (1/N) sum_n C(u^n, X^n) of
the lift or drag coefficient of the wall-face force.

Adjoint (the Lagrangian of the time-discrete equations): going backwards from n = N,
    (dF^n/du^n)^T lam^n = (1/N) dC^n/du^n - b_(n+1) lam^(n+1) - c_(n+2) lam^(n+2),
with lam^(N+1) = lam^(N+2) = 0 (the couplings dF^(n+1)/du^n = b_(n+1) I and
dF^(n+2)/du^n = c_(n+2) I come from the time terms, which are per unit volume).  The shape
gradient with the initial state held fixed is
    dJ/dp = sum_n [(1/N) dC^n/dX - lam^n . dF^n/dX] dX^n/dp,
both X-derivatives by central differences over deformed grids rotated to phi(t_n) (the time
terms do not depend on X), and the sensitivity to the initial state is
    dJ/du^0 = -(b_1 lam^1 + c_2 lam^2).
Every state u^n is stored (no checkpointing) and every adjoint system is solved by a sparse LU.
With a turbulence model the eddy viscosity is frozen at its Baldwin-Lomax value at each level's
state u^n (in the Jacobian and in the X-derivatives alike), the linearisation the library's
adjoint takes.

Only tests/ import this module; it shares nothing with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import Oracle
from .adjoint import adjoint, force_coefficients, jacobian


def pitch(t: float, amp: float, omega: float) -> tuple[float, float]:
    """Grid rotation phi(t) and its rate for the pitching motion alpha(t) = alpha_m + amp sin(omega t):
    a nose-up pitch turns the grid clockwise, phi = -amp sin(omega t)."""
    return -amp * np.sin(omega * t), -amp * omega * np.cos(omega * t)


def time_coefficients(n: int, dt: float, bdf_order: int = 2) -> tuple[float, float, float]:
    """(a_n, b_n, c_n): implicit Euler at n = 1 (and for bdf_order 1), BDF2 after (section 6)."""
    if n <= 1 or bdf_order == 1:
        return 1.0 / dt, -1.0 / dt, 0.0
    return 1.5 / dt, -2.0 / dt, 0.5 / dt


def _objective(o: Oracle, which: int, alpha_deg: float) -> float:
    return force_coefficients(*o.wall_force(), alpha_deg)[which]


def forward(grid, params, u0: np.ndarray, amp: float, omega: float, xc: float, yc: float, dt: float, nsteps: int,
            drop: float, max_cycles: int, which: int):
    """(J, states): the time-averaged objective and u^0..u^N of nsteps dual-time steps from u0
    (the grid at rest at t = 0)."""
    o = Oracle(grid, params)
    o.set_state(u0)
    states = [np.array(u0, dtype=np.float64)]
    J = 0.0
    for n in range(1, nsteps + 1):
        o.set_motion(*pitch(n * dt, amp, omega), xc, yc)
        nc, _ = o.dual_time_step(dt, drop, max_cycles)
        if nc < 0:
            raise FloatingPointError(f"dual-time step {n} diverged")
        states.append(o.get_state())
        J += _objective(o, which, params.alpha_deg) / nsteps
    return J, states


def gradient(grid, params, u0: np.ndarray, fields: np.ndarray, amp: float, omega: float, xc: float, yc: float,
             dt: float, nsteps: int, drop: float, max_cycles: int, which: int, h_rel: float = 1e-6,
             h_x: float = 1e-6):
    """(J, dJ/dp with u0 fixed, dJ/du0, [lam^1..lam^N]) for the y-displacement fields
    (nparam, nj+1, ni+1) of the grid at rest."""
    from synth.shape import deformed

    alpha = params.alpha_deg
    J, states = forward(grid, params, u0, amp, omega, xc, yc, dt, nsteps, drop, max_cycles, which)
    N = nsteps
    w = 1.0 / N
    nparam = fields.shape[0]
    grad = np.zeros(nparam)
    lam = [None] * (N + 3)
    zero = np.zeros(states[0].size)
    lam[N + 1] = lam[N + 2] = zero
    bo = params.bdf_order
    for n in range(N, 0, -1):
        phi, phidot = pitch(n * dt, amp, omega)
        a_n = time_coefficients(n, dt, bo)[0]
        o = Oracle(grid, params)
        o.set_motion(phi, phidot, xc, yc)
        o.set_state(states[n])
        mut = o.compute_mut() if params.turb else None  # frozen at its value for u^n
        o.set_time_source(a_n, None)
        Jn, gL, gD = jacobian(o, alpha, h_rel)
        rhs = w * (gL if which == 0 else gD)
        if n + 1 <= N:
            rhs = rhs - time_coefficients(n + 1, dt, bo)[1] * lam[n + 1]
        if n + 2 <= N:
            rhs = rhs - time_coefficients(n + 2, dt, bo)[2] * lam[n + 2]
        lam[n] = adjoint(Jn, rhs)
        for k in range(nparam):
            e = np.zeros(nparam)
            e[k] = h_x
            F, C = [], []
            for sgn in (1.0, -1.0):
                ok = Oracle(deformed(grid, sgn * e, fields), params)
                ok.set_motion(phi, phidot, xc, yc)
                ok.set_state(states[n])
                if mut is not None:
                    ok.set_mut(mut)
                F.append(ok.residual()[0].ravel())
                C.append(_objective(ok, which, alpha))
            grad[k] += w * (C[0] - C[1]) / (2.0 * h_x) - lam[n] @ (F[0] - F[1]) / (2.0 * h_x)
    g0 = -time_coefficients(1, dt, bo)[1] * lam[1]
    if N >= 2:
        g0 = g0 - time_coefficients(2, dt, bo)[2] * lam[2]
    return J, grad, g0.reshape(states[0].shape), [lam[n].reshape(states[0].shape) for n in range(1, N + 1)]
