"""Pins of the oracle's unsteady discrete adjoint (dual time stepping on a pitching grid).

- the adjoint gradient equals the direct (tangent) gradient that carries du^n/dp forward
  through the same time-discrete equations, an identity of linear algebra: a wrong coupling
  coefficient, sign or time index in the backward recursion breaks it at O(1);
- the same for the sensitivity to the initial state;
- both equal central differences of full nonlinear unsteady solves (deformed grids, perturbed
  initial state) to the accuracy a piecewise-smooth residual allows.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from oracle import unsteady_adjoint as U
from oracle.adjoint import force_coefficients, jacobian
from synth.cgrid import make_cgrid
from synth.shape import bump_fields, deformed

AMP, OMEGA, XC, YC = np.radians(2.0), 0.4, 0.25, 0.0
DT = 2.0 * np.pi / OMEGA / 16
N = 4
DROP, CYCLES = 1e-12, 400


@pytest.fixture(scope="module")
def case():
    g = make_cgrid(32, 8, n_wake=4, wall_spacing=2e-3)
    p = O.make_params("AW3", nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    o = O.Oracle(g, p)
    for k in range(200):
        o.fas_cycle(k)
    u0 = o.get_state()
    V = bump_fields(g, 2)
    J, grad, g0, lam = U.gradient(g, p, u0, V, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    return g, p, u0, V, J, grad, g0


def _tangent(g, p, u0, V, k, du0, h_x=1e-6):
    """dJ along bump k (k >= 0) or along the initial-state direction du0 (k < 0), forward."""
    _, states = U.forward(g, p, u0, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    du = {0: du0.ravel() if k < 0 else np.zeros(u0.size)}
    dJ = 0.0
    for n in range(1, N + 1):
        phi, phidot = U.pitch(n * DT, AMP, OMEGA)
        a, b, c = U.time_coefficients(n, DT)
        on = O.Oracle(g, p)
        on.set_motion(phi, phidot, XC, YC)
        on.set_state(states[n])
        on.set_time_source(a, None)
        Jn, _, gD = jacobian(on, 0.0)
        rhs = -b * du[n - 1] - (c * du[n - 2] if n >= 2 else 0.0)
        dC = 0.0
        if k >= 0:
            e = np.zeros(V.shape[0])
            e[k] = h_x
            F, C = [], []
            for s in (1.0, -1.0):
                ok = O.Oracle(deformed(g, s * e, V), p)
                ok.set_motion(phi, phidot, XC, YC)
                ok.set_state(states[n])
                F.append(ok.residual()[0].ravel())
                C.append(force_coefficients(*ok.wall_force(), 0.0)[1])
            rhs = rhs - (F[0] - F[1]) / (2.0 * h_x)
            dC = (C[0] - C[1]) / (2.0 * h_x)
        du[n] = spla.spsolve(Jn.tocsc(), rhs)
        dJ += (dC + gD @ du[n]) / N
    return dJ


def test_time_coefficients_are_implicit_euler_then_bdf2():
    # BDF2 differentiates a quadratic exactly; implicit Euler a linear function
    dt = 0.3
    t = np.array([0.0, dt, 2 * dt])
    q = 1.0 + 2.0 * t + 3.0 * t ** 2
    a, b, c = U.time_coefficients(2, dt)
    assert abs(a * q[2] + b * q[1] + c * q[0] - (2.0 + 6.0 * t[2])) < 1e-12
    a, b, c = U.time_coefficients(1, dt)
    assert (a, b, c) == (1.0 / dt, -1.0 / dt, 0.0)


def test_adjoint_shape_gradient_equals_tangent(case):
    g, p, u0, V, J, grad, g0 = case
    for k in range(V.shape[0]):
        t = _tangent(g, p, u0, V, k, None)
        assert abs(t - grad[k]) <= 1e-9 * max(abs(grad[k]), 1.0), (k, t, grad[k])


def test_initial_state_sensitivity_equals_tangent(case):
    g, p, u0, V, J, grad, g0 = case
    d = np.random.default_rng(0).standard_normal(u0.shape)
    t = _tangent(g, p, u0, V, -1, d)
    assert abs(t - np.sum(g0 * d)) <= 1e-9 * max(abs(t), np.abs(g0).max())


def test_adjoint_matches_finite_differences_of_unsteady_solves(case):
    g, p, u0, V, J, grad, g0 = case
    h = 1e-6
    for k in range(V.shape[0]):
        e = np.zeros(V.shape[0])
        e[k] = h
        Jp, _ = U.forward(deformed(g, e, V), p, u0, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
        Jm, _ = U.forward(deformed(g, -e, V), p, u0, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
        # switches of the JST sensor and radii make the residual piecewise smooth; the
        # linearisation holds them fixed.  A wrong sign or a dropped term is an O(1) error.
        assert abs((Jp - Jm) / (2 * h) - grad[k]) <= 1e-3 * abs(grad[k])
    jj, ii = np.meshgrid(np.arange(g.nj), np.arange(g.ni), indexing="ij")
    d = np.sin(2 * np.pi * ii / g.ni) * np.exp(-jj / 3.0)
    d = np.stack([0.01 * d, 0.02 * d, -0.01 * d, 0.05 * d])
    hp = 1e-5
    Jp, _ = U.forward(g, p, u0 + hp * d, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    Jm, _ = U.forward(g, p, u0 - hp * d, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    assert abs((Jp - Jm) / (2 * hp) - np.sum(g0 * d)) <= 1e-3 * abs(np.sum(g0 * d))


@pytest.mark.parametrize("turb", [0, 1])
def test_viscous_adjoint_equals_tangent(turb):
    """The same identity with the thin-layer viscous flux on the moving no-slip wall, laminar and
    with Baldwin-Lomax (frozen at each level's value on both sides of the identity)."""
    g = make_cgrid(32, 8, n_wake=4, wall_spacing=5e-3)
    p = O.make_params("AW3", nlevels=2, viscous=1, turb=turb, sensor=1, mach=0.5, alpha_deg=0.0,
                      re=5e3 if turb == 0 else 1e5, cfl=1e3 if turb == 0 else 100.0)
    o = O.Oracle(g, p)
    for k in range(300):
        o.fas_cycle(k)
    u0 = o.get_state()
    V = bump_fields(g, 2)
    n = 3
    J, grad, g0, _ = U.gradient(g, p, u0, V, AMP, OMEGA, XC, YC, DT, n, DROP, CYCLES, 1)
    _, states = U.forward(g, p, u0, AMP, OMEGA, XC, YC, DT, n, DROP, CYCLES, 1)
    e = np.zeros(2)
    e[0] = 1e-6
    du = {0: np.zeros(u0.size)}
    dJ = 0.0
    for m in range(1, n + 1):
        phi, phidot = U.pitch(m * DT, AMP, OMEGA)
        a, b, c = U.time_coefficients(m, DT)
        on = O.Oracle(g, p)
        on.set_motion(phi, phidot, XC, YC)
        on.set_state(states[m])
        mut = on.compute_mut() if turb else None
        on.set_time_source(a, None)
        Jn, _, gD = jacobian(on, 0.0)
        F, C = [], []
        for sgn in (1.0, -1.0):
            ok = O.Oracle(deformed(g, sgn * e, V), p)
            ok.set_motion(phi, phidot, XC, YC)
            ok.set_state(states[m])
            if mut is not None:
                ok.set_mut(mut)
            F.append(ok.residual()[0].ravel())
            C.append(force_coefficients(*ok.wall_force(), 0.0)[1])
        rhs = -(F[0] - F[1]) / 2e-6 - b * du[m - 1] - (c * du[m - 2] if m >= 2 else 0.0)
        du[m] = spla.spsolve(Jn.tocsc(), rhs)
        dJ += ((C[0] - C[1]) / 2e-6 + gD @ du[m]) / n
    assert abs(dJ - grad[0]) <= 1e-9 * max(abs(grad[0]), 1.0), (dJ, grad[0])

