"""Pins of the oracle's moving-grid (rigid pitching, ALE) and dual-time paths: the discrete
geometric conservation law, rotated metrics, uniform-flow preservation away from walls, the
moving-wall ghost, and the implicit-Euler / BDF2 equations of eq. (nonlin-eq) satisfied by
converged time steps.  CPU only."""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid


def _pitch(t, amp=np.radians(2.0), omega=0.4):
    """Grid rotation (nose up = clockwise) and its rate for alpha(t) = amp sin(omega t)."""
    return -amp * np.sin(omega * t), -amp * omega * np.cos(omega * t)


def test_rigid_rotation_conserves_grid_volume_flux_per_cell():
    g = make_cgrid(64, 16, jitter=0.1, seed=3)
    o = O.Oracle(g, O.make_params(nlevels=3))
    o.set_motion(0.3, 0.7)
    for l in range(3):
        vfx, vfe = o.grid_fluxes(l)
        div = vfx[:, 1:] - vfx[:, :-1] + vfe[1:, :] - vfe[:-1, :]
        assert np.abs(div).max() < 1e-13 * max(np.abs(vfx).max(), np.abs(vfe).max())


def test_rotated_metrics_are_rotated_copies():
    g = make_cgrid(32, 8)
    o = O.Oracle(g, O.make_params(nlevels=1))
    sxx0, sxy0, sex0, sey0, vol0 = o.metrics(0)
    phi = 0.37
    o.set_motion(phi, 0.0)
    sxx, sxy, sex, sey, vol = o.metrics(0)
    c, s = np.cos(phi), np.sin(phi)
    np.testing.assert_allclose(sxx, c * sxx0 - s * sxy0, atol=1e-12)
    np.testing.assert_allclose(sxy, s * sxx0 + c * sxy0, atol=1e-12)
    np.testing.assert_allclose(sex, c * sex0 - s * sey0, atol=1e-12)
    np.testing.assert_allclose(vol, vol0, rtol=1e-12)


def test_uniform_flow_preserved_on_a_pitching_grid_away_from_walls():
    ni, nj = 64, 16
    g = make_cgrid(ni, nj)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=0.0))
    o.set_motion(*_pitch(1.3))
    w = O.free_stream(0.8, 0.0)
    o.set_state(np.broadcast_to(w[:, None, None], (4, nj, ni)).copy())
    F, _, _ = o.residual()
    assert np.abs(F[:, 3:nj - 3, 3:ni - 3]).max() < 1e-12


@pytest.mark.parametrize("viscous", [0, 1])
def test_moving_wall_ghost_gives_wall_velocity_at_the_face(viscous):
    ni, nj, nw = 32, 8, 4
    g = make_cgrid(ni, nj, n_wake=nw, wall_spacing=1e-3)
    o = O.Oracle(g, O.make_params(nlevels=1, viscous=viscous, mach=0.5, re=1e5))
    phi, phidot = 0.05, 0.2
    o.set_motion(phi, phidot)
    rng = np.random.default_rng(1)
    u = O.free_stream(0.5, 0.0)[:, None, None] * (1 + 0.02 * rng.standard_normal((4, nj, ni)))
    o.set_state(u)
    G = o.ghosted()
    c, s = np.cos(phi), np.sin(phi)
    for i in range(nw, ni - nw):
        # wall face midpoint of the rotated grid and its velocity
        xa, ya = g.x[0, i] - 0.25, g.y[0, i]
        xb, yb = g.x[0, i + 1] - 0.25, g.y[0, i + 1]
        mx = 0.25 + c * 0.5 * (xa + xb) - s * 0.5 * (ya + yb)
        my = s * 0.5 * (xa + xb) + c * 0.5 * (ya + yb)
        wv = np.array([-phidot * my, phidot * (mx - 0.25)])
        v0 = G[1:3, 2, i + 2] / G[0, 2, i + 2]
        vg = G[1:3, 1, i + 2] / G[0, 1, i + 2]
        face = 0.5 * (v0 + vg)
        dx = c * (xb - xa) - s * (yb - ya)
        dy = s * (xb - xa) + c * (yb - ya)
        n = np.array([-dy, dx]) / np.hypot(dx, dy)
        if viscous:
            np.testing.assert_allclose(face, wv, atol=1e-13)
        else:
            assert abs((face - wv) @ n) < 1e-13


@pytest.mark.parametrize("moving", [False, True])
def test_converged_time_steps_satisfy_implicit_euler_then_bdf2(moving):
    """eq. (nonlin-eq): after converged steps, (u1 - u0)/dt + F(u1) = 0 (first step, implicit
    Euler) and (3u2 - 4u1 + u0)/(2 dt) + F(u2) = 0 (BDF2), with F the steady residual at the
    same grid position, evaluated by a second oracle instance."""
    ni, nj = 32, 8
    g = make_cgrid(ni, nj, wall_spacing=2e-3)
    kw = dict(nlevels=2, mach=0.5, alpha_deg=1.0, cfl=1e4)
    o = O.Oracle(g, O.make_params(**kw))
    o.solve(1e-3, 300)                  # start from a partly converged state (a real transient)
    u0 = o.get_state()
    dt = 0.25
    states = [u0]
    ref = O.Oracle(g, O.make_params(**kw))
    for step in (1, 2):
        if moving:
            o.set_motion(*_pitch(step * dt))
        nc, hist = o.dual_time_step(dt, 1e-10, 400)
        assert 0 < nc < 400
        states.append(o.get_state())
        if moving:
            ref.set_motion(*_pitch(step * dt))
        ref.set_state(states[-1])
        F, _, _ = ref.residual()
        if step == 1:
            dudt = (states[1] - states[0]) / dt
        else:
            dudt = (3 * states[2] - 4 * states[1] + states[0]) / (2 * dt)
        assert np.abs(dudt + F).max() < 1e-7 * np.abs(F).max()
