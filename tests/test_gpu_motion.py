"""GPU parity with the oracle on a pitching grid (rigid rotation, ALE fluxes, moving walls)
and for dual time stepping (implicit Euler first step, then BDF2)."""
import numpy as np
import pytest

from synth.cgrid import make_cgrid
from tests.helpers import make_pair, perturbed_state, rel_err

pytestmark = pytest.mark.gpu


def _pitch(t, amp=np.radians(2.0), omega=0.4):
    return -amp * np.sin(omega * t), -amp * omega * np.cos(omega * t)


@pytest.mark.parametrize("viscous", [0, 1])
@pytest.mark.parametrize("level", [1, 0])
def test_residual_and_blocks_on_a_pitching_grid(viscous, level):
    ni, nj, nw = 72, 20, 8
    g = make_cgrid(ni, nj, n_wake=nw, wall_spacing=1e-3)
    o, s = make_pair(g, nlevels=2, viscous=viscous, mach=0.6, alpha_deg=0.5, re=1e5)
    for solver in (o, s):
        solver.set_motion(0.04, 0.03)
    ni_l, nj_l, _ = o.dims(level)
    u = perturbed_state(0.6, 0.5, nj_l, ni_l, amp=0.03, seed=2)
    o.set_state(u, level); s.set_state(u, level)
    Fo, _, _ = o.residual(level)
    Fg, _, _ = s.residual(level)
    assert rel_err(Fg, Fo) < 1e-11
    for a, b in zip(s.face_blocks(level), o.face_blocks(level)):
        assert rel_err(a, b) < 1e-12


def test_pitching_dual_time_steps_match_the_oracle():
    """Three physical steps (implicit Euler, then BDF2) of the pitching airfoil, each
    converged in pseudo time; states and per-step cycle counts agree."""
    g = make_cgrid(64, 16, wall_spacing=2e-3)
    o, s = make_pair(g, nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    for solver in (o, s):
        solver.solve(1e-4, 200)
    dt = 2 * np.pi / 0.4 / 64
    for step in (1, 2, 3):
        for solver in (o, s):
            solver.set_motion(*_pitch(step * dt))
        nco, ho = o.dual_time_step(dt, 1e-9, 300)
        code, ncg, hg = s.dual_time_step(dt, 1e-9, 300)
        assert code == 0 and nco == ncg, (step, nco, ncg)
        m = ho > 1e-12 * ho[0]
        assert np.all(np.abs(hg - ho)[m] <= 1e-7 * ho[m] + 1e-13 * ho[0])
        assert rel_err(s.get_state(), o.get_state()) < 1e-9
