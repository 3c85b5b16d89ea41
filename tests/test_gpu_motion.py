"""GPU parity with the oracle on a pitching grid (rigid rotation, ALE fluxes, moving walls)
and for dual time stepping (implicit Euler first step, then BDF2)."""
import numpy as np
import pytest

import oracle as O
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


def test_pitching_dual_step_parity_full_size():
    """The first pitching step on the 512x128 RANS grid (M 0.8, Re 1e6, 4-level W-cycles, moving
    walls and grid fluxes at full size): three pseudo-time cycles from the same state."""
    from synth.cases import config_c3
    import paper_1710_04875_gb300 as P
    from tests.helpers import pair_params
    c = config_c3()
    g = c.grid()
    po, pg = pair_params(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=c.mach, alpha_deg=0.0, re=c.reynolds,
                         cfl=100.0)
    o, s = O.Oracle(g, po), P.Solver(g, pg)
    for k in range(10):
        o.fas_cycle(k)
    u = o.get_state()
    s.set_state(u)
    dt = 2 * np.pi / 0.4 / 64
    for solver in (o, s):
        solver.set_motion(*_pitch(dt))
    nco, ho = o.dual_time_step(dt, 1e-12, 3)
    code, ncg, hg = s.dual_time_step(dt, 1e-12, 3)
    assert nco == ncg == 3
    assert np.all(np.abs(hg - ho) <= 1e-8 * ho)
    assert rel_err(s.get_state(), o.get_state()) < 1e-12

