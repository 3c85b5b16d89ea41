"""The stated parity targets on every RANS configuration, in both builds of the library: the
residual after one FAS cycle to 1e-11 relative and convergence histories to 1e-8 relative.

Both builds run the same kernels; ``perf`` contracts multiply-adds into FMAs, ``parity`` is
built with -fmad=false like the oracle (-ffp-contract=off), so only the order of operations
inside each formula differs between GPU and CPU there.  A history is compared cycle by cycle
while it is above the roundoff floor of the residual itself: the difference between the two
FP64 evaluations of the residual norm at one and the same state (GPU and oracle), which no
iteration can undercut."""
import numpy as np
import pytest

import oracle as O
from synth.cases import config_c3
from synth.cgrid import make_cgrid
from tests.helpers import pair_params, rel_err

pytestmark = pytest.mark.gpu

VARIANTS = ["perf", "parity"]


def _pair(g, variant, **kw):
    import paper_1710_04875_gb300 as P
    po, pg = pair_params(**kw)
    return O.Oracle(g, po), P.Solver(g, pg, variant=variant)


def _c2():
    return make_cgrid(256, 64, wall_spacing=1e-5), dict(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=0.5,
                                                        alpha_deg=0.0, re=1e7, cfl=100.0)


def _c3():
    c = config_c3()
    return c.grid(), dict(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=c.mach, alpha_deg=0.0, re=c.reynolds,
                          cfl=100.0)


def _c5():
    return make_cgrid(1024, 256, n_wake=128, wall_spacing=1e-5), dict(nlevels=5, gamma_cycle=2, viscous=1, turb=1,
                                                                      mach=0.75, alpha_deg=0.0, re=6.5e6, cfl=100.0)


def _floor(o, s):
    """Roundoff floor of the density-residual RMS: the GPU's and the oracle's residual at the
    GPU's current state (set on both sides)."""
    u = s.get_state()
    o.set_state(u)
    s.set_state(u)
    Fo = o.residual()[0]
    Fg = s.residual()[0]
    return float(np.sqrt(np.mean((Fg[0] - Fo[0]) ** 2))) + 1e-300


def _history_ok(hg, ho, floor, rel=1e-8):
    hg, ho = np.asarray(hg), np.asarray(ho)
    return np.all(np.abs(hg - ho) <= rel * ho + 4.0 * floor), np.max(np.abs(hg - ho) / ho)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", ["c2_256x64", "c3_512x128", "c5_1024x256"])
def test_one_cycle_residual_parity_rans(case, variant):
    """Residual F (every cell, every component) after one W-cycle from the free stream: 1e-11
    relative to max |F|, and the cycle's norm to 1e-12."""
    g, kw = {"c2_256x64": _c2, "c3_512x128": _c3, "c5_1024x256": _c5}[case]()
    o, s = _pair(g, variant, **kw)
    no, ng = o.fas_cycle(0), s.fas_cycle(0)
    assert abs(ng - no) <= 1e-12 * abs(no)
    assert rel_err(s.residual()[0], o.residual()[0]) < 1e-11
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_convergence_history_parity_c2(variant):
    """30 W-cycles of the 256x64 RANS workload (Baldwin-Lomax recomputed every cycle): the
    norm history to 1e-8 relative, the state to 1e-12."""
    g, kw = _c2()
    o, s = _pair(g, variant, **kw)
    ho = [o.fas_cycle(k) for k in range(30)]
    hg = [s.fas_cycle(k) for k in range(30)]
    assert rel_err(s.get_state(), o.get_state()) < 1e-12
    ok, worst = _history_ok(hg, ho, _floor(o, s))
    assert ok, worst
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_convergence_history_parity_c1(variant):
    """The 40-cycle history of the 128x32 Euler case (3-level V-cycle)."""
    g = make_cgrid(128, 32)
    o, s = _pair(g, variant, nlevels=3, mach=0.8, alpha_deg=1.25)
    ho = [o.fas_cycle(k) for k in range(40)]
    hg = [s.fas_cycle(k) for k in range(40)]
    ok, worst = _history_ok(hg, ho, _floor(o, s))
    assert ok, worst
    s.close()


def _pitch(t, amp=np.radians(2.0), omega=0.4):
    return -amp * np.sin(omega * t), -amp * omega * np.cos(omega * t)


@pytest.mark.parametrize("variant", VARIANTS)
def test_first_pitching_step_history_parity_c3(variant):
    """The 512x128 pitching case: ten steady cycles, then the first physical step (implicit
    Euler, moving walls and grid fluxes) for eight pseudo-time cycles from the same state:
    history to 1e-8, state to 1e-12."""
    g, kw = _c3()
    o, s = _pair(g, variant, **kw)
    for k in range(10):
        o.fas_cycle(k)
    s.set_state(o.get_state())
    dt = 2 * np.pi / 0.4 / 64
    for solver in (o, s):
        solver.set_motion(*_pitch(dt))
    nco, ho = o.dual_time_step(dt, 1e-14, 8)
    code, ncg, hg = s.dual_time_step(dt, 1e-14, 8)
    assert nco == ncg == 8
    assert rel_err(s.get_state(), o.get_state()) < 1e-12
    ok, worst = _history_ok(hg, ho, 0.0)
    assert ok, worst
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_dual_time_histories_to_1e8(variant):
    """Three physical steps (implicit Euler, then BDF2) of the pitching 64x16 Euler case, each
    converged nine orders in pseudo time: the same cycle counts, each cycle's norm to 1e-8
    relative above the residual's roundoff floor, the states to 1e-12."""
    g = make_cgrid(64, 16, wall_spacing=2e-3)
    o, s = _pair(g, variant, nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    for solver in (o, s):
        solver.solve(1e-4, 200)
    dt = 2 * np.pi / 0.4 / 64
    for step in (1, 2, 3):
        for solver in (o, s):
            solver.set_motion(*_pitch(step * dt))
        nco, ho = o.dual_time_step(dt, 1e-9, 300)
        code, ncg, hg = s.dual_time_step(dt, 1e-9, 300)
        assert code == 0 and nco == ncg, (step, nco, ncg)
        assert rel_err(s.get_state(), o.get_state()) < 1e-12
        floor = _floor(o, s)
        ok, worst = _history_ok(hg, ho, floor)
        assert ok, (step, worst, floor / ho[0])
    s.close()
