"""GPU unsteady discrete adjoint (dual time stepping on a pitching grid, binomial
checkpointing) against the oracle and against differences of full unsteady GPU solves."""
import numpy as np
import pytest

import oracle as O
from oracle import unsteady_adjoint as U
from synth.cgrid import make_cgrid
from synth.shape import bump_fields, deformed
from tests.helpers import pair_params, rel_err

pytestmark = pytest.mark.gpu

AMP, OMEGA, XC, YC = np.radians(2.0), 0.4, 0.25, 0.0
DT = 2.0 * np.pi / OMEGA / 16
DROP, CYCLES = 1e-11, 400


def _steady(g, po, n=300):
    o = O.Oracle(g, po)
    for k in range(n):
        o.fas_cycle(k)
    return o.get_state()


@pytest.fixture(scope="module")
def euler_case():
    g = make_cgrid(64, 16, wall_spacing=2e-3)
    po, pg = pair_params(nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    u0 = _steady(g, po)
    V = bump_fields(g, 2)
    return g, po, pg, u0, V


def test_unsteady_adjoint_matches_the_oracle(euler_case):
    """Four steps (implicit Euler, then BDF2) from the same initial state: objective, shape
    gradient with u^0 fixed and the initial-state sensitivity."""
    import paper_1710_04875_gb300 as P
    g, po, pg, u0, V = euler_case
    N = 4
    Jo, go, g0o, _ = U.gradient(g, po, u0, V, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    s = P.Solver(g, pg)
    s.set_state(u0)
    s.adjoint_set_jacobian("differences")         # the oracle's definition: central differences
    Jg, gg, g0g, code, st = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, which=1, xc=XC, yc=YC, drop=DROP,
                                               max_cycles=CYCLES, tol=1e-11, max_iters=400, restart=60)
    assert code == 0, st
    assert abs(Jg - Jo) <= 1e-9 * abs(Jo)
    assert rel_err(gg, go) < 1e-6, (gg, go)
    assert rel_err(g0g, g0o) < 1e-6
    assert st["forward_steps"] == N and st["recomputed_steps"] == 0
    # the context is back at u^0 on the grid at rest
    assert rel_err(s.get_state(), u0) == 0.0
    s.close()


def test_laminar_unsteady_adjoint_matches_the_oracle():
    """Thin-layer viscous flux on the pitching no-slip wall (moving-wall ghosts, grid velocities in
    the viscous terms): three levels against the oracle."""
    import paper_1710_04875_gb300 as P
    g = make_cgrid(64, 16, wall_spacing=5e-3)
    kw = dict(nlevels=2, viscous=1, turb=0, mach=0.5, alpha_deg=0.0, re=5e3, cfl=1e3)
    po, pg = pair_params(**kw)
    u0 = _steady(g, po)
    V = bump_fields(g, 2)
    N = 3
    Jo, go, g0o, _ = U.gradient(g, po, u0, V, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    s = P.Solver(g, pg)
    s.set_state(u0)
    s.adjoint_set_jacobian("differences")         # the oracle's definition: central differences
    Jg, gg, g0g, code, st = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, which=1, xc=XC, yc=YC, drop=DROP,
                                               max_cycles=CYCLES, tol=1e-11, max_iters=600, restart=250)
    assert code == 0, st
    assert abs(Jg - Jo) <= 1e-9 * abs(Jo)
    assert rel_err(gg, go) < 1e-6, (gg, go)
    assert rel_err(g0g, g0o) < 1e-6
    s.close()


def test_rans_unsteady_adjoint_matches_the_oracle():
    """Thin-layer RANS with Baldwin-Lomax on the pitching grid: the eddy viscosity frozen at each
    level's value on both sides; three levels against the oracle."""
    import paper_1710_04875_gb300 as P
    g = make_cgrid(64, 16, wall_spacing=1e-3)
    kw = dict(nlevels=2, viscous=1, turb=1, mach=0.5, alpha_deg=0.0, re=1e5, cfl=100.0)
    po, pg = pair_params(**kw)
    o = O.Oracle(g, po)
    for k in range(400):
        o.fas_cycle(k)
    u0 = o.get_state()
    V = bump_fields(g, 2)
    N = 3
    drop = 1e-10
    Jo, go, g0o, _ = U.gradient(g, po, u0, V, AMP, OMEGA, XC, YC, DT, N, drop, CYCLES, 1)
    s = P.Solver(g, pg)
    s.set_state(u0)
    s.adjoint_set_jacobian("differences")         # the oracle's definition: central differences
    Jg, gg, g0g, code, st = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, which=1, xc=XC, yc=YC, drop=drop,
                                               max_cycles=CYCLES, tol=1e-11, max_iters=600, restart=250)
    assert code == 0, st
    assert abs(Jg - Jo) <= 1e-8 * abs(Jo)
    assert rel_err(gg, go) < 1e-5, (gg, go)
    assert rel_err(g0g, g0o) < 1e-5
    s.close()


def test_implicit_euler_unsteady_adjoint_matches_the_oracle(euler_case):
    """bdf_order 1: implicit Euler on every level (no second history term in the adjoint)."""
    import paper_1710_04875_gb300 as P
    g, po, pg, u0, V = euler_case
    N = 3
    po1 = O.make_params("AW3", nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4, bdf_order=1)
    Jo, go, g0o, _ = U.gradient(g, po1, u0, V, AMP, OMEGA, XC, YC, DT, N, DROP, CYCLES, 1)
    s = P.Solver(g, pg)
    s.set_state(u0)
    s.adjoint_set_jacobian("differences")         # the oracle's definition: central differences
    Jg, gg, g0g, code, st = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, which=1, xc=XC, yc=YC, bdf_order=1,
                                               drop=DROP, max_cycles=CYCLES, tol=1e-11, max_iters=400, restart=60)
    assert code == 0, st
    assert abs(Jg - Jo) <= 1e-9 * abs(Jo)
    assert rel_err(gg, go) < 1e-6
    assert rel_err(g0g, g0o) < 1e-6
    s.close()


def test_checkpointed_reverse_sweep_is_bit_identical(euler_case):
    """Binomial checkpointing with no, one and two stored levels recomputes states exactly
    (deterministic kernels), so the adjoint equals the store-every-level run bit for bit; the
    recomputed step count is the binomial optimum."""
    import paper_1710_04875_gb300 as P
    g, po, pg, u0, V = euler_case
    N = 8
    s = P.Solver(g, pg)
    s.set_state(u0)
    kw = dict(which=0, xc=XC, yc=YC, drop=1e-10, max_cycles=CYCLES, tol=1e-10, max_iters=400, restart=60)
    ref = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, **kw)
    for snaps in (0, 1, 2):
        out = s.unsteady_adjoint(AMP, OMEGA, DT, N, V, snapshots=snaps, **kw)
        assert out[0] == ref[0]
        assert np.array_equal(out[1], ref[1])
        assert np.array_equal(out[2], ref[2])
        assert out[4]["forward_steps"] == P.checkpoint_schedule(N, snaps)[1] > N
    s.close()


def _unsteady_objective(P, g, pg, N, which):
    s = P.Solver(g, pg)
    code, nc, hist = s.solve(1e-12, 2000)
    assert code == 0
    J = 0.0
    for n in range(1, N + 1):
        phi, phidot = U.pitch(n * DT, AMP, OMEGA)
        s.set_motion(phi, phidot, XC, YC)
        code, nc, hist = s.dual_time_step(DT, DROP, CYCLES)
        assert code == 0
        J += s.force_coefficients()[which] / N
    s.close()
    return J


def test_total_pitching_gradient_matches_differences_of_full_solves(euler_case):
    """Steady start on the deformed grid, then N pitching steps: the unsteady adjoint plus the
    steady adjoint of the initial state against central differences of complete GPU solves."""
    import paper_1710_04875_gb300 as P
    from paper_1710_04875_gb300.adjoint import pitching_gradient
    g, po, pg, u0, V = euler_case
    N = 6
    s = P.Solver(g, pg)
    code, nc, hist = s.solve(1e-12, 2000)
    assert code == 0
    J, grad, info = pitching_gradient(s, V, AMP, OMEGA, DT, N, which=1, xc=XC, yc=YC, snapshots=2, drop=DROP,
                                      max_cycles=CYCLES, tol=1e-10, max_iters=600, restart=60)
    s.close()
    assert info["unsteady_status"] == 0 and info["steady_status"] == 0, info
    assert abs(J - _unsteady_objective(P, g, pg, N, 1)) <= 1e-10 * abs(J)
    h = 1e-6
    for k in range(V.shape[0]):
        e = np.zeros(V.shape[0])
        e[k] = h
        fd = (_unsteady_objective(P, deformed(g, e, V), pg, N, 1)
              - _unsteady_objective(P, deformed(g, -e, V), pg, N, 1)) / (2 * h)
        # JST switches make the residual piecewise smooth; an O(1) error shows far above this
        assert abs(fd - grad[k]) <= 1e-3 * abs(grad[k]), (k, fd, grad[k])


def test_pitching_forces_autograd():
    """torch.autograd.Function around the pitching objective: the forward value is the time
    average of the dual-time steps, the backward gradient the unsteady adjoint's."""
    import torch
    import paper_1710_04875_gb300 as P
    from paper_1710_04875_gb300.adjoint import PitchingContext, PitchingForces, pitching_gradient
    g = make_cgrid(64, 16, wall_spacing=2e-3)
    _, pg = pair_params(nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    V = bump_fields(g, 2)
    N = 3
    actx = PitchingContext(lambda q: deformed(g, q, V), V, pg, AMP, OMEGA, DT, N, which=1, drop=DROP,
                           max_cycles=CYCLES, tol=1e-11)
    p = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    J = PitchingForces.apply(p, actx)
    J.backward()
    s = P.Solver(g, pg)
    s.solve(actx.steady_drop, actx.steady_cycles)
    Jr, gr, _ = pitching_gradient(s, V, AMP, OMEGA, DT, N, which=1, drop=DROP, max_cycles=CYCLES, tol=1e-11)
    s.close()
    assert abs(float(J.detach()) - Jr) <= 1e-12 * abs(Jr)
    assert rel_err(p.grad.numpy(), gr) < 1e-12



def test_library_pitching_objective_and_state_term(euler_case):
    """The library's time average of C_D over the pitching steps equals the step-by-step loop
    through the single-step calls, and the shape gradient without the explicit objective part
    (which -1) equals the full one minus the one at lam = 0."""
    import paper_1710_04875_gb300 as P
    g, po, pg, u0, V = euler_case
    N = 3
    s = P.Solver(g, pg)
    assert s.solve(1e-12, 2000)[0] == 0
    J, code, cycles = s.pitching_objective(AMP, OMEGA, DT, N, which=1, xc=XC, yc=YC, drop=DROP,
                                           max_cycles=CYCLES)
    s.close()
    assert code == 0 and cycles > 0
    assert abs(J - _unsteady_objective(P, g, pg, N, 1)) <= 1e-13 * abs(J)
    s = P.Solver(g, pg)
    assert s.solve(1e-12, 2000)[0] == 0
    lam = np.random.default_rng(5).standard_normal((4, g.nj, g.ni))
    full = s.adjoint_shape_gradient(1, lam, V)
    expl = s.adjoint_shape_gradient(1, 0.0 * lam, V)
    state = s.adjoint_shape_gradient(-1, lam, V)
    s.close()
    assert rel_err(state, full - expl) < 1e-12
