"""The adjoint's transposed smoother and transposed FAS cycle.

The linear operators are pinned to the primal itself: one primal smoothing step (or FAS cycle)
from a converged state plus a small perturbation eps*e moves the state by eps*(e - M J e) to
first order, M the linearised smoothing step (or cycle) as a solver of J; and the adjoint's
operators are the exact transposes of those (dot-product tests).  Then the cycle-preconditioned
adjoint solves the same system as the stage-loop-preconditioned one."""
import numpy as np
import pytest

from synth.cgrid import make_cgrid
from tests.helpers import pair_params, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

ALPHA = 1.25


def _direction(nj, ni, seed):
    """A smooth perturbation direction scaled like the conservative variables."""
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(nj), np.arange(ni), indexing="ij")
    e = np.zeros((4, nj, ni))
    for k, scale in enumerate((1.0, 0.6, 0.6, 2.5)):
        a, b = rng.uniform(0.5, 2.0, 2)
        e[k] = scale * np.sin(2 * np.pi * a * ii / ni + k) * np.cos(np.pi * b * jj / nj)
    return e


def _converged_solver(g, **kw):
    import paper_1710_04875_gb300 as P
    _, p = pair_params(**kw)
    s = P.Solver(g, p)
    code, nc, hist = s.solve(1e-13, 3000)
    assert hist[-1] <= 1e-12 * hist[0], (code, nc, hist[-1] / hist[0])
    return s


def _primal_response(s, u, e, eps, step):
    """(step(u + eps e) - step(u) - eps e) / eps for one primal smoothing step or FAS cycle."""
    s.set_state(u)
    step()
    a = s.get_state()
    s.set_state(u + eps * e)
    step()
    b = s.get_state()
    s.set_state(u)
    return (b - a - eps * e) / eps


def test_linearised_smoothing_step_is_the_primals():
    g = make_cgrid(64, 16)
    s = _converged_solver(g, nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    u = s.get_state()
    e = _direction(16, 64, 1)
    s.adjoint_jacobian(1e-7)
    s.adjoint_set_precond_steps(1)
    cfl = 1e4
    lin = -s.adjoint_cycle_apply(s.adjoint_apply(e), cfl, kind="smoother", transpose=False)
    d = _primal_response(s, u, e, 1e-6, lambda: s.smooth(1, cfl))
    assert rel_err(d, lin) < 1e-4, rel_err(d, lin)
    s.close()


@pytest.mark.parametrize("gamma,cfl", [(1, 1e4), (2, 100.0)])
def test_linearised_fas_cycle_is_the_primals(gamma, cfl):
    """V-cycle at c* = 1e4 and W-cycle at c* = 100 (the 2-level W-cycle stalls at c* = 1e4 here)."""
    g = make_cgrid(64, 16)
    s = _converged_solver(g, nlevels=2, gamma_cycle=gamma, mach=0.6, alpha_deg=ALPHA, cfl=cfl)
    u = s.get_state()
    e = _direction(16, 64, 2)
    s.adjoint_jacobian(1e-7)
    lin = -s.adjoint_cycle_apply(s.adjoint_apply(e), cfl, kind="cycle", transpose=False)
    d = _primal_response(s, u, e, 1e-6, lambda: s.fas_cycle(100))
    assert rel_err(d, lin) < 1e-4, rel_err(d, lin)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_transposed_smoother_and_cycle_are_exact_transposes(precision):
    """<M b, v> = <b, M^T v> for the smoothing step and a 3-level W-cycle (wake cut, ragged
    strips); in mixed precision the transposed sweeps are FP32, so the identity holds to FP32
    accuracy only."""
    import paper_1710_04875_gb300 as P
    ni, nj, nw = 72, 20, 8
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=5)
    _, p = pair_params(nlevels=3, gamma_cycle=2, mach=0.6, alpha_deg=ALPHA, cfl=50.0, precision=precision)
    s = P.Solver(g, p)
    s.set_state(perturbed_state(0.6, ALPHA, nj, ni, amp=0.03, seed=9))
    s.adjoint_jacobian(1e-6)
    rng = np.random.default_rng(13)
    b = rng.standard_normal((4, nj, ni)); v = rng.standard_normal((4, nj, ni))
    tol = 1e-12 if precision == "fp64" else 1e-5
    for kind in ("smoother", "cycle"):
        if precision == "mixed":  # the forward operator exists in FP64 only; compare with FP64
            continue
        Mb = s.adjoint_cycle_apply(b, 50.0, kind=kind, transpose=False)
        MTv = s.adjoint_cycle_apply(v, 50.0, kind=kind, transpose=True)
        x, y = float(np.sum(Mb * v)), float(np.sum(b * MTv))
        assert abs(x - y) <= tol * np.linalg.norm(Mb) * np.linalg.norm(v), (kind, x, y)
    if precision == "mixed":
        _, p64 = pair_params(nlevels=3, gamma_cycle=2, mach=0.6, alpha_deg=ALPHA, cfl=50.0)
        s64 = P.Solver(g, p64)
        s64.set_state(perturbed_state(0.6, ALPHA, nj, ni, amp=0.03, seed=9))
        s64.adjoint_jacobian(1e-6)
        z32 = s.adjoint_cycle_apply(v, 50.0, kind="cycle", transpose=True)
        z64 = s64.adjoint_cycle_apply(v, 50.0, kind="cycle", transpose=True)
        assert rel_err(z32, z64) < 1e-4
        s64.close()
    s.close()


def test_cycle_preconditioned_adjoint_solves_the_rans_workload():
    """The 256x64 RANS workload at its 6-order state: the adjoint preconditioned by the
    transposed W-cycle and by the stage loop on J^T reach the same lambda, and the drag
    gradient of upper and lower bumps has the antisymmetry of the symmetric section."""
    import paper_1710_04875_gb300 as P
    g = make_cgrid(256, 64, wall_spacing=1e-5)
    kw = dict(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=0.5, alpha_deg=0.0, re=1e7, cfl=100.0)
    _, p = pair_params(**kw)
    s = P.Solver(g, p)
    code, nc, hist = s.solve(1e-6, 1500)
    assert code == 0
    out = {}
    for kind in ("cycle", "stage_loop"):
        s.adjoint_set_precond(kind)
        s.adjoint_jacobian(1e-6)
        lam, code, it, rr = s.adjoint_solve(1, tol=1e-9, max_iters=3000, restart=250)
        assert code == 0 and rr <= 1e-9, (kind, code, it, rr)
        out[kind] = (lam, it)
    assert rel_err(out["cycle"][0], out["stage_loop"][0]) < 1e-6
    # the section is symmetric and alpha = 0: a bump raising the upper surface changes the drag
    # as the same bump lowering the lower surface, i.e. dC_D/dp_upper = -dC_D/dp_lower, to the
    # symmetry of a state converged by 6 orders (measured 1e-3 relative here; a wrong sign or a
    # missing mirror coupling on one side is an O(1) error)
    from synth.shape import bump_fields
    grad = s.adjoint_shape_gradient(1, out["cycle"][0], bump_fields(g, 16))
    assert np.abs(grad[:8] + grad[8:]).max() <= 5e-3 * np.abs(grad).max(), grad
    s.close()


def _asymptotic_rate(norms, floor):
    """Mean per-iteration reduction over the last 10 iterations above `floor`."""
    n = [x for x in norms if x > floor]
    assert len(n) >= 12, len(n)
    return (n[-1] / n[-11]) ** 0.1


def test_adjoint_iteration_converges_at_the_primal_rate():
    """The adjoint iteration lam <- lam + C^T (g - J^T lam) has the iteration matrix (I - J C)^T,
    whose spectrum is that of the primal's linearised iteration I - C J: both reduce their
    residuals at the same asymptotic rate (and so does the nonlinear FAS iteration near its
    fixed point)."""
    g = make_cgrid(64, 16)
    s = _converged_solver(g, nlevels=2, gamma_cycle=1, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    s.adjoint_jacobian(1e-7)
    cfl = 1e4
    e = _direction(16, 64, 7)
    primal = []
    for _ in range(60):
        e = e - s.adjoint_cycle_apply(s.adjoint_apply(e), cfl, kind="cycle", transpose=False)
        primal.append(float(np.linalg.norm(e)))
    gD = s.adjoint_objective_gradient(1)
    lam = np.zeros_like(gD)
    adjoint = []
    for _ in range(60):
        r = gD - s.adjoint_apply(lam, transpose=True)
        adjoint.append(float(np.linalg.norm(r)))
        lam = lam + s.adjoint_cycle_apply(r, cfl, kind="cycle", transpose=True)
    rp = _asymptotic_rate(primal, 1e-9 * primal[0])
    ra = _asymptotic_rate(adjoint, 1e-9 * adjoint[0])
    print(f"asymptotic rates: linearised primal {rp:.4f}, adjoint {ra:.4f}")
    assert rp < 0.95 and abs(ra - rp) <= 0.05 * rp, (rp, ra)
    s.close()


def test_rans_gradient_matches_differences_of_frozen_eddy_viscosity_solves():
    """RANS (Baldwin-Lomax): the discrete adjoint holds mu_t at the converged state's value, so
    central differences of complete solves with mu_t frozen at that value (fasw_freeze_mut) are
    the derivative it computes.  Two bumps of the drag gradient against such differences."""
    import paper_1710_04875_gb300 as P
    from synth.shape import bump_fields, deformed
    g = make_cgrid(128, 32, wall_spacing=1e-4)
    kw = dict(nlevels=3, gamma_cycle=2, viscous=1, turb=1, mach=0.6, alpha_deg=2.0, re=1e6, cfl=100.0)
    _, p = pair_params(**kw)
    s = P.Solver(g, p)
    code, nc, hist = s.solve(1e-6, 3000)
    assert code == 0
    mut = s.get_mut()
    s.freeze_mut(mut)
    code, nc, hist = s.solve(1e-7, 4000)           # a further 7 orders with mu_t held
    assert code == 0
    u = s.get_state()
    np.testing.assert_array_equal(s.get_mut(), mut)
    V = bump_fields(g, 16)[[2, 11]]
    s.adjoint_jacobian(1e-6)
    lam, code, it, rr = s.adjoint_solve(1, tol=1e-11, max_iters=3000, restart=250)
    assert code == 0
    grad = s.adjoint_shape_gradient(1, lam, V)
    s.close()
    h = 1e-6
    for k in range(V.shape[0]):
        cd = []
        for sgn in (1.0, -1.0):
            e = np.zeros(V.shape[0])
            e[k] = sgn * h
            sd = P.Solver(deformed(g, e, V), p)
            sd.set_state(u)
            sd.freeze_mut(mut)
            code, nc, hist = sd.solve(1e-6, 4000)
            assert code == 0
            cd.append(sd.force_coefficients()[1])
            sd.close()
        fd = (cd[0] - cd[1]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-4 * abs(grad[k]), (k, fd, grad[k])
