"""GPU discrete adjoint against the oracle's (coloured-difference Jacobian, sparse direct
transposed solve) and against differences of full GPU solves."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import adjoint as A
from synth.cgrid import make_cgrid
from synth.shape import bump_fields, deformed
from tests.helpers import make_pair, pair_params, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

ALPHA = 1.25


def _euler_pair(g, **kw):
    return make_pair(g, nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4, **kw)


@pytest.mark.parametrize("viscous", [0, 1])
def test_jacobian_products_match_the_oracle(viscous):
    g = make_cgrid(64, 16, jitter=0.02, seed=4)
    o, s = make_pair(g, nlevels=1, mach=0.6, alpha_deg=ALPHA, viscous=viscous, turb=0, re=1e4)
    u = perturbed_state(0.6, ALPHA, 16, 64, amp=0.03, seed=2)
    o.set_state(u); s.set_state(u)
    J, gL, gD = A.jacobian(o, ALPHA)
    s.adjoint_set_jacobian("differences")         # the oracle's definition: central differences
    s.adjoint_jacobian(1e-6)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((4, 16, 64)); w = rng.standard_normal((4, 16, 64))
    Jv = s.adjoint_apply(v)
    JTw = s.adjoint_apply(w, transpose=True)
    assert rel_err(Jv.ravel(), J @ v.ravel()) < 1e-6
    assert rel_err(JTw.ravel(), J.T @ w.ravel()) < 1e-6
    # dot-product test of the GPU's own pair of products
    a, b = float(np.sum(Jv * w)), float(np.sum(v * JTw))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert rel_err(s.adjoint_objective_gradient(0).ravel(), gL) < 1e-6
    assert rel_err(s.adjoint_objective_gradient(1).ravel(), gD) < 1e-6


def test_adjoint_preconditioner_is_the_transposed_primal_w():
    """z = S M^-T r with M the primal AW preconditioner: compare with the transpose of the
    oracle's M^-1 (applied column by column on a tiny grid with a wake cut), S = eta dt*."""
    ni, nj = 16, 6
    g = make_cgrid(ni, nj, n_wake=2, jitter=0.03, seed=7)
    o, s = make_pair(g, nlevels=1, mach=0.6, alpha_deg=ALPHA, d_cut=0.5)
    u = perturbed_state(0.6, ALPHA, nj, ni, amp=0.04, seed=8)
    o.set_state(u); s.set_state(u)
    n = ni * nj
    Minv = np.zeros((4 * n, 4 * n))
    for col in range(4 * n):
        e = np.zeros(4 * n); e[col] = 1.0
        Minv[:, col] = o.precond_apply(e.reshape(4, nj, ni), 50.0)[0].ravel()
    r = np.random.default_rng(9).standard_normal((4, nj, ni))
    S = 0.8 * o.pseudo_dt(50.0).ravel()                 # eta dt*
    ref = (Minv.T @ r.ravel()) * np.tile(S, 4)
    z = s.adjoint_precond_apply(r, 50.0)
    assert rel_err(z.ravel(), ref) < 1e-11


@pytest.mark.parametrize("ni,nj,nw,viscous", [(72, 20, 8, 0), (128, 32, 16, 1)])
def test_adjoint_preconditioner_transposes_the_primal_sweep_on_several_strips(ni, nj, nw, viscous):
    """<S M^-T r, v> = <r, M^-1 S v> with M^-1 the primal's own FP64 preconditioner sweep, on
    grids whose transposed sweep runs in several pipelined row strips with a ragged last strip
    and a wake cut: pins the transposed transfer blocks, including the wake-cut mirror blocks."""
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=5, wall_spacing=1e-3)
    _, s = make_pair(g, nlevels=1, mach=0.6, alpha_deg=ALPHA, viscous=viscous, re=1e4, d_cut=0.5)
    s.set_state(perturbed_state(0.6, ALPHA, nj, ni, amp=0.04, seed=6))
    rng = np.random.default_rng(12)
    r = rng.standard_normal((4, nj, ni)); v = rng.standard_normal((4, nj, ni))
    cfl = 50.0
    z = s.adjoint_precond_apply(r, cfl)
    S = 0.8 * s.pseudo_dt(cfl)
    w = s.precond_apply(S[None] * v, cfl)
    a, b = float(np.sum(z * v)), float(np.sum(r * w))
    assert abs(a - b) <= 1e-12 * np.linalg.norm(z) * np.linalg.norm(v)


def test_adjoint_smoother_is_the_transposed_stage_loop():
    """One smoothing step of the adjoint preconditioner equals the transposed AW3 stage loop
    x_i = x_0 + (alpha_i / eta) P^-T (r - J^T x_{i-1}) assembled here from the library's own
    J^T and P^-T products."""
    g = make_cgrid(64, 16)
    _, s = _euler_pair(g)
    u = perturbed_state(0.6, ALPHA, 16, 64, amp=0.03, seed=4)
    s.set_state(u)
    s.adjoint_jacobian(1e-6)
    r = np.random.default_rng(11).standard_normal((4, 16, 64))
    cfl = 1e4
    x = np.zeros_like(r)
    for a in (0.1481, 2.0 / 5.0, 1.0):                      # AW3 stage coefficients (eta = 0.8)
        x = a / 0.8 * s.adjoint_precond_apply(r - s.adjoint_apply(x, transpose=True), cfl)
    z = s.adjoint_precond_apply(r, cfl, steps=1)
    assert rel_err(z, x) < 1e-12


def test_force_coefficients_match_the_oracle():
    g = make_cgrid(64, 16)
    o, s = _euler_pair(g)
    u = perturbed_state(0.6, ALPHA, 16, 64, amp=0.03, seed=3)
    o.set_state(u); s.set_state(u)
    cl_o, cd_o = A.force_coefficients(*o.wall_force(), ALPHA)
    cl_g, cd_g = s.force_coefficients()
    assert abs(cl_g - cl_o) <= 1e-11 * abs(cl_o)
    assert abs(cd_g - cd_o) <= 1e-11 * max(abs(cd_o), 1e-3)


def test_adjoint_solution_and_shape_gradient_match_the_oracle():
    g = make_cgrid(64, 16)
    o, s = _euler_pair(g)
    code, nc, hist = s.solve(1e-13, 800)
    assert code == 0
    u = s.get_state()
    o.set_state(u)
    V = bump_fields(g, 4)
    _, p = pair_params(nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    po, _ = pair_params(nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    dL_o, dD_o, lamL_o, lamD_o = A.shape_gradient(g, po, u, None, V, ALPHA)
    s.adjoint_set_jacobian("differences")
    s.adjoint_jacobian(1e-6)
    lams = {}
    for which, lam_o, d_o in ((0, lamL_o, dL_o), (1, lamD_o, dD_o)):
        lam, code, it, rr = s.adjoint_solve(which, tol=1e-10, max_iters=1500, restart=60)
        assert code == 0 and rr <= 1e-10, (code, it, rr)
        assert rel_err(lam.ravel(), lam_o) < 1e-6
        grad = s.adjoint_shape_gradient(which, lam, V)
        assert rel_err(grad, d_o) < 1e-5
        lams[which] = (lam_o, d_o)
    # The default forward-mode Jacobian takes one branch of each |.| and max of the pressure
    # switch where the central differences average the two one-sided slopes (the converged
    # state has many near-zero second differences of p): the same lambda to 1e-4.
    s.adjoint_set_jacobian("tangent")
    s.adjoint_jacobian(1e-6)
    for which in (0, 1):
        lam, code, it, rr = s.adjoint_solve(which, tol=1e-10, max_iters=1500, restart=60)
        assert code == 0 and rr <= 1e-10, (code, it, rr)
        lam_o, d_o = lams[which]
        assert rel_err(lam.ravel(), lam_o) < 1e-4
        assert rel_err(s.adjoint_shape_gradient(which, lam, V), d_o) < 1e-4


@pytest.mark.parametrize("case", ["euler_64x16", "rans_256x64"])
def test_mixed_precision_adjoint_solves_the_same_system(case):
    """A mixed-precision context preconditions the adjoint GMRES with FP32 transposed sweeps
    (hyperplane-staged); flexible GMRES keeps the preconditioned vectors, so the adjoint reaches
    the same tolerance and the same lambda as the FP64 context (same Jacobian: both are
    differences of the FP64 residual, with the same frozen eddy viscosity).  The second case is
    the stiff 256x64 RANS workload at its 6-order state."""
    import paper_1710_04875_gb300 as P
    if case == "euler_64x16":
        g = make_cgrid(64, 16)
        kw = dict(nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
        drop = 1e-12
    else:
        g = make_cgrid(256, 64, wall_spacing=1e-5)
        kw = dict(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=0.5, alpha_deg=0.0, re=1e7, cfl=100.0)
        drop = 1e-6
    _, p64 = pair_params(**kw)
    _, p32 = pair_params(precision="mixed", **kw)
    s = P.Solver(g, p64)
    code, nc, hist = s.solve(drop, 1500)
    assert code == 0
    u = s.get_state()
    s.close()
    out = []
    for prm in (p64, p32):
        s = P.Solver(g, prm)
        s.set_state(u)
        s.get_mut()                  # Baldwin-Lomax at u, frozen for the adjoint (zero for Euler)
        s.adjoint_jacobian(1e-6)
        lam, code, it, rr = s.adjoint_solve(1, tol=1e-9, max_iters=3000, restart=250)
        assert code == 0 and rr <= 1e-9, (prm.precision, code, it, rr)
        out.append(lam)
        s.close()
    assert rel_err(out[1], out[0]) < 1e-6


@pytest.mark.parametrize("viscous", [0, 1])
def test_vertex_gradient_is_the_transposed_grid_derivative(viscous):
    """(dF/dX)^T lam with the objective's part, for every vertex, contracted with a displacement
    field in x and y, equals central differences of the oracle's residual and wall force over
    the displaced grids (any lam: the identity is linear)."""
    from synth.cgrid import CGrid
    g = make_cgrid(64, 16, wall_spacing=5e-3, jitter=0.02, seed=3)
    o, s = make_pair(g, nlevels=1, mach=0.6, alpha_deg=ALPHA, viscous=viscous, turb=0, re=5e3)
    u = perturbed_state(0.6, ALPHA, 16, 64, amp=0.03, seed=5)
    o.set_state(u); s.set_state(u)
    lam = np.random.default_rng(17).standard_normal((4, 16, 64))
    gx, gy = s.adjoint_vertex_gradient(1, lam)
    V = bump_fields(g, 4)
    DX, DY = V[0] - 0.5 * V[3], V[1] + 0.3 * V[2]
    pred = float(np.sum(gx * DX) + np.sum(gy * DY))
    h = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        gs = CGrid(g.ni, g.nj, g.n_wake, g.x + sgn * h * DX, g.y + sgn * h * DY, dict(g.meta))
        os_ = O.Oracle(gs, o.params)
        os_.set_state(u)
        vals.append((os_.residual()[0].ravel(), A.force_coefficients(*os_.wall_force(), ALPHA)[1]))
    fd = (vals[0][1] - vals[1][1]) / (2 * h) - lam.ravel() @ (vals[0][0] - vals[1][0]) / (2 * h)
    assert abs(pred - fd) <= 1e-6 * abs(fd), (pred, fd)
    # the same contraction of the y part is the library's per-field shape gradient
    ref = s.adjoint_shape_gradient(1, lam, V)
    via = np.array([np.sum(gy * V[k]) for k in range(4)])
    assert rel_err(via, ref) < 1e-6


def test_adjoint_gradient_matches_differences_of_gpu_solves():
    import paper_1710_04875_gb300 as P
    g = make_cgrid(64, 16)
    _, p = pair_params(nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    s = P.Solver(g, p)
    s.solve(1e-13, 800)
    u = s.get_state()
    V = bump_fields(g, 4)
    s.adjoint_jacobian(1e-6)
    lam, code, _, _ = s.adjoint_solve(0, tol=1e-10, max_iters=1500, restart=60)
    gradL = s.adjoint_shape_gradient(0, lam, V)
    h = 1e-5
    for k in (0, 2):
        cs = []
        for sgn in (1, -1):
            e = np.zeros(4); e[k] = sgn * h
            sk = P.Solver(deformed(g, e, V), p)
            sk.set_state(u)
            sk.solve(1e-13, 800)
            cs.append(sk.force_coefficients()[0])
            sk.close()
        fd = (cs[0] - cs[1]) / (2 * h)
        assert abs(fd - gradL[k]) <= 1e-3 * abs(gradL[k])   # piecewise-smooth JST residual


def test_autograd_function_gives_the_adjoint_gradient():
    from paper_1710_04875_gb300.adjoint import AdjointContext, ShapeForces
    g = make_cgrid(64, 16)
    _, p = pair_params(nlevels=2, mach=0.6, alpha_deg=ALPHA, cfl=1e4)
    V = bump_fields(g, 4)
    actx = AdjointContext(lambda q: deformed(g, q, V), V, p, drop=1e-13, max_cycles=800, tol=1e-10,
                          max_iters=1500, restart=60)
    q = torch.zeros(4, dtype=torch.float64, requires_grad=True)
    c = ShapeForces.apply(q, actx)
    (c[0] + 10.0 * c[1]).backward()
    s = actx.solver
    lamL, _, _, _ = s.adjoint_solve(0, tol=1e-10, max_iters=1500, restart=60)
    lamD, _, _, _ = s.adjoint_solve(1, tol=1e-10, max_iters=1500, restart=60)
    ref = s.adjoint_shape_gradient(0, lamL, V) + 10.0 * s.adjoint_shape_gradient(1, lamD, V)
    # the same adjoint systems solved twice to relative residual 1e-10
    assert rel_err(q.grad.numpy(), ref) < 1e-7
    assert all(actx.info[("adjoint", w)][0] == 0 for w in (0, 1)), actx.info
    assert actx.info["primal"][0] == 0
