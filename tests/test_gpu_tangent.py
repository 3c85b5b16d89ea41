"""The forward-mode linearization of the residual (kernels_tangent.cu; fasw_tangent_residual and
the default Jacobian assembly of the adjoint).

Checks, each against something independent of the tangent code: (1) its value part reproduces
the residual kernels' F (the same discrete operator); (2) its tangent equals central differences
of the GPU residual kernels along the same direction (to the differences' truncation); (3) the
assembled Jacobian times a vector equals the matrix-free tangent (colouring and extraction), and
the dot-product identity <w, J v> = <J^T w, v> holds between the matrix-free tangent and the
assembled transpose; (4) the assembled Jacobian agrees with the coloured central-difference
assembly of the library and with the oracle's sparse Jacobian (built by its own differences of
the C++ residual)."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from synth.cgrid import make_cgrid
from tests.helpers import make_pair, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "euler": dict(viscous=0, turb=0, mach=0.7, alpha_deg=1.5),
    "laminar": dict(viscous=1, turb=0, mach=0.5, alpha_deg=1.0, re=1e4),
    "fvs": dict(viscous=0, turb=0, mach=0.7, alpha_deg=1.5, flux="fvs"),
}


def _setup(kind, ni=48, nj=12, nw=6, seed=3):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=seed, wall_spacing=2e-3)
    o, s = make_pair(g, nlevels=1, d_cut=0.4, **CASES[kind])
    kw = CASES[kind]
    u = perturbed_state(kw["mach"], kw["alpha_deg"], nj, ni, amp=0.02, seed=seed)
    o.set_state(u); s.set_state(u)
    return g, o, s, u


@pytest.mark.parametrize("kind", list(CASES))
def test_value_part_is_the_residual(kind):
    g, o, s, u = _setup(kind)
    v = np.random.default_rng(1).standard_normal(u.shape)
    dF, F = s.tangent_residual(v, with_value=True)
    Fk, _, _ = s.residual()
    assert rel_err(F, Fk) < 1e-13
    assert rel_err(F, o.residual()[0]) < 1e-11


@pytest.mark.parametrize("kind", list(CASES))
def test_tangent_equals_differences_of_the_residual_kernels(kind):
    g, o, s, u = _setup(kind)
    v = np.random.default_rng(2).standard_normal(u.shape) * np.abs(u)
    dF = s.tangent_residual(v)
    eps = 1e-6
    s.set_state(np.ascontiguousarray(u + eps * v)); Fp = s.residual()[0]
    s.set_state(np.ascontiguousarray(u - eps * v)); Fm = s.residual()[0]
    s.set_state(u)
    fd = (Fp - Fm) / (2 * eps)
    assert rel_err(dF, fd) < 1e-6


@pytest.mark.parametrize("kind", list(CASES))
def test_assembled_jacobian_is_the_tangent(kind):
    g, o, s, u = _setup(kind)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(u.shape)
    w = rng.standard_normal(u.shape)
    s.adjoint_jacobian(1e-6)                      # forward-mode assembly (the default)
    Jv = s.adjoint_apply(v)
    dF = s.tangent_residual(v)
    assert rel_err(Jv, dF) < 1e-12
    JTw = s.adjoint_apply(w, transpose=True)
    lhs, rhs = float(np.sum(w * dF)), float(np.sum(JTw * v))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(w * dF).sum() + np.abs(JTw * v).sum())
    # against the coloured central-difference assembly of the same residual kernels
    s.adjoint_set_jacobian("differences")
    s.adjoint_jacobian(1e-6)
    Jv_fd = s.adjoint_apply(v)
    assert rel_err(Jv_fd, Jv) < 1e-6
    # and the objective gradients
    s.adjoint_set_jacobian("tangent")
    s.adjoint_jacobian(1e-6)
    g_t = s.adjoint_objective_gradient(1)
    s.adjoint_set_jacobian("differences")
    s.adjoint_jacobian(1e-6)
    g_fd = s.adjoint_objective_gradient(1)
    assert rel_err(g_t, g_fd) < 1e-6


@pytest.mark.parametrize("kind", ["euler", "laminar"])
def test_tangent_against_the_oracles_jacobian(kind):
    g, o, s, u = _setup(kind, ni=32, nj=8, nw=4, seed=5)
    J, gL, gD = OA.jacobian(o, CASES[kind]["alpha_deg"], 1e-6)
    v = np.random.default_rng(6).standard_normal(u.shape)
    dF = s.tangent_residual(v)
    assert rel_err(dF.ravel(), J @ v.ravel()) < 1e-6
    s.adjoint_jacobian(1e-6)
    assert rel_err(s.adjoint_objective_gradient(1).ravel(), gD) < 1e-6


def test_symmetric_flow_gives_a_symmetric_gradient():
    """Symmetric airfoil at zero incidence: the switches tie exactly across the wake cut and on the
    symmetry line.  The forward-mode Jacobian takes the central derivative at a tie, so the drag
    gradient of a bump on the upper surface is minus that of its mirror bump on the lower surface,
    as with the central-difference assembly."""
    import paper_1710_04875_gb300 as P
    from synth.shape import bump_fields
    from tests.helpers import pair_params
    g = make_cgrid(64, 16, wall_spacing=2e-3)
    _, pg = pair_params(nlevels=2, mach=0.6, alpha_deg=0.0, cfl=1e4)
    V = bump_fields(g, 2)
    out = {}
    for mode in ("tangent", "differences"):
        s = P.Solver(g, pg)
        s.adjoint_set_jacobian(mode)
        code, nc, hist = s.solve(1e-12, 2000)
        assert code == 0
        s.adjoint_jacobian(1e-6)
        lam, code, it, rr = s.adjoint_solve(1, tol=1e-11, max_iters=1500, restart=60)
        assert code == 0
        out[mode] = s.adjoint_shape_gradient(1, lam, V)
        s.close()
    gt, gd = out["tangent"], out["differences"]
    assert abs(gt[0] + gt[1]) <= 1e-6 * abs(gt[0]), gt
    # central differences of complete solves on the deformed grids (the difference-assembled
    # Jacobian carries its own O(h) averaging at the near-ties: 1e-3 from either)
    from synth.shape import deformed
    h = 1e-6
    fd = []
    for k in range(V.shape[0]):
        vals = []
        for sgn in (1.0, -1.0):
            e = np.zeros(V.shape[0])
            e[k] = sgn * h
            s = P.Solver(deformed(g, e, V), pg)
            code, nc, hist = s.solve(1e-13, 3000)
            assert code == 0
            vals.append(s.force_coefficients()[1])
            s.close()
        fd.append((vals[0] - vals[1]) / (2 * h))
    assert rel_err(gt, np.array(fd)) < 1e-4, (gt, fd)
    assert rel_err(gd, gt) < 1e-3, (gt, gd)


@pytest.mark.parametrize("kind", ["euler", "laminar", "fvs", "rans"])
def test_tangent_equals_the_oracles_complex_step(kind):
    """The matrix-free tangent and the assembled forward-mode Jacobian against the oracle's
    complex-step derivative of its own residual (exact to rounding, no differencing step, no
    shared code): agreement to rounding.  RANS: the eddy viscosity of the state frozen on both
    sides (each computed by its own Baldwin-Lomax, equal to 1e-10)."""
    if kind == "rans":
        g = make_cgrid(48, 12, n_wake=6, jitter=0.03, seed=3, wall_spacing=2e-4)
        kw = dict(viscous=1, turb=1, mach=0.6, alpha_deg=2.0, re=1e6)
        o, s = make_pair(g, nlevels=1, d_cut=0.4, **kw)
        u = perturbed_state(0.6, 2.0, 12, 48, amp=0.02, seed=3)
        o.set_state(u); s.set_state(u)
        assert rel_err(s.get_mut(), o.compute_mut()) < 1e-10      # each side's own Baldwin-Lomax
        tol = 1e-9
    else:
        g, o, s, u = _setup(kind)
        tol = 1e-11
    v = np.random.default_rng(7).standard_normal(u.shape)
    _, dF_cs = o.residual_complex_step(v)
    assert rel_err(s.tangent_residual(v), dF_cs) < tol
    s.adjoint_jacobian(1e-6)
    assert rel_err(s.adjoint_apply(v), dF_cs) < tol
