"""Pins of the oracle's discrete adjoint (steady residual, frozen eddy viscosity).

- the coloured Jacobian equals the Jacobian built one column at a time (a missing stencil
  entry would put two cells of one colour into one residual stencil and corrupt entries);
- the adjoint (transposed-solve) shape gradient equals the direct (tangent-solve) gradient,
  an identity of linear algebra that pins the transposition;
- the adjoint gradient of lift and drag equals central differences of full nonlinear solves
  on deformed grids (Hicks-Henne bumps), to the accuracy a piecewise-smooth residual allows.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from oracle import adjoint as A
from synth.cgrid import make_cgrid
from synth.shape import bump_fields, deformed, hicks_henne
from tests.helpers import perturbed_state


def test_hicks_henne_bump_shape():
    x = np.linspace(0.0, 1.0, 201)
    for t in (0.1, 0.3, 0.5, 0.9):
        b = hicks_henne(x, t)
        assert b[0] == 0.0 and abs(b[-1]) < 1e-12
        assert abs(hicks_henne(np.array([t]), t)[0] - 1.0) < 1e-12
        assert np.all(b >= 0.0) and b.max() <= 1.0 + 1e-12


def test_deformation_keeps_cut_far_field_and_is_linear():
    g = make_cgrid(64, 16)
    V = bump_fields(g, 4)
    p = np.array([0.01, -0.02, 0.005, 0.01])
    d = deformed(g, p, V)
    assert np.array_equal(d.y[-1], g.y[-1])                       # far field fixed
    nw = g.n_wake
    assert np.array_equal(d.y[0, :nw + 1], g.y[0, :nw + 1])      # wake cut fixed
    assert np.array_equal(d.y[0, g.ni - nw:], g.y[0, g.ni - nw:])
    d2 = deformed(g, 2 * p, V)
    assert np.allclose(d2.y - g.y, 2 * (d.y - g.y), rtol=0, atol=1e-13)


@pytest.mark.parametrize("viscous", [0, 1])
def test_coloured_jacobian_equals_columnwise(viscous):
    g = make_cgrid(16, 6, n_wake=2, jitter=0.03, seed=3)
    p = O.make_params("AW3", nlevels=1, viscous=viscous, turb=0, sensor=viscous, mach=0.7, alpha_deg=2.0, re=1e4)
    o = O.Oracle(g, p)
    u = perturbed_state(0.7, 2.0, 6, 16, amp=0.05, seed=1)
    o.set_state(u)
    J, gL, gD = A.jacobian(o, 2.0, h_rel=1e-6)
    n = 16 * 6
    Jd = J.toarray()
    u0 = u.reshape(4, n)
    hs = 1e-6 * np.maximum(1.0, np.abs(u0))
    for m in range(4):
        for x in range(0, n, 7):
            up = u0.copy(); um = u0.copy()
            up[m, x] += hs[m, x]; um[m, x] -= hs[m, x]
            o.set_state(up.reshape(4, 6, 16)); Fp = o.residual()[0].ravel()
            o.set_state(um.reshape(4, 6, 16)); Fm = o.residual()[0].ravel()
            col = (Fp - Fm) / (2 * hs[m, x])
            assert np.allclose(Jd[:, m * n + x], col, rtol=0, atol=1e-9 * np.abs(col).max())


def _converged(g, p, n=600):
    o = O.Oracle(g, p)
    for k in range(n):
        o.fas_cycle(k)
    return o


def test_adjoint_gradient_equals_direct_gradient():
    g = make_cgrid(64, 16)
    p = O.make_params("AW3", nlevels=2, mach=0.6, alpha_deg=1.25, cfl=1e4)
    o = _converged(g, p, 300)
    u = o.get_state()
    V = bump_fields(g, 3)
    dL, dD, lamL, lamD = A.shape_gradient(g, p, u, None, V, 1.25)
    J, gL, gD = A.jacobian(o, 1.25)
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-6
        op, om = O.Oracle(deformed(g, e, V), p), O.Oracle(deformed(g, -e, V), p)
        op.set_state(u); om.set_state(u)
        dF = (op.residual()[0] - om.residual()[0]).ravel() / 2e-6
        du = spla.spsolve(J.tocsc(), -dF)          # tangent: J du/dp = -dF/dX V
        cLp, cDp = A.force_coefficients(*op.wall_force(), 1.25)
        cLm, cDm = A.force_coefficients(*om.wall_force(), 1.25)
        dL_direct = (cLp - cLm) / 2e-6 + gL @ du
        dD_direct = (cDp - cDm) / 2e-6 + gD @ du
        assert abs(dL_direct - dL[k]) <= 1e-9 * max(abs(dL[k]), 1.0)
        assert abs(dD_direct - dD[k]) <= 1e-9 * max(abs(dD[k]), 1.0)


def test_adjoint_gradient_matches_finite_differences_of_full_solves():
    g = make_cgrid(64, 16)
    p = O.make_params("AW3", nlevels=2, mach=0.6, alpha_deg=1.25, cfl=1e4)
    o = _converged(g, p)
    u = o.get_state()
    V = bump_fields(g, 4)
    dL, dD, _, _ = A.shape_gradient(g, p, u, None, V, 1.25)
    h = 1e-5
    for k in (0, 3):
        e = np.zeros(4); e[k] = h
        cs = []
        for sgn in (1, -1):
            ok = O.Oracle(deformed(g, sgn * e, V), p)
            ok.set_state(u)
            for c in range(300):
                ok.fas_cycle(c + 10)  # past the c* ramp
            cs.append(A.force_coefficients(*ok.wall_force(), 1.25))
        fdL = (cs[0][0] - cs[1][0]) / (2 * h)
        fdD = (cs[0][1] - cs[1][1]) / (2 * h)
        # The JST residual is piecewise smooth (max/min switches of the sensor, the radii and
        # eps4); the linearization holds the switches fixed, which agrees with differences of
        # full solves to a few 1e-4 here.  A wrong sign or a missing term is an O(1) error.
        assert abs(fdL - dL[k]) <= 1e-3 * abs(dL[k])
        assert abs(fdD - dD[k]) <= 1e-3 * max(abs(dD[k]), 0.05)
