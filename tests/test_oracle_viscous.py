"""Closed-form pins of the oracle's thin-layer viscous flux (section 2) in plane Couette flow.

u = a y, v = 0 with constant density and pressure is an exact parallel-shear solution: the
convective fluxes balance in every cell (no mass or energy crosses a j-face, the pressure
force on a j-face is the same above and below), the JST dissipation vanishes (the conservative
variables are at most quadratic in y, so their third differences are zero, and the pressure
sensor is zero), and the thin-layer stress on a j-face is exactly the continuum one, (mu +
mu_t) a, because the jump of a linear field across a face divided by the mean cell height is
its slope.  What remains per unit volume is the textbook balance

    x-momentum:  -d/dy((mu + mu_t) a)          = -a dmu_t/dy
    energy:      -d/dy(u (mu + mu_t) du/dy)    = -a^2 (mu + mu_t(y) + y dmu_t/dy)

i.e. the viscous heating -mu a^2 for a laminar flow.  A wrong sign, a dropped viscous work
term, the wrong face area, a face eddy viscosity other than the mean of the two cells, or a
gradient over a single cell's height instead of the mean, each breaks one of these.
"""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import CGrid, make_rect_grid

GAM = 1.4


def _couette(g, a, rho=1.0, p=1.0 / GAM):
    yc = 0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1])
    u = a * yc
    E = p / (GAM - 1.0) + 0.5 * rho * u * u
    one = np.ones_like(yc)
    return np.stack([rho * one, rho * u, 0.0 * one, E]), yc


def _interior(F):
    return F[:, 2:-2, 2:-2]


@pytest.mark.parametrize("re", [100.0, 2000.0])
def test_laminar_couette_flow_leaves_only_viscous_heating(re):
    ni, nj = 12, 16
    g = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    a = 0.5
    u, yc = _couette(g, a)
    o = O.Oracle(g, O.make_params(nlevels=1, viscous=1, sensor=1, mach=0.5, alpha_deg=0.0, re=re))
    o.set_state(u)
    F, Fc, Fv = o.residual()
    mu = 1.0 / re
    assert np.abs(_interior(Fc)).max() < 1e-13
    expect = np.zeros_like(_interior(F))
    expect[3] = -mu * a * a
    assert np.abs(_interior(F) - expect).max() < 1e-13, np.abs(_interior(F) - expect).max()


def test_couette_flow_with_a_linear_eddy_viscosity():
    """mu_t = m0 + m1 y (frozen, given per cell): its face values are the means of the two cells,
    exact for a linear field, so the balance above holds to rounding."""
    ni, nj = 12, 16
    g = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    a, re, m0, m1 = 0.5, 1000.0, 2e-3, 5e-3
    u, yc = _couette(g, a)
    o = O.Oracle(g, O.make_params(nlevels=1, viscous=1, turb=1, sensor=1, mach=0.5, alpha_deg=0.0, re=re))
    o.set_state(u)
    o.set_mut(m0 + m1 * yc)
    F, _, _ = o.residual()
    mu = 1.0 / re
    expect = np.zeros((4, nj, ni))
    expect[1] = -a * m1
    expect[3] = -a * a * (mu + m0 + 2.0 * m1 * yc)
    err = np.abs(_interior(F) - _interior(expect)).max()
    assert err < 1e-13, err


def test_couette_viscous_flux_on_a_stretched_grid():
    """Cells growing geometrically in y (ratio r).  The JST dissipation no longer vanishes (a
    linear field in y is not linear in the cell index), so the viscous contribution is taken as
    the residual with the viscous flux minus the same residual without it (same sensor, same
    dissipation, interior cells).  The gradient across a j-face (jump over the mean of the two
    cell heights) is still the exact slope of a linear velocity, so the x-momentum contribution
    stays zero; with a single cell's height it would not.  The viscous work uses the mean of the
    two cells' velocities at a face, which on a geometric grid makes the heating
    -mu a^2 (1 + (r - 1)^2 / (4 r))."""
    ni, nj, r = 12, 16, 1.25
    g0 = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    h = 0.01 * r ** np.arange(nj)
    yv = np.concatenate([[0.0], np.cumsum(h)])
    y = np.repeat(yv[:, None], ni + 1, axis=1)
    g = CGrid(ni, nj, 0, g0.x.copy(), np.ascontiguousarray(y), {})
    a, re = 0.5 / yv[-1], 100.0
    u, yc = _couette(g, a)
    F = {}
    for viscous in (1, 0):
        o = O.Oracle(g, O.make_params(nlevels=1, viscous=viscous, sensor=1, mach=0.5, alpha_deg=0.0, re=re))
        o.set_state(u)
        F[viscous] = _interior(o.residual()[0])
    visc = F[1] - F[0]
    mu = 1.0 / re
    rounding = 1e-13 * np.abs(F[0]).max()
    assert np.abs(visc[:3]).max() <= rounding, (np.abs(visc[:3]).max(), rounding)
    heat = visc[3] / (-mu * a * a)
    assert np.abs(heat - (1.0 + (r - 1.0) ** 2 / (4.0 * r))).max() < 1e-9, heat


def _viscous_part(g, u, re, mut=None, **kw):
    """Residual with the viscous flux minus the same residual without it (interior cells)."""
    F = {}
    for viscous in (1, 0):
        o = O.Oracle(g, O.make_params(nlevels=1, viscous=viscous, turb=1 if mut is not None else 0, sensor=1,
                                      mach=0.5, alpha_deg=0.0, re=re, **kw))
        o.set_state(u)
        if mut is not None:
            o.set_mut(mut)
        F[viscous] = _interior(o.residual()[0])
    # rounding scale: the larger of the two residuals
    return F[1] - F[0], max(np.abs(F[0]).max(), np.abs(F[1]).max())


def _rotated(g, th):
    """The grid turned by th about the origin (a rotated Cartesian grid: j-faces with both
    components of their area vector)."""
    c, s = np.cos(th), np.sin(th)
    return CGrid(g.ni, g.nj, g.n_wake, np.ascontiguousarray(c * g.x - s * g.y), np.ascontiguousarray(s * g.x + c * g.y), {})


@pytest.mark.parametrize("th", [0.0, 0.4])
def test_normal_stress_work_carries_the_bulk_term(th):
    """Velocity b y' along the grid's normal direction n, y' the distance along n (on the
    unturned grid v = b y): the normal stress on a j-face is mu (2 b - (2/3) b) = (4/3) mu b,
    uniform, so the momentum contributions vanish and its work (4/3) mu b^2 is the energy
    contribution (Stokes' hypothesis for the bulk viscosity).  Turned by th, every stress
    component enters the face fluxes."""
    ni, nj = 12, 16
    g0 = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    g = _rotated(g0, th)
    b, re, rho, p = 0.3, 200.0, 1.0, 1.0 / GAM
    yc = 0.25 * (g0.y[:-1, :-1] + g0.y[:-1, 1:] + g0.y[1:, 1:] + g0.y[1:, :-1])
    vn = b * yc
    uu, vv = -np.sin(th) * vn, np.cos(th) * vn
    one = np.ones_like(yc)
    u = np.stack([rho * one, rho * uu, rho * vv, p / (GAM - 1.0) + 0.5 * rho * vn * vn])
    visc, scale = _viscous_part(g, u, re)
    assert np.abs(visc[:3]).max() <= 1e-12 * scale
    assert np.abs(visc[3] / (-(4.0 / 3.0) * b * b / re) - 1.0).max() < 1e-10


@pytest.mark.parametrize("th", [0.4, -1.1])
def test_couette_flow_on_a_turned_grid(th):
    """The laminar Couette balance with grid and flow turned by th: shear along the grid's i
    direction t, growing along n; viscous contribution (0, 0, 0, -mu a^2)."""
    ni, nj = 12, 16
    g0 = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    g = _rotated(g0, th)
    a, re, rho, p = 0.5, 150.0, 1.0, 1.0 / GAM
    yc = 0.25 * (g0.y[:-1, :-1] + g0.y[:-1, 1:] + g0.y[1:, 1:] + g0.y[1:, :-1])
    ut = a * yc
    one = np.ones_like(yc)
    u = np.stack([rho * one, rho * np.cos(th) * ut, rho * np.sin(th) * ut, p / (GAM - 1.0) + 0.5 * rho * ut * ut])
    visc, scale = _viscous_part(g, u, re)
    assert np.abs(visc[:3]).max() <= 1e-12 * scale
    assert np.abs(visc[3] / (-a * a / re) - 1.0).max() < 1e-10


@pytest.mark.parametrize("mut0", [0.0, 4e-3])
def test_heat_conduction_uses_both_prandtl_numbers(mut0):
    """Fluid at rest at uniform pressure with the enthalpy h = cp p / rho = h0 + beta y^2 at the cell
    centres: the face gradient of h is exactly 2 beta y_face, and the conduction term of the energy
    equation is d/dy((mu/Pr + mu_t/Pr_t) dh/dy) = 2 beta (mu/Pr + mu_t/Pr_t) for a uniform mu_t."""
    ni, nj = 12, 16
    g = make_rect_grid(ni, nj, lx=1.2, ly=1.0)
    re, pr, prt, p, h0, beta = 300.0, 0.72, 0.9, 1.0 / GAM, 2.5, 0.4
    yc = 0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1])
    h = h0 + beta * yc * yc
    rho = GAM / (GAM - 1.0) * p / h
    one = np.ones_like(yc)
    u = np.stack([rho, 0.0 * one, 0.0 * one, p / (GAM - 1.0) * one])
    visc, scale = _viscous_part(g, u, re, mut=mut0 * one if mut0 else None, pr=pr, prt=prt)
    assert np.abs(visc[:3]).max() <= 1e-13 * scale
    expect = -2.0 * beta * (1.0 / (re * pr) + mut0 / prt)
    assert np.abs(visc[3] / expect - 1.0).max() < 1e-10, visc[3] / expect
