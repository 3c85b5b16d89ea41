"""Pins of the oracle's Baldwin-Lomax eddy viscosity (the algebraic model that section 2 cites).

Two kinds of pins, neither of which re-runs the oracle's own steps:

- Closed forms.  Linear shear u = a |y|, v = 0 over a zero-thickness plate, on a grid whose
  wall-normal lines are vertical and evenly spaced (cells are rectangles of height h).  There
  the Green-Gauss vorticity of face-averaged velocities is exactly a in every cell (the wall
  ghost mirrors the velocity, so the wall face sees u = 0), the centroid-to-wall distance is
  exactly (j + 1/2) h and the wall shear is mu a, whatever the density profile.  F(y) = a y D(y) grows with y, so F_max sits
  on the last searched cell, U_dif is the largest speed, and the model reduces to closed forms
  in a, h, rho and mu that the test writes from the model's definition (inner mixing length
  with van Driest damping; outer Clauser form with F_wake and the Klebanoff factor; switch at
  the first cell where the inner value reaches the outer one) with the model's constants
  kappa = 0.4, A+ = 26, C_cp = 1.6, C_kleb = 0.3, C_wk = 0.25, K = 0.0168.  Two shear rates
  select the two branches of F_wake; wake lines (no damping, U_dif = max - min) are checked
  with u = U0 + a y across the cut.  A wrong constant, a dropped square or root, a signed
  vorticity, a wrong switch or Klebanoff exponent is an O(1) error here.
- Similarity.  The model is built from dimensional quantities only, so mu_t is homogeneous of
  degree one under each of: velocities x s with mu x s; density and energy x c with mu x c;
  lengths x L with mu x L.  With s, c, L powers of two every rounded operation commutes with
  the scaling and the identities hold bit for bit on any grid and state (here a jittered
  airfoil C-grid and a random boundary-layer-like state).  A wrong power of y, a missing
  density, a y+ without the square root or a U_dif without its square breaks one of them.
- A uniform stream gives mu_t = 0 on the wake lines (irrotational there); the model is local
  to wall-normal lines.

Cells whose value depends on the far-field ghost states (the outflow lines 0 and ni - 1, the
last row) are left out of the similarity comparisons: the far-field state is fixed by the
free stream and does not scale with the state.
"""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import CGrid, make_cgrid

GAM = 1.4
KAPPA, APLUS, CCP, CKLEB, CWK, KCL = 0.4, 26.0, 1.6, 0.3, 0.25, 0.0168


def _plate_grid(ni, nj, nw, h):
    """Zero-thickness plate C-grid: the wall/cut curve of the plate C-grid, with straight lines
    leaving it vertically (down on the lower side, up on the upper side, upstream at the
    leading edge), vertices every h along each line."""
    g0 = make_cgrid(ni, nj, thickness=0.0, n_wake=nw)
    x0, y0 = g0.x[0].copy(), g0.y[0].copy()
    mx = np.zeros(ni + 1)
    my = np.where(np.arange(ni + 1) < ni // 2, -1.0, 1.0)
    mx[ni // 2], my[ni // 2] = -1.0, 0.0
    d = h * np.arange(nj + 1)
    x = x0[None, :] + d[:, None] * mx[None, :]
    y = y0[None, :] + d[:, None] * my[None, :]
    return CGrid(ni, nj, nw, np.ascontiguousarray(x), np.ascontiguousarray(y), {})


def _state(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (GAM - 1.0) + 0.5 * rho * (u * u + v * v)])


def _mut(grid, u, re):
    o = O.Oracle(grid, O.make_params("AW3", nlevels=1, viscous=1, turb=1, mach=0.5, re=re))
    o.set_state(u)
    return o.compute_mut()


def _wall_line_closed_form(a, h, rho, mu, nj):
    """mu_t on a wall line under u = a y with density rho[j] per cell: (mu_t, inner, outer).
    The wall density is the wall cell's (the wall ghost carries the same density)."""
    y = (np.arange(nj) + 0.5) * h
    ys = y[nj // 2 - 1]                           # last searched cell: F = a y D(y) is increasing
    yplus = y * np.sqrt(rho[0] * mu * a) / mu     # sqrt(rho_w tau_w) y / mu_w with tau_w = mu a
    D = 1.0 - np.exp(-yplus / APLUS)
    inner = rho * (KAPPA * y * D) ** 2 * a
    Dm = D[nj // 2 - 1]
    fmax = a * ys * Dm
    udif = a * ys                                 # wall line: largest speed minus zero
    fwake = min(ys * fmax, CWK * ys * udif ** 2 / fmax)
    outer = KCL * CCP * rho * fwake / (1.0 + 5.5 * (CKLEB * y / ys) ** 6)
    cross = np.argmax(inner >= outer)
    assert inner[cross] >= outer[cross] and cross > 0
    mut = np.where(np.arange(nj) < cross, inner, outer)
    return mut, inner, outer


@pytest.mark.parametrize("h,branch", [(1.3e-3, "clauser"), (6e-5, "ymax_fmax")])
def test_linear_shear_over_plate_is_the_closed_form(h, branch):
    """Density falls through the layer (a heated wall), so the local and the wall density
    differ everywhere but in the wall cell; the velocity is still exactly linear."""
    ni, nj, nw = 64, 32, 8
    g = _plate_grid(ni, nj, nw, h)
    a, re = 100.0, 1e6
    mu = 1.0 / re
    yc = np.abs(0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1]))
    rho_of = lambda y: 0.7 + 0.3 * y / (y + 4.0 * h)
    u = _state(rho_of(yc), a * yc, np.zeros((nj, ni)), np.full((nj, ni), 100.0))
    m = _mut(g, u, re)
    expect, inner, outer = _wall_line_closed_form(a, h, rho_of((np.arange(nj) + 0.5) * h), mu, nj)
    # the two branches of F_wake: y_max F_max against C_wk y_max U_dif^2 / F_max
    ys = (nj // 2 - 0.5) * h
    Dm = 1.0 - np.exp(-ys * np.sqrt(rho_of(0.5 * h) * a / mu) / APLUS)
    assert (Dm > CWK / Dm) == (branch == "clauser")
    # no near-tie at the switch, so rounding cannot move it
    assert np.abs(inner / outer - 1.0).min() > 1e-6
    plate = [i for i in range(nw, ni - nw) if i not in (ni // 2 - 1, ni // 2)]  # leading-edge cells are not rectangles
    for i in plate:
        assert np.allclose(m[:, i], expect, rtol=1e-11, atol=0.0), (i, m[:, i], expect)


def test_linear_shear_across_wake_cut_is_the_closed_form():
    """Wake lines: no damping, U_dif = max - min over the searched cells, outer form from the
    cut outwards.  u = U0 + a y (y signed) is smooth across the cut, so the vorticity is a in
    every wake cell, the cut cells included."""
    ni, nj, nw = 64, 32, 8
    h, a, U0, rho, re = 1e-3, 50.0, 3.0, 1.0, 1e6
    g = _plate_grid(ni, nj, nw, h)
    yc = 0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1])
    u = _state(np.full((nj, ni), rho), U0 + a * yc, np.zeros((nj, ni)), np.full((nj, ni), 100.0))
    m = _mut(g, u, re)
    y = (np.arange(nj) + 0.5) * h
    ys = y[nj // 2 - 1]
    fmax = a * ys
    udif = a * (ys - y[0])                        # speeds U0 -+ a y are monotone along the line
    fwake = min(ys * fmax, CWK * ys * udif ** 2 / fmax)
    expect = KCL * CCP * rho * fwake / (1.0 + 5.5 * (CKLEB * y / ys) ** 6)
    for i in list(range(1, nw)) + list(range(ni - nw, ni - 1)):  # 0 and ni-1 border the outflow
        assert np.allclose(m[:, i], expect, rtol=1e-11, atol=0.0), (i, m[:, i], expect)


def _bl_state(g, seed):
    """A random boundary-layer-like state: velocity growing away from the wall at an angle,
    plus noise in every variable."""
    nj, ni = g.nj, g.ni
    rng = np.random.default_rng(seed)
    jj = np.arange(nj)[:, None] * np.ones((1, ni))
    f = 1.0 - np.exp(-(jj + 0.5) / 3.0)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, (nj, ni))
    uu = 0.6 * np.cos(0.05) * f + 0.02 * rng.standard_normal((nj, ni))
    vv = 0.6 * np.sin(0.05) * f + 0.02 * rng.standard_normal((nj, ni))
    p = (1.0 + 0.05 * rng.uniform(-1, 1, (nj, ni))) / GAM
    return rho, uu, vv, p


@pytest.fixture(scope="module")
def curvilinear():
    g = make_cgrid(64, 32, wall_spacing=1e-4, jitter=0.02, seed=3)
    rho, uu, vv, p = _bl_state(g, 5)
    re = 2.0 ** 20
    m = _mut(g, _state(rho, uu, vv, p), re)
    assert np.count_nonzero(m) > 0.9 * m.size
    return g, (rho, uu, vv, p), re, m


def _inner_cells(m):
    return m[:-1, 1:-1]


def test_velocity_scaling(curvilinear):
    g, (rho, uu, vv, p), re, m = curvilinear
    s = 4.0
    ms = _mut(g, _state(rho, s * uu, s * vv, p), re / s)
    np.testing.assert_array_equal(_inner_cells(ms), s * _inner_cells(m))


def test_density_scaling(curvilinear):
    g, (rho, uu, vv, p), re, m = curvilinear
    c = 2.0
    mc = _mut(g, _state(c * rho, uu, vv, c * p), re / c)
    np.testing.assert_array_equal(_inner_cells(mc), c * _inner_cells(m))


def test_length_scaling(curvilinear):
    g, (rho, uu, vv, p), re, m = curvilinear
    L = 0.5
    gl = CGrid(g.ni, g.nj, g.n_wake, L * g.x, L * g.y, {})
    ml = _mut(gl, _state(rho, uu, vv, p), re / L)
    np.testing.assert_array_equal(_inner_cells(ml), L * _inner_cells(m))


def test_lines_are_independent(curvilinear):
    """The vorticity stencil reaches the neighbouring lines only: changing the state of one
    body line changes mu_t on that line and its two neighbours and nowhere else."""
    g, (rho, uu, vv, p), re, m = curvilinear
    i0 = 30
    u2 = uu.copy()
    u2[:, i0] *= 1.3
    m2 = _mut(g, _state(rho, u2, vv, p), re)
    changed = np.flatnonzero(np.any(m2 != m, axis=0))
    assert set(changed) == {i0 - 1, i0, i0 + 1}, changed


def test_uniform_flow_has_no_eddy_viscosity_on_the_wake():
    """A uniform stream is irrotational away from the no-slip wall (at the wall it is a vortex
    sheet: the wall cells see the slip).  Wake lines see no wall: mu_t vanishes there."""
    g = make_cgrid(64, 32, wall_spacing=1e-4, jitter=0.02, seed=3)
    nj, ni, nw = g.nj, g.ni, g.n_wake
    w = O.free_stream(0.5, 2.0)
    u = np.broadcast_to(np.asarray(w)[:, None, None], (4, nj, ni)).copy()
    m = _mut(g, u, 1e6)
    wake = list(range(1, nw)) + list(range(ni - nw, ni - 1))
    # |omega| is rounding noise (the face vectors of a cell close); mu_t is far below mu
    assert np.abs(m[:, wake]).max() < 1e-12 * 1e-6
    assert m[0, nw:ni - nw].min() > 0.0          # the body lines see the slip at the wall
