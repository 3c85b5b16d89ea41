"""Closed-form pins of the oracle's local pseudo-time step and of the JST fourth-difference
dissipation with Martinelli's radius scaling (section 2, eq. spectralcorrection).

On a Cartesian grid of cells dx x dy the mean face vectors of a cell are (dy, 0) and (0, dx),
so a cell's directional radii are r_xi = (|u| + a) dy and r_eta = (|v| + a) dx, and the local
step is c* dx dy / (r_xi + r_eta).

Fluid at rest at uniform pressure with a density that is a cubic in the cell index has no
convective residual (no mass or energy flux, a uniform pressure force) and no pressure switch
(eps2 = 0), and only the density component of w = (rho, rho u, rho v, rho H) varies, with the
constant third difference 6 c3.  The residual is then exactly the dissipation
    F_rho = (eps4_e - eps4_w) 6 c3 / (dx dy),   eps4 = r~_face / 32,
with r~ = r (1 + (r_other / r)^(2/3)) of each cell (a = sqrt(gamma p / rho) exact per cell) and
the face value the larger of its two cells' (the reading of the face radius).  A wrong Martinelli
exponent or ratio, a mean instead of the larger value, a wrong 1/32, or a sign error each
change it at O(1).
"""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_rect_grid

GAM = 1.4


@pytest.mark.parametrize("alpha_deg", [0.0, 30.0, -120.0])
def test_local_pseudo_time_step_closed_form(alpha_deg):
    ni, nj, lx, ly = 10, 6, 2.0, 0.45
    g = make_rect_grid(ni, nj, lx=lx, ly=ly)
    dx, dy = lx / ni, ly / nj
    rho, p, q = 0.8, 0.6, 0.7
    al = np.radians(alpha_deg)
    u, v = q * np.cos(al), q * np.sin(al)
    one = np.ones((nj, ni))
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.5, alpha_deg=0.0))
    o.set_state(np.stack([rho * one, rho * u * one, rho * v * one, (p / (GAM - 1.0) + 0.5 * rho * q * q) * one]))
    a = np.sqrt(GAM * p / rho)
    for cfl in (3.0, 1e4):
        expect = cfl * dx * dy / ((abs(u) + a) * dy + (abs(v) + a) * dx)
        assert np.allclose(o.pseudo_dt(cfl), expect, rtol=1e-13, atol=0.0)


def _martinelli(r, other):
    return r * (1.0 + (other / r) ** (2.0 / 3.0))


@pytest.mark.parametrize("direction", ["xi", "eta"])
def test_fourth_difference_dissipation_with_martinelli_radii(direction):
    ni, nj, lx, ly = 20, 20, 1.0, 0.37
    g = make_rect_grid(ni, nj, lx=lx, ly=ly)
    dx, dy = lx / ni, ly / nj
    p, c1, c3 = 0.7, 0.01, 3e-4
    k = np.arange(ni if direction == "xi" else nj) - 9.5
    prof = 1.0 + c1 * k + c3 * k ** 3
    rho = np.tile(prof, (nj, 1)) if direction == "xi" else np.tile(prof[:, None], (1, ni))
    zero = np.zeros((nj, ni))
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.5, alpha_deg=0.0))
    o.set_state(np.stack([rho, zero, zero, p / (GAM - 1.0) + zero]))
    F, Fc, Fv = o.residual()
    # closed form along the varying direction
    a = np.sqrt(GAM * p / prof)
    if direction == "xi":
        rt = _martinelli(a * dy, a * dx)
    else:
        rt = _martinelli(a * dx, a * dy)
    eps4 = np.maximum(rt[:-1], rt[1:]) / 32.0      # face between cells m and m+1
    d3 = 6.0 * c3                                   # third difference of the cubic
    n = len(prof)
    Frho = np.zeros(n)
    Frho[2:n - 2] = (eps4[2:n - 2] - eps4[1:n - 3]) * d3 / (dx * dy)
    inner = (slice(2, nj - 2), slice(2, ni - 2))
    got = F[0][inner]
    want = (np.tile(Frho, (nj, 1)) if direction == "xi" else np.tile(Frho[:, None], (1, ni)))[inner]
    assert np.abs(Frho[2:n - 2]).min() > 1e-8          # the dissipation does not vanish here
    assert np.allclose(got, want, rtol=1e-9, atol=1e-15), np.abs(got - want).max()
    assert np.abs(F[1:][(slice(None),) + inner]).max() < 1e-13
    assert np.abs(Fc[(slice(None),) + inner]).max() < 1e-13


@pytest.mark.parametrize("switch", ["pressure", "entropy"])
def test_switch_dissipation_on_an_odd_even_pressure(switch):
    """Fluid at rest, constant density, p = p0 + c (-1)^i.  The switch quantity q is p (Euler) or
    p / rho^gamma (viscous flows; the thin-layer flux has no jump across a j-face here), and
    |q+ - 2q + q-| / (q+ + 2q + q- + 0.001) is 4|c'| / (4 q0 + 0.001) in every cell (c', q0 the
    scaled amplitude and mean), above 1/64 here, so eps4 = max(0, r/32 - 2 eps2) = 0 and
    eps2 = s r with r the larger Martinelli radius of the two cells (the high-pressure cell's).
    Only rho H = gamma p / (gamma - 1) varies in w, so the energy residual is
    4 eps2 gamma/(gamma-1) c (-1)^i / (dx dy) and the other components vanish; with rho E in w
    the factor gamma would be missing."""
    ni, nj, lx, ly = 16, 8, 1.0, 0.3
    g = make_rect_grid(ni, nj, lx=lx, ly=ly)
    dx, dy = lx / ni, ly / nj
    rho, p0 = 1.1, 0.7
    c = 0.05 * p0
    sgn = (-1.0) ** np.arange(ni)
    p = np.tile(p0 + c * sgn, (nj, 1))
    zero = np.zeros((nj, ni))
    viscous = 1 if switch == "entropy" else 0
    o = O.Oracle(g, O.make_params(nlevels=1, viscous=viscous, sensor=viscous, mach=0.5, alpha_deg=0.0, re=1e3))
    o.set_state(np.stack([rho + zero, zero, zero, p / (GAM - 1.0)]))
    _, _, Fv = o.residual()
    scale = rho ** -GAM if switch == "entropy" else 1.0
    s = 4.0 * c * scale / (4.0 * p0 * scale + 0.001)
    assert 1.0 / 64.0 < s < 0.25
    a_hi = np.sqrt(GAM * (p0 + c) / rho)
    r = _martinelli(a_hi * dy, a_hi * dx)
    eps2 = s * r
    want = 4.0 * eps2 * GAM / (GAM - 1.0) * c * sgn / (dx * dy)
    inner = (slice(2, nj - 2), slice(2, ni - 2))
    got = Fv[3][inner]
    assert np.allclose(got, np.tile(want, (nj, 1))[inner], rtol=1e-11, atol=0.0), got[0] / want[2:ni - 2]
    assert np.abs(Fv[:3][(slice(None),) + inner]).max() < 1e-12 * np.abs(want).max()


def test_coarse_level_first_order_dissipation():
    """A coarse level (2x2 agglomeration of a Cartesian grid: cells 2dx x 2dy) uses first-order
    dissipation eps2 = s_c r with s_c = 0.25 and no fourth difference (the reading of the
    paper's coarse-grid scheme).  At rest, uniform pressure, density linear in the coarse cell
    index with slope c1: F_rho = -s_c c1 (r~_e - r~_w) / (4 dx dy), r~ the larger Martinelli
    radius of each face's two cells."""
    ni, nj, lx, ly = 32, 16, 1.0, 0.45
    g = make_rect_grid(ni, nj, lx=lx, ly=ly)
    o = O.Oracle(g, O.make_params(nlevels=2, mach=0.5, alpha_deg=0.0, s_coarse=0.25))
    nic, njc, _ = o.dims(0)
    assert (nic, njc) == (ni // 2, nj // 2)
    dx, dy = 2 * lx / ni, 2 * ly / nj
    p, c1 = 0.7, 0.03
    prof = 1.0 + c1 * (np.arange(nic) - 7.5)
    rho = np.tile(prof, (njc, 1))
    zero = np.zeros((njc, nic))
    o.set_state(np.stack([rho, zero, zero, p / (GAM - 1.0) + zero]), 0)
    o.set_forcing(np.zeros((4, njc, nic)), 0)
    F, Fc, Fv = o.residual(0)
    a = np.sqrt(GAM * p / prof)
    rt = _martinelli(a * dy, a * dx)
    rf = np.maximum(rt[:-1], rt[1:])             # face between coarse cells m and m+1
    Frho = np.zeros(nic)
    Frho[1:-1] = -0.25 * c1 * (rf[1:] - rf[:-1]) / (dx * dy)
    inner = (slice(1, njc - 1), slice(1, nic - 1))
    want = np.tile(Frho, (njc, 1))[inner]
    assert np.allclose(F[0][inner], want, rtol=1e-11, atol=0.0), F[0][inner][0] / want[0]
    assert np.abs(F[1:][(slice(None),) + inner]).max() < 1e-12 * np.abs(want).max()
