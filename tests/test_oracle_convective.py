"""Closed-form pin of the oracle's central convective flux (section 2).

Uniform velocity V = (U, W), density and pressure linear in x and y, on a Cartesian grid of
uniform cells (also turned by an angle): the average of two neighbouring cells is the value at
their common face, so the central flux of every linear flux component is exact, and the
residual per unit volume is the divergence of the Euler flux,
    (V.grad rho,  U V.grad rho + dp/dx,  W V.grad rho + dp/dy,
     gamma/(gamma-1) V.grad p + |V|^2/2 V.grad rho),
the last from E + p = gamma p/(gamma-1) + rho |V|^2/2.  The JST dissipation vanishes: w is
linear (no third differences) and the pressure switch sees no second difference.  A missing
pressure term, E in place of E + p, or a wrong face-vector orientation breaks it.
"""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import CGrid, make_rect_grid

GAM = 1.4


@pytest.mark.parametrize("th", [0.0, 0.7])
def test_linear_fields_give_the_flux_divergence(th):
    ni, nj = 14, 12
    g0 = make_rect_grid(ni, nj, lx=1.4, ly=0.9)
    c, s = np.cos(th), np.sin(th)
    g = CGrid(ni, nj, 0, np.ascontiguousarray(c * g0.x - s * g0.y), np.ascontiguousarray(s * g0.x + c * g0.y), {})
    xc = 0.25 * (g.x[:-1, :-1] + g.x[:-1, 1:] + g.x[1:, 1:] + g.x[1:, :-1])
    yc = 0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1])
    U, W = 0.35, -0.2
    grho, gp = np.array([0.08, -0.05]), np.array([-0.04, 0.03])
    rho = 1.0 + grho[0] * xc + grho[1] * yc
    p = 0.7 + gp[0] * xc + gp[1] * yc
    E = p / (GAM - 1.0) + 0.5 * rho * (U * U + W * W)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.5, alpha_deg=0.0))
    o.set_state(np.stack([rho, rho * U, rho * W, E]))
    F, Fc, Fv = o.residual()
    vr = U * grho[0] + W * grho[1]                       # V . grad rho
    vp = U * gp[0] + W * gp[1]                           # V . grad p
    want = np.array([vr, U * vr + gp[0], W * vr + gp[1], GAM / (GAM - 1.0) * vp + 0.5 * (U * U + W * W) * vr])
    inner = (slice(None), slice(2, nj - 2), slice(2, ni - 2))
    got = F[inner]
    err = np.abs(got - want[:, None, None]).max()
    assert err < 1e-12, (err, got[:, 0, 0], want)
    assert np.abs(Fv[inner]).max() < 1e-12
