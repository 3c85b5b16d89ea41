"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, invariants of the discretization, an independent
dense solve, or a finite-difference derivative.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid, make_rect_grid

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
GAM = 1.4


def _uniform(w, nj, ni):
    return np.broadcast_to(np.asarray(w)[:, None, None], (4, nj, ni)).copy()


def _perturbed(w, nj, ni, amp, seed):
    rng = np.random.default_rng(seed)
    return np.asarray(w)[:, None, None] * (1.0 + amp * rng.standard_normal((4, nj, ni)))


# ---------------------------------------------------------------- nondimensionalization
@pytest.mark.parametrize("key", ["u1_mach08_alpha45", "u3_mach08_alpha0"])
def test_free_stream_matches_paper_linearization_points(key):
    """Section 5.4 prints the two LFA linearization points at Mach 0.8."""
    ref = GOLD["linearization_points"][key]
    w = O.free_stream(ref["mach"], ref["alpha_deg"])
    np.testing.assert_allclose(w, ref["u"], atol=0.5 * 10 ** (-ref["digits"]))


def test_free_stream_sound_speed_and_pressure():
    w = O.free_stream(0.75, 3.0)
    rho, u, v = w[0], w[1] / w[0], w[2] / w[0]
    p = (GAM - 1) * (w[3] - 0.5 * rho * (u * u + v * v))
    assert abs(rho - 1) < 1e-15 and abs(math.hypot(u, v) - 1) < 1e-15
    assert abs(math.sqrt(GAM * p / rho) - 1 / 0.75) < 1e-14


# ---------------------------------------------------------------- metrics
def _shoelace(px, py):
    return 0.5 * np.sum(px * np.roll(py, -1) - np.roll(px, -1) * py)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_metrics_closure_and_total_volume(jitter):
    g = make_cgrid(64, 16, jitter=jitter, seed=5)
    o = O.Oracle(g, O.make_params(nlevels=3))
    for l in range(3):
        sxx, sxy, sex, sey, vol = o.metrics(l)
        clx = sxx[:, 1:] - sxx[:, :-1] + sex[1:, :] - sex[:-1, :]
        cly = sxy[:, 1:] - sxy[:, :-1] + sey[1:, :] - sey[:-1, :]
        scale = np.abs(sxx).max() + np.abs(sey).max()
        assert np.abs(clx).max() < 1e-14 * scale and np.abs(cly).max() < 1e-14 * scale
        assert np.all(vol > 0)
    # total volume = area enclosed by the grid's boundary loop (wake cut traversed twice)
    x, y = g.x, g.y
    px = np.concatenate([x[0, :], x[1:, -1], x[-1, -2::-1], x[-2:0:-1, 0]])
    py = np.concatenate([y[0, :], y[1:, -1], y[-1, -2::-1], y[-2:0:-1, 0]])
    area = _shoelace(px, py)
    for l in range(3):
        vol = o.metrics(l)[4]
        assert abs(vol.sum() - area) < 1e-12 * area


# ---------------------------------------------------------------- residual invariants
def test_free_stream_preservation_curvilinear():
    """Uniform flow tangent to a flat slip wall on a randomly jittered grid: F = 0 to roundoff."""
    g = make_rect_grid(12, 8, lx=2.0, ly=1.0, jitter=0.3, seed=1)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=0.0))
    o.set_state(_uniform(O.free_stream(0.8, 0.0), 8, 12))
    F, Fc, Fv = o.residual()
    assert np.abs(F).max() < 1e-12
    assert np.abs(Fv).max() < 1e-12


def test_free_stream_preservation_cgrid_plate_all_levels():
    """Zero-thickness plate C-grid at alpha = 0 (wall tangent, cut interior): F = 0 on every level."""
    g = make_cgrid(32, 8, thickness=0.0)
    o = O.Oracle(g, O.make_params(nlevels=3, mach=0.8, alpha_deg=0.0))
    w = O.free_stream(0.8, 0.0)
    for l in range(3):
        ni, nj, _ = o.dims(l)
        o.set_state(_uniform(w, nj, ni), l)
        F, _, _ = o.residual(l)
        assert np.abs(F).max() < 1e-11, l


@pytest.mark.parametrize("cell", [(10, 6), (16, 5), (2, 0), (29, 0), (3, 0), (28, 0)])
def test_discrete_conservation(cell):
    """Interior and wake-cut face fluxes telescope: sum(Omega F) depends only on boundary fluxes,
    so perturbing a cell more than two cells from any wall or far-field face leaves it unchanged."""
    ni, nj = 32, 12
    g = make_cgrid(ni, nj, jitter=0.1, seed=2)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=1.0))
    vol = o.metrics(0)[4]
    u = _perturbed(O.free_stream(0.8, 1.0), nj, ni, 0.05, 0)
    o.set_state(u)
    F, _, _ = o.residual()
    s0 = (F * vol).sum(axis=(1, 2))
    i, j = cell
    u[:, j, i] *= 1.02
    o.set_state(u)
    F, _, _ = o.residual()
    s1 = (F * vol).sum(axis=(1, 2))
    assert np.abs(s1 - s0).max() < 1e-12 * np.abs(F * vol).max()


def test_conservation_detects_wall_row():
    """Control: a cell next to the wall does move the boundary flux (the test above can fail)."""
    ni, nj = 32, 12
    g = make_cgrid(ni, nj, jitter=0.1, seed=2)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=1.0))
    vol = o.metrics(0)[4]
    u = _perturbed(O.free_stream(0.8, 1.0), nj, ni, 0.05, 0)
    o.set_state(u)
    s0 = (o.residual()[0] * vol).sum(axis=(1, 2))
    u[:, 1, 12] *= 1.02
    o.set_state(u)
    s1 = (o.residual()[0] * vol).sum(axis=(1, 2))
    assert np.abs(s1 - s0).max() > 1e-8


def test_jst_dissipation_vanishes_on_linear_w():
    """With p linear in the index the sensor is 0, eps2 = 0, and the third difference of a
    linear w vanishes: no dissipation in cells whose stencils stay inside the domain."""
    ni, nj = 16, 10
    g = make_rect_grid(ni, nj, lx=1.6, ly=1.0)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.5, alpha_deg=0.0))
    u = np.zeros((4, nj, ni))
    ii, jj = np.meshgrid(np.arange(ni), np.arange(nj))
    p = 2.0 + 0.01 * ii + 0.02 * jj
    u[0] = 1.0
    u[1] = 0.6
    u[2] = 0.1
    u[3] = p / (GAM - 1) + 0.5 * (0.6**2 + 0.1**2)
    o.set_state(u)
    _, _, Fv = o.residual()
    assert np.abs(Fv[:, 3:-3, 3:-3]).max() < 1e-12
    # control: a quadratic pressure field is dissipated
    u[3] = (2.0 + 0.01 * ii**2) / (GAM - 1) + 0.5 * (0.6**2 + 0.1**2)
    o.set_state(u)
    _, _, Fv = o.residual()
    assert np.abs(Fv[:, 3:-3, 3:-3]).max() > 1e-6


def test_sensor_formula_special_values():
    assert O.sensor(1.0, 1.0, 1.0) == 0.0
    assert abs(O.sensor(1.0, 2.0, 3.0)) < 1e-16
    assert abs(O.sensor(0.0, 1.0, 0.0) - 2.0 / 2.001) < 1e-15


# ---------------------------------------------------------------- flux-vector splitting
STATES = [np.array([1.1, 0.3, -0.2, 2.9]), np.array([0.9, 0.95, 0.05, 2.4]),
          np.array([1.0, 0.0, 0.0, 3.29])]


def _fd_jacobian(w, sx, sy, h=1e-6):
    J = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        J[:, k] = (O.conv_flux(w + e, sx, sy) - O.conv_flux(w - e, sx, sy)) / (2 * h)
    return J


@pytest.mark.parametrize("w", STATES)
@pytest.mark.parametrize("d", [0.0, 0.05, 0.5, 1.0])
def test_split_jacobians_sum_to_flux_jacobian(w, d):
    sx, sy = 0.3, 0.7
    Ap, Am = O.split_jacobians(w, sx, sy, d)
    J = _fd_jacobian(w, sx, sy)
    np.testing.assert_allclose(Ap + Am, J, atol=1e-8 * np.abs(J).max())
    ep = np.linalg.eigvals(Ap).real
    em = np.linalg.eigvals(Am).real
    assert ep.min() > -1e-12 and em.max() < 1e-12


@pytest.mark.parametrize("w", STATES)
def test_eigenvectors(w):
    nx, ny = 0.6, 0.8
    R, Ri = O.eigvecs(w, nx, ny)
    np.testing.assert_allclose(R @ Ri, np.eye(4), atol=1e-14)
    A = _fd_jacobian(w, nx, ny)
    lam = np.diag(Ri @ A @ R)
    rho = w[0]
    u, v = w[1] / rho, w[2] / rho
    p = (GAM - 1) * (w[3] - 0.5 * rho * (u * u + v * v))
    a = math.sqrt(GAM * p / rho)
    vn = u * nx + v * ny
    np.testing.assert_allclose(lam, [vn, vn, vn + a, vn - a], atol=1e-8)


def test_cutoff_parabola():
    """Eq. (cutoff): continuous with slope 1 at |lambda| = ad, ad/2 at 0, identity for d = 0."""
    a, d = 1.25, 0.3
    ad = a * d
    assert abs(O.cutoff(ad, a, d) - ad) < 1e-15
    eps = 1e-7
    slope = (O.cutoff(ad + eps, a, d) - O.cutoff(ad - eps, a, d)) / (2 * eps)
    assert abs(slope - 1.0) < 1e-6
    assert abs(O.cutoff(0.0, a, d) - ad / 2) < 1e-15
    assert O.cutoff(-0.1, a, d) == O.cutoff(0.1, a, d)
    assert O.cutoff(0.01, a, 0.0) == 0.01
    assert O.cutoff(1.0, a, d) == 1.0


def test_farfield_riemann_invariants():
    winf = O.free_stream(0.8, 2.0)
    assert np.abs(O.farfield_state(winf, winf, 0.6, -0.8) - winf).max() < 1e-13
    wi = np.array([1.05, 0.9, 0.1, 3.4])
    for nx, ny in [(0.6, -0.8), (-1.0, 0.0), (0.0, 1.0)]:
        b = O.farfield_state(wi, winf, nx, ny)

        def inv(w):
            rho, u, v = w[0], w[1] / w[0], w[2] / w[0]
            p = (GAM - 1) * (w[3] - 0.5 * rho * (u * u + v * v))
            a = math.sqrt(GAM * p / rho)
            return u * nx + v * ny, a

        vb, ab = inv(b)
        vi, ai = inv(wi)
        vf, af = inv(winf)
        assert abs((vb + 2 * ab / (GAM - 1)) - (vi + 2 * ai / (GAM - 1))) < 1e-12
        assert abs((vb - 2 * ab / (GAM - 1)) - (vf - 2 * af / (GAM - 1))) < 1e-12


# ---------------------------------------------------------------- SGS preconditioner
@pytest.mark.parametrize("shape", [(8, 3, 1), (12, 4, 2), (16, 4, 2)])
@pytest.mark.parametrize("scheme", ["AW3", "ARK3J"])
def test_sgs_sweep_equals_dense_solve(shape, scheme):
    """Eq. (sgs-precon): the forward/backward sweep equals a dense solve of (D+L) D^-1 (D+U)."""
    ni, nj, nw = shape
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.1, seed=3)
    o = O.Oracle(g, O.make_params(scheme, nlevels=1, mach=0.8, alpha_deg=1.0, d_cut=0.3))
    o.set_state(_perturbed(O.free_stream(0.8, 1.0), nj, ni, 0.05, 4))
    r = np.random.default_rng(7).standard_normal((4, nj, ni))
    z1, _ = o.precond_apply(r, 50.0)
    z2, _ = o.precond_apply(r, 50.0, dense=True)
    assert np.abs(z1 - z2).max() < 1e-11 * np.abs(z2).max()


def test_sgs_blocks_are_first_order_upwind_jacobian():
    """D + L + U applied to v equals I v + eta dt*/Omega * (linearized first-order FVS residual),
    eq. (steadylinearized) with eq. (d-l-u-matrices-W); checked through a dense solve on a tiny grid."""
    ni, nj, nw = 8, 3, 1
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=9)
    p = O.make_params("AW3", nlevels=1, mach=0.8, alpha_deg=1.0, d_cut=0.4, eta=0.7)
    o = O.Oracle(g, p)
    o.set_state(_perturbed(O.free_stream(0.8, 1.0), nj, ni, 0.03, 11))
    cfl = 30.0
    dts = o.pseudo_dt(cfl)
    axp, axm, aep, aem = o.face_blocks()
    vol = o.metrics(0)[4]
    # build W = I + eta T J_FVS directly from face blocks (outward normals, first-order upwind)
    n = ni * nj
    W = np.eye(4 * n)
    idx = lambda i, j: j * ni + i
    for j in range(nj):
        for i in range(ni):
            c = idx(i, j)
            cf = p.eta * dts[j, i] / vol[j, i]
            def add(nb, B):
                if nb is None:
                    return
                W[4 * c:4 * c + 4, 4 * nb:4 * nb + 4] += cf * B
            # east face: outward +n: A+ u_i + A- u_e
            W[4 * c:4 * c + 4, 4 * c:4 * c + 4] += cf * (axp[j, i + 1] - axm[j, i] + aep[j + 1, i] - aem[j, i])
            add(idx(i + 1, j) if i < ni - 1 else None, axm[j, i + 1])
            add(idx(i - 1, j) if i > 0 else None, -axp[j, i])
            add(idx(i, j + 1) if j < nj - 1 else None, aem[j + 1, i])
            if j > 0:
                add(idx(i, j - 1), -aep[j, i])
            elif i < nw or i >= ni - nw:
                add(idx(ni - 1 - i, 0), -aep[0, i])
    # SGS with exact splitting of W: check P = (D+L) D^-1 (D+U) against W + L D^-1 U
    Dm = np.zeros_like(W)
    for c in range(n):
        Dm[4 * c:4 * c + 4, 4 * c:4 * c + 4] = W[4 * c:4 * c + 4, 4 * c:4 * c + 4]
    Lm = np.zeros_like(W)
    Um = np.zeros_like(W)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            (Lm if b < a else Um)[4 * a:4 * a + 4, 4 * b:4 * b + 4] = W[4 * a:4 * a + 4, 4 * b:4 * b + 4]
    P = (Dm + Lm) @ np.linalg.inv(Dm) @ (Dm + Um)
    r = np.random.default_rng(3).standard_normal((4, nj, ni))
    rv = r.transpose(1, 2, 0).reshape(-1)
    z_ref = np.linalg.solve(P, dts.reshape(-1).repeat(4) * rv)
    z, _ = o.precond_apply(r, cfl)
    # the oracle's precond_apply does not include T; AW applies W^-1 (T r) in the smoother
    z2, _ = o.precond_apply(r * dts[None], cfl)
    np.testing.assert_allclose(z2.transpose(1, 2, 0).reshape(-1), z_ref, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------- stage loop
def _G_paper(a, b, c, v):
    """Section 5.3: amplification operator of the 3-stage ARK scheme (scalar form)."""
    a1, a2, a3 = a
    _, b2, b3 = b
    g1 = 1 - a1 * (c + v)
    inner = (c + b2 * v) * g1 + (1 - b2) * v
    return 1 - a3 * ((c + b3 * v) * (1 - a2 * inner) + (1 - b3) * (b2 * v * g1 + (1 - b2) * v))


@pytest.mark.parametrize("lc,lv,dts,w", [(0.7, 0.3, 1.0, 1.0), (2.0, 5.0, 0.3, 1.7),
                                         (-0.4, 1.2, 2.0, 3.0), (10.0, 0.1, 5.0, 41.0)])
def test_stage_loop_matches_paper_amplification_operator(lc, lv, dts, w):
    al, be = O.SCHEMES["ARK3J"]
    g = O.stage_scalar("ARK3J", lc, lv, dts, w)
    s = dts / w
    assert abs(g - _G_paper(al, be, lc * s, lv * s)) < 1e-14


@pytest.mark.parametrize("z", [0.1, 0.8, 1.6, 2.5])
def test_stage_loop_unsplit_polynomial(z):
    """beta = 1: the low-storage recursion is the polynomial 1 - a3 z + a3 a2 z^2 - a3 a2 a1 z^3."""
    a1, a2, a3 = O.SCHEMES["ARK3J"][0]
    g = O.stage_scalar("ERK3J", z, 0.0, 1.0, 1.0)
    assert abs(g - (1 - a3 * z + a3 * a2 * z**2 - a3 * a2 * a1 * z**3)) < 1e-14


def test_w_method_limit_large_dt():
    """AW with W = 1 + eta dt* lambda: as dt* -> inf, z -> 1/eta (section 4.3)."""
    a1, a2, a3 = O.SCHEMES["W3"][0]
    eta, lam = 0.8, 2.0
    dts = 1e12
    g = O.stage_scalar("W3", lam, 0.0, dts, 1 + eta * dts * lam)
    z = 1 / eta
    assert abs(g - (1 - a3 * z + a3 * a2 * z**2 - a3 * a2 * a1 * z**3)) < 1e-9


# ---------------------------------------------------------------- multigrid transfer
def test_restriction_conserves_integral():
    g = make_cgrid(32, 8, jitter=0.1, seed=4)
    o = O.Oracle(g, O.make_params(nlevels=3))
    rng = np.random.default_rng(5)
    for l in (2, 1):
        ni, nj, _ = o.dims(l)
        vf = rng.standard_normal((4, nj, ni))
        vc = o.restrict(l, vf)
        volf = o.metrics(l)[4]
        volc = o.metrics(l - 1)[4]
        np.testing.assert_allclose((vc * volc).sum(axis=(1, 2)), (vf * volf).sum(axis=(1, 2)), rtol=1e-12)


def test_prolongation_constants_and_linears():
    g = make_rect_grid(16, 8)
    o = O.Oracle(g, O.make_params(nlevels=2))
    dc = np.ones((4, 4, 8)) * np.array([1.0, -2.0, 0.5, 3.0])[:, None, None]
    df = o.prolong(1, dc)
    np.testing.assert_allclose(df, np.ones((4, 8, 16)) * np.array([1.0, -2.0, 0.5, 3.0])[:, None, None],
                               rtol=0, atol=1e-15)
    I, J = np.meshgrid(np.arange(8), np.arange(4))
    lin_c = 0.3 + 0.7 * (2 * I + 1) - 1.1 * (2 * J + 1)
    dc = np.stack([lin_c] * 4)
    df = o.prolong(1, dc)
    i, j = np.meshgrid(np.arange(16), np.arange(8))
    lin_f = 0.3 + 0.7 * (i + 0.5) - 1.1 * (j + 0.5)
    np.testing.assert_allclose(df[0, 1:-1, 1:-1], lin_f[1:-1, 1:-1], atol=1e-13)


# ---------------------------------------------------------------- solver behaviour
def test_fixed_point_of_the_cycle():
    """A converged discrete solution is a fixed point of the FAS cycle (section 3)."""
    g = make_cgrid(32, 8, wall_spacing=2e-3)
    o = O.Oracle(g, O.make_params("AW3", nlevels=2, mach=0.5, alpha_deg=1.0, cfl=1e4, eta=0.8))
    n0 = o.fas_cycle(0)
    for k in range(1, 400):
        nk = o.fas_cycle(k)
        if nk < 1e-11 * n0:
            break
    assert nk < 1e-11 * n0
    u0 = o.get_state()
    o.fas_cycle(1000)
    u1 = o.get_state()
    assert np.abs(u1 - u0).max() < 1e-9 * np.abs(u0).max()


def test_aw3_converges_on_transonic_c_grid():
    """Qualitative: AW3 (robust mode, d = 0.5, c* = 1e4, ramp 20) reduces the residual by
    three orders in 50 V-cycles on a 128x32 transonic Euler case."""
    g = make_cgrid(128, 32)
    o = O.Oracle(g, O.make_params("AW3", nlevels=3, mach=0.8, alpha_deg=1.25))
    nc, hist = o.solve(1e-3, 50)
    assert 0 < nc < 50 and hist[-1] <= 1e-3 * hist[0]
