"""Discrete Fourier (local Fourier) analysis of the preconditioned smoothers, section 5.

TEST INFRASTRUCTURE ONLY (part of the oracle): imported by tests and by the script that writes
the stored LFA tables, never by the product package.

The linearized Euler equations of section 5 (eq. linearized-euler) on a periodic Cartesian grid
of nx x ny cells of width dx x dy = AR dx, the JST symbols H_c and H_v of section 5.1 with the
linearized pressure switch, the SGS preconditioner of section 5.2 built from the flux-vector-split
Jacobians with the cutoff (eq. cutoff), or the exact preconditioner D + L + U, or none (the
explicit schemes), and the low-storage stage loop of sections 4.1-4.2 written for a linear
operator.  Every quantity is a 4 x 4 matrix per pair of phase angles theta = 2 pi k / n
(k = -n/2+1 .. n/2, section 5.3); rho(M) is the largest spectral radius over the angle pairs, the
smoothing factor (eq. smoothfactor) the largest over the high-frequency pairs.  All angle pairs
are evaluated at once (batched 4 x 4 algebra).

Readings (each listed with its reason in the design notes):
 * pseudo and physical time steps in the CFL form dt* = c* / lam, dt = c / lam with
   lam = (|u|+a)/dx + (|v|+a)/dy; the unsteady symbol adds 3/(2 dt) I to H_c (section 5.1);
 * the zero angle pair is part of rho(M) when the problem is unsteady (it carries the 3/(2 dt)
   shift; the tables' AR = 1 entries of rho(M) for the explicit schemes are exactly the
   stability function at -1.5 c*/c); the steady analysis leaves it out (its factor is 1);
 * the pressure switch of section 5.1 with the pressure factors of numerator and denominator
   cancelling (the denominator's -2|v|^2 read as -|v|^2/2): s(theta) = tan^2(theta/2), capped
   at 0.25, eps2 = r s, eps4 = max(0, r/32 - 2 eps2); sensor="off" drops the switch;
 * high frequencies: hf="either" takes a pair when |theta_x| >= pi/2 or |theta_y| >= pi/2,
   hf="both" when both are;
 * the ARK diagonal of section 5.2 is 3/(2 dt) I + (1/Omega)(...) by default (the form the
   solver uses); ark_identity=True adds the I that the analysis section writes into D^s;
 * the AW step applies W^-1 to dt* H u, W = (1 + eta dt* 3/(2 dt)) I + eta dt* (1/Omega)(...).
The matrices are evaluated at the constant state (the simplification stated in section 5.2).
"""
from __future__ import annotations

import numpy as np

from . import SCHEMES, free_stream, split_jacobians

GAM = 1.4


def _prims(w):
    rho, u, v = w[0], w[1] / w[0], w[2] / w[0]
    p = (GAM - 1) * (w[3] - 0.5 * rho * (u * u + v * v))
    return u, v, np.sqrt(GAM * p / rho)


class Model:
    """The symbols of one linearization point w, cell widths dx x dy and cutoff d."""

    def __init__(self, w, dx, dy, d, sensor="symbol", ark_identity=False):
        self.w = np.asarray(w, float)
        self.dx, self.dy, self.d = dx, dy, d
        self.sensor, self.ark_identity = sensor, ark_identity
        self.Ap, self.Am = split_jacobians(self.w, 1.0, 0.0, d)
        self.Bp, self.Bm = split_jacobians(self.w, 0.0, 1.0, d)
        self.A, self.B = self.Ap + self.Am, self.Bp + self.Bm
        u, v, a = _prims(self.w)
        self.rx, self.ry = abs(u) + a, abs(v) + a
        self.lam = self.rx / dx + self.ry / dy
        M = np.eye(4)
        M[3, 0] = -(GAM - 1) * (u * u + v * v) / 2
        M[3, 3] = GAM
        self.M = M

    def coefficients(self, t, r):
        """(eps2, eps4) arrays of faces whose neighbours differ by the phase angles t, radius r."""
        t = np.asarray(t, float)
        if self.sensor == "off":
            return np.zeros_like(t), np.full_like(t, r / 32.0)
        c = np.cos(t)
        num, den = np.abs(2 * c - 2), np.abs(2 * c + 2)
        if self.sensor == "point":
            # the printed quotient evaluated at the linearization point: pressure factors
            # (gamma-1)(rho E - |v|^2/2 rho) over (gamma-1)(rho E - 2 |v|^2 rho), plus 0.001
            rho, q2 = self.w[0], (self.w[1] ** 2 + self.w[2] ** 2) / self.w[0] ** 2
            fn = (GAM - 1) * abs(self.w[3] - 0.5 * q2 * rho)
            fd = (GAM - 1) * abs(self.w[3] - 2.0 * q2 * rho)
            num, den = num * fn, den * fd + 0.001
        s = np.where(den * 0.25 >= num, num / np.where(den > 0, den, 1.0), 0.25)
        e2 = r * s
        return e2, np.maximum(0.0, r / 32.0 - 2.0 * e2)

    def symbols(self, tx, ty, a_t):
        """H_c and H_v (N x 4 x 4, complex) at the angle arrays tx, ty:
        H_c = i/Omega (A sin(tx) dy + B sin(ty) dx) + a_t I,
        H_v = M [eps2 (2 - 2 cos) + eps4 (2 - 2 cos)^2] summed over the two directions / Omega."""
        dx, dy = self.dx, self.dy
        om = dx * dy
        sx, sy = np.sin(tx)[:, None, None], np.sin(ty)[:, None, None]
        Hc = 1j / om * (self.A * sx * dy + self.B * sy * dx) + a_t * np.eye(4)
        e2x, e4x = self.coefficients(tx, self.rx)
        e2y, e4y = self.coefficients(ty, self.ry)
        kx, ky = 2 - 2 * np.cos(tx), 2 - 2 * np.cos(ty)
        h = ((e2x * kx + e4x * kx * kx) * dy + (e2y * ky + e4y * ky * ky) * dx) / om
        Hv = self.M[None] * h[:, None, None]
        return Hc.astype(complex), Hv.astype(complex)

    def precond_inverse(self, tx, ty, dts, eta, a_t, aw, kind):
        """P^-1 (N x 4 x 4) of section 5.2: SGS (D+L) D^-1 (D+U), the exact D+L+U, or the identity
        (kind "none", the explicit schemes)."""
        n = len(tx)
        if kind == "none":
            return np.broadcast_to(np.eye(4, dtype=complex), (n, 4, 4))
        dx, dy = self.dx, self.dy
        om = dx * dy
        s = (eta * dts if aw else 1.0) / om
        if aw:
            sig = 1 + eta * dts * a_t
        else:
            sig = a_t + (1.0 if self.ark_identity else 0.0)
        I = np.eye(4)
        D = sig * I + s * (dy * (self.Ap - self.Am) + dx * (self.Bp - self.Bm))
        ex_m, ey_m = np.exp(-1j * tx)[:, None, None], np.exp(-1j * ty)[:, None, None]
        L = -s * (dy * self.Ap * ex_m + dx * self.Bp * ey_m)
        U = s * (dy * self.Am / ex_m + dx * self.Bm / ey_m)
        if kind == "exact":
            return np.linalg.inv(D + L + U)
        Dinv = np.linalg.inv(D)
        return np.linalg.inv((D + L) @ Dinv @ (D + U))


def amplification(model, scheme, tx, ty, cstar, c_phys=None, eta=0.8, precond="sgs"):
    """The amplification matrices (N x 4 x 4) of one smoothing step of `scheme` (Table "RK
    smoothers") at the angle arrays tx, ty: the low-storage recursion
    u_i = u_0 - alpha_i dt* P^-1 (H_c u_(i-1) + f_(i-1)),
    f_i = beta_(i+1) H_v u_i + (1 - beta_(i+1)) f_(i-1), f_0 = H_v u_0,
    written for the matrices X_i (u_i = X_i u_0) and Y_i (P^-1 f_i = Y_i u_0)."""
    tx = np.atleast_1d(np.asarray(tx, float))
    ty = np.atleast_1d(np.asarray(ty, float))
    al, be = SCHEMES[scheme]
    aw = scheme.startswith("AW") or scheme == "W3"
    kind = precond if (aw or scheme.startswith("ARK")) else "none"
    dts = cstar / model.lam
    a_t = 0.0 if c_phys is None else 1.5 * model.lam / c_phys
    Hc, Hv = model.symbols(tx, ty, a_t)
    Pi = model.precond_inverse(tx, ty, dts, eta, a_t, aw, kind)
    hc, hv = Pi @ Hc, Pi @ Hv
    I = np.eye(4, dtype=complex)
    X = np.broadcast_to(I, hc.shape).copy()
    Yp = hv
    s = len(al)
    for i in range(s):
        X = I - dts * al[i] * (hc @ X + Yp)
        if i + 1 < s:
            b = be[i + 1]
            Yp = b * (hv @ X) + (1 - b) * Yp
    return X


def angles(nx, ny):
    """The phase-angle pairs of an nx x ny periodic grid, one of each conjugate pair
    (theta and -theta give conjugate amplification matrices, so equal spectral radii)."""
    kx = np.arange(-nx // 2 + 1, nx // 2 + 1)
    ky = np.arange(-ny // 2 + 1, ny // 2 + 1)
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    KX, KY = KX.ravel(), KY.ravel()
    # keep (kx, ky) if (-kx, -ky) is not an earlier pair of the set; -n/2 is not in the range, so
    # kx = n/2 maps to itself modulo n.
    def canon(k, n):
        return np.where(k == n // 2, k, -k)
    nkx, nky = canon(KX, nx), canon(KY, ny)
    keep = (KX > nkx) | ((KX == nkx) & (KY >= nky))
    return 2 * np.pi * KX[keep] / nx, 2 * np.pi * KY[keep] / ny


def spectral_radii(model, scheme, nx, ny, cstar, c_phys=None, eta=0.8, precond="sgs", chunk=65536):
    """(tx, ty, r): the angle pairs and the spectral radius of each amplification matrix."""
    tx, ty = angles(nx, ny)
    r = np.empty(len(tx))
    for k in range(0, len(tx), chunk):
        G = amplification(model, scheme, tx[k:k + chunk], ty[k:k + chunk], cstar, c_phys, eta, precond)
        r[k:k + chunk] = np.abs(np.linalg.eigvals(G)).max(axis=1)
    return tx, ty, r


def factors(model, scheme, nx, ny, cstar, c_phys=None, eta=0.8, precond="sgs", hf="either"):
    """(rho(M), smoothing factor) over the angle pairs of an nx x ny grid (the zero pair counted
    in rho(M) only for an unsteady problem)."""
    tx, ty, r = spectral_radii(model, scheme, nx, ny, cstar, c_phys, eta, precond)
    zero = (tx == 0) & (ty == 0)
    rho = r[~zero].max() if c_phys is None else r.max()
    hx, hy = np.abs(tx) >= np.pi / 2 - 1e-12, np.abs(ty) >= np.pi / 2 - 1e-12
    sel = (hx & hy) if hf == "both" else (hx | hy)
    return float(rho), float(r[sel].max())


def table_model(mach, alpha_deg, ar, d, nx=8, sensor="symbol", ark_identity=False):
    """The setting of section 5.4: the linearization point at (M, alpha) and an nx x (nx AR)
    grid with dy = AR dx (dx = 1/nx)."""
    w = free_stream(mach, alpha_deg)
    dx = 1.0 / nx
    return Model(w, dx, ar * dx, d, sensor, ark_identity), nx, int(round(nx * ar))


# c* values searched: 1..19 in steps of 1, then 90 values log-spaced from 20 to 1e6.
CSTAR_GRID = np.array(sorted({round(float(x), 10) for x in
                              np.concatenate([np.arange(1, 20), np.round(np.logspace(np.log10(20), 6, 90))])}))
ETA_GRID = np.round(np.arange(0.1, 1.01, 0.1), 10)


def max_stable_cstar(model, scheme, nx, ny, c_phys=200.0, eta=0.8, precond="sgs", grid=CSTAR_GRID):
    """The largest c* of the grid with rho(M) <= 1 before the first unstable one, or None if every
    c* of the grid (up to 1e6) is stable (the tables' "A")."""
    last = None
    for cs in grid:
        rho, _ = factors(model, scheme, nx, ny, cs, c_phys, eta, precond)
        if rho > 1.0 + 1e-12:
            return last
        last = float(cs)
    return None


def optimal_cstar(model, scheme, nx, ny, c_phys=200.0, eta=0.8, precond="sgs", hf="either",
                  grid=CSTAR_GRID):
    """(c*, rho(M), smoothing factor) at the stable c* of the grid with the smallest smoothing
    factor (the first such c* on ties), or None if no c* of the grid is stable."""
    best = None
    for cs in grid:
        rho, sm = factors(model, scheme, nx, ny, cs, c_phys, eta, precond, hf)
        if rho > 1.0 + 1e-12:
            continue
        if best is None or sm < best[2] - 1e-12:
            best = (float(cs), rho, sm)
    return best


def optimal_eta_cstar(model, scheme, nx, ny, c_phys=200.0, precond="sgs", hf="either",
                      etas=ETA_GRID, grid=CSTAR_GRID):
    """(eta, c*, rho(M), smoothing factor) minimizing the smoothing factor over eta and c*
    (Tables AWa0 and AWa45)."""
    best = None
    for eta in etas:
        r = optimal_cstar(model, scheme, nx, ny, c_phys, float(eta), precond, hf, grid)
        if r is not None and (best is None or r[2] < best[3] - 1e-12):
            best = (float(eta),) + r
    return best
