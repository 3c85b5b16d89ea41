"""Oracle discrete adjoint of the steady finest-level residual (test infrastructure only).

Plain and slow: the Jacobian dF/du of the oracle's own residual (section 2, with the eddy
viscosity frozen at its current value) by central differences on groups of cells that share
no residual stencil (a greedy distance-2 colouring of the stencil graph), assembled as a
scipy sparse matrix; the adjoint system (dF/du)^T lambda = (dJ/du)^T solved directly by a
sparse LU; the shape gradient dJ/dp = dJ/dX dX/dp - lambda^T dF/dX dX/dp with the X-derivatives
by central differences over deformed grids.  The objectives J are the lift and drag
coefficients of the force the scheme's wall-face fluxes exert on the body.

Only tests/ and the bench's CPU legs import this module.  It shares nothing with the CUDA
library: its colouring, finite differences and solves are written here from the definitions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Oracle


def stencil(ni: int, nj: int, nw: int) -> list[list[int]]:
    """For every cell c = j*ni + i, the cells its residual F_c depends on: the JST cross of
    half-width 2 inside the grid (ghosts are functions of the cell next to them) and, on the
    wake cut, the mirror cells (ni-1-i, 0) (rows 0 and 1) and (ni-1-i, 1) (row 0) that the
    cut's ghost layers copy."""
    deps = []
    for j in range(nj):
        for i in range(ni):
            d = [j * ni + i]
            for a in (-2, -1, 1, 2):
                if 0 <= i + a < ni:
                    d.append(j * ni + i + a)
                if 0 <= j + a < nj:
                    d.append((j + a) * ni + i)
            if nw > 0 and (i < nw or i >= ni - nw) and j <= 1:
                m = ni - 1 - i
                d.append(m)
                if j == 0:
                    d.append(ni + m)
            deps.append(sorted(set(d)))
    return deps


def colouring(deps: list[list[int]], n: int) -> np.ndarray:
    """Greedy colouring such that no residual stencil holds two cells of one colour."""
    users = [[] for _ in range(n)]
    for c, d in enumerate(deps):
        for x in d:
            users[x].append(c)
    col = -np.ones(n, dtype=np.int64)
    for d in range(n):
        taken = set()
        for c in users[d]:
            for x in deps[c]:
                if col[x] >= 0:
                    taken.add(int(col[x]))
        k = 0
        while k in taken:
            k += 1
        col[d] = k
    return col


def _steps(u: np.ndarray, h_rel: float) -> np.ndarray:
    return h_rel * np.maximum(1.0, np.abs(u))


def force_coefficients(fx: np.ndarray, fy: np.ndarray, alpha_deg: float) -> tuple[float, float]:
    """Lift and drag coefficients (free stream rho = 1, |v| = 1, chord 1) of the body force."""
    a = np.radians(alpha_deg)
    Fx, Fy = float(np.sum(fx)), float(np.sum(fy))
    return 2.0 * (-Fx * np.sin(a) + Fy * np.cos(a)), 2.0 * (Fx * np.cos(a) + Fy * np.sin(a))


def jacobian(o: Oracle, alpha_deg: float, h_rel: float = 1e-6):
    """(J, gL, gD): the sparse residual Jacobian (4n x 4n, index k*n + c for component k of cell
    c) at the oracle's current state, and the state gradients of the lift and drag coefficients
    (4n), all by central differences over colour groups."""
    g = o.grid
    ni, nj, nw = g.ni, g.nj, g.n_wake
    n = ni * nj
    deps = stencil(ni, nj, nw)
    col = colouring(deps, n)
    u0 = o.get_state().reshape(4, n)
    hs = _steps(u0, h_rel)
    owner = {}  # (c, colour) -> the dependency of that colour
    for c, d in enumerate(deps):
        for x in d:
            owner[(c, int(col[x]))] = x
    rows, cols, vals = [], [], []
    gL = np.zeros(4 * n)
    gD = np.zeros(4 * n)
    a = np.radians(alpha_deg)
    for k in range(int(col.max()) + 1):
        sel = col == k
        for m in range(4):
            up = u0.copy(); um = u0.copy()
            up[m, sel] += hs[m, sel]
            um[m, sel] -= hs[m, sel]
            o.set_state(up.reshape(4, nj, ni)); Fp = o.residual()[0].reshape(4, n); fxp, fyp = o.wall_force()
            o.set_state(um.reshape(4, nj, ni)); Fm = o.residual()[0].reshape(4, n); fxm, fym = o.wall_force()
            for c in range(n):
                x = owner.get((c, k))
                if x is None:
                    continue
                dF = (Fp[:, c] - Fm[:, c]) / (2.0 * hs[m, x])
                for r in range(4):
                    if dF[r] != 0.0:
                        rows.append(r * n + c); cols.append(m * n + x); vals.append(dF[r])
            # wall face i depends on cells (i, 0) and (i, 1) only
            for i in range(ni):
                x = None
                for cand in (i, ni + i):
                    if col[cand] == k:
                        x = cand
                if x is None:
                    continue
                dfx = (fxp[i] - fxm[i]) / (2.0 * hs[m, x])
                dfy = (fyp[i] - fym[i]) / (2.0 * hs[m, x])
                gL[m * n + x] += 2.0 * (-dfx * np.sin(a) + dfy * np.cos(a))
                gD[m * n + x] += 2.0 * (dfx * np.cos(a) + dfy * np.sin(a))
    o.set_state(u0.reshape(4, nj, ni))
    J = sp.csr_matrix((vals, (rows, cols)), shape=(4 * n, 4 * n))
    return J, gL, gD


def adjoint(J, g: np.ndarray) -> np.ndarray:
    """lambda with J^T lambda = g (sparse direct solve)."""
    return spla.spsolve(sp.csc_matrix(J.T), g)


def shape_gradient(grid, params, state: np.ndarray, mut: np.ndarray | None, fields: np.ndarray,
                   alpha_deg: float, h_rel: float = 1e-6, h_x: float = 1e-6):
    """Adjoint shape gradients (dCL/dp, dCD/dp) at a converged state for the bump fields
    (nparam, nj+1, ni+1) of y-displacements; mut frozen at the given eddy viscosity."""
    from synth.shape import deformed

    def make(gr):
        o = Oracle(gr, params)
        o.set_state(state)
        if mut is not None:
            o.set_mut(mut)
        return o

    o = make(grid)
    J, gL, gD = jacobian(o, alpha_deg, h_rel)
    lamL, lamD = adjoint(J, gL), adjoint(J, gD)
    nparam = fields.shape[0]
    dL = np.zeros(nparam)
    dD = np.zeros(nparam)
    for k in range(nparam):
        e = np.zeros(nparam); e[k] = h_x
        op, om = make(deformed(grid, e, fields)), make(deformed(grid, -e, fields))
        dF = (op.residual()[0] - om.residual()[0]).ravel() / (2.0 * h_x)
        cLp, cDp = force_coefficients(*op.wall_force(), alpha_deg)
        cLm, cDm = force_coefficients(*om.wall_force(), alpha_deg)
        dL[k] = (cLp - cLm) / (2.0 * h_x) - lamL @ dF
        dD[k] = (cDp - cDm) / (2.0 * h_x) - lamD @ dF
        del op, om
    del o
    return dL, dD, lamL, lamD
