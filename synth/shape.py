"""Shape parameters for sensitivity studies: Hicks-Henne bumps on the airfoil surface and an
algebraic deformation of the C-grid.

Geometry only (vertex displacements).  The bump of peak position t in (0, 1) and width w is
b(x) = sin(pi * x^e)^w with e = ln(0.5) / ln(t), so b(0) = b(1) = 0 and b(t) = 1.  Bump k moves
the wall vertices of one side (upper or lower) by p_k * b_k(x) in y.  Every grid line j leaves
its wall vertex along a straight ray (see ``cgrid.make_cgrid``); a vertex at arc-length
fraction s along its line moves by the wall displacement times (1 - s)^2, so the far field
and the wake cut stay fixed and the deformation is linear in p.
"""
from __future__ import annotations

import numpy as np

from .cgrid import CGrid


def hicks_henne(x: np.ndarray, t: float, width: float = 3.0) -> np.ndarray:
    """Bump with peak 1 at x = t, zero at both ends of [0, 1]."""
    xc = np.clip(x, 0.0, 1.0)
    e = np.log(0.5) / np.log(t)
    return np.sin(np.pi * xc ** e) ** width


def bump_layout(n_bumps: int) -> list[tuple[str, float]]:
    """Half of the bumps on the upper surface, half on the lower, peaks spread over the chord."""
    half = n_bumps // 2
    peaks = np.linspace(0.1, 0.9, max(half, 1))
    return [("upper", float(t)) for t in peaks] + [("lower", float(t)) for t in peaks][: n_bumps - half]


def line_fraction(g: CGrid) -> np.ndarray:
    """(nj+1, ni+1) arc-length fraction of each vertex along its grid line i (0 at j = 0)."""
    d = np.sqrt(np.diff(g.x, axis=0) ** 2 + np.diff(g.y, axis=0) ** 2)
    s = np.vstack([np.zeros((1, g.ni + 1)), np.cumsum(d, axis=0)])
    return s / s[-1:]


def bump_fields(g: CGrid, n_bumps: int = 16, width: float = 3.0) -> np.ndarray:
    """(n_bumps, nj+1, ni+1) y-displacement of every vertex per unit bump amplitude."""
    ni, nw = g.ni, g.n_wake
    mid = ni // 2
    x0 = g.x[0]
    decay = (1.0 - line_fraction(g)) ** 2
    out = np.zeros((n_bumps, g.nj + 1, ni + 1))
    for k, (side, t) in enumerate(bump_layout(n_bumps)):
        w = np.zeros(ni + 1)
        idx = np.arange(mid, ni - nw + 1) if side == "upper" else np.arange(nw, mid + 1)
        w[idx] = hicks_henne(x0[idx], t, width)
        w[mid] = 0.0          # leading edge and trailing edge stay put
        w[nw] = w[ni - nw] = 0.0
        out[k] = decay * w[None, :]
    return out


def deformed(g: CGrid, p: np.ndarray, fields: np.ndarray) -> CGrid:
    """Grid with vertex y moved by sum_k p_k fields[k]."""
    dy = np.tensordot(np.asarray(p, dtype=np.float64), fields, axes=1)
    return CGrid(g.ni, g.nj, g.n_wake, g.x.copy(), g.y + dy, dict(g.meta, deformed=True))
