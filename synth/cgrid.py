"""Structured C-grids around a closed-trailing-edge NACA 4-digit symmetric airfoil.

Geometry only (vertex coordinates).  Index convention shared by everything that
consumes these grids: vertex (i, j) is stored at ``x[j, i]`` (row j, column i),
i = 0..ni along the C (lower wake outflow -> trailing edge -> lower surface ->
leading edge -> upper surface -> trailing edge -> upper wake outflow), j = 0..nj
from the wall / wake cut outwards to the far field.  Cells are (i, j) with
i < ni, j < nj.  Cells (i, 0) with i < n_wake or i >= ni - n_wake touch the
wake cut; vertex (i, 0) coincides bitwise with vertex (ni - i, 0) for
i <= n_wake.

The j-distribution follows the paper's description of its grids (section 6):
the half of the cells nearest the wall get a boundary-layer scaling (geometric
growth from the wall spacing); the other half stretch out to the far field.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CGrid:
    ni: int
    nj: int
    n_wake: int
    x: np.ndarray  # (nj+1, ni+1) float64
    y: np.ndarray  # (nj+1, ni+1) float64
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.ni * self.nj

    def coords(self):
        """Contiguous float64 vertex arrays, index j*(ni+1)+i."""
        return (np.ascontiguousarray(self.x, dtype=np.float64).ravel(),
                np.ascontiguousarray(self.y, dtype=np.float64).ravel())


def naca_thickness(x: np.ndarray, t: float) -> np.ndarray:
    """Half thickness of the NACA 4-digit symmetric section, closed trailing edge."""
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                      + 0.2843 * x**3 - 0.1036 * x**4)


def _geometric_ratio(first: float, n: int, length: float) -> float:
    """Ratio r with first*(r^n - 1)/(r - 1) == length (r > 1), by bisection."""
    if first * n >= length:
        raise ValueError("spacing too large for the requested length")
    lo, hi = 1.0 + 1e-12, 4.0
    while first * (hi**n - 1.0) / (hi - 1.0) < length:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if first * (mid**n - 1.0) / (mid - 1.0) < length:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _line_distribution(nj: int, dw: float, delta_bl: float, length: float) -> np.ndarray:
    """Cumulative distances d_0..d_nj along one wall-normal line.

    Cells 0..nj/2-1 grow geometrically from the wall spacing ``dw`` up to the
    height ``delta_bl``; the remaining cells grow geometrically to ``length``.
    """
    nh = nj // 2
    sp = np.empty(nj)
    if dw * nh >= delta_bl:   # many wall-normal cells with a coarse wall spacing: widen the layer
        delta_bl = 2.0 * dw * nh
    r_bl = _geometric_ratio(dw, nh, delta_bl) if nh > 0 else 1.0
    sp[:nh] = dw * r_bl ** np.arange(nh)
    rest = length - sp[:nh].sum()
    if rest <= 0:
        raise ValueError("boundary-layer half exceeds the line length")
    nrest = nj - nh
    first = sp[nh - 1] if nh > 0 else dw
    # spacing of cell nh+m is first * r2^(m+1), m = 0..nrest-1
    # sum = first*r2*(r2^nrest - 1)/(r2 - 1) == rest
    lo, hi = 1.0 + 1e-12, 4.0

    def total(r):
        return first * r * (r**nrest - 1.0) / (r - 1.0)

    if total(lo) > rest:
        raise ValueError("far-field half too short for the boundary-layer spacing")
    while total(hi) < rest:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < rest:
            lo = mid
        else:
            hi = mid
    r2 = 0.5 * (lo + hi)
    sp[nh:] = first * r2 ** (np.arange(nrest) + 1.0)
    d = np.concatenate([[0.0], np.cumsum(sp)])
    d[-1] = length
    return d


def make_cgrid(ni: int, nj: int, thickness: float = 0.10, wall_spacing: float = 2e-3,
               n_wake: int | None = None, wake_length: float = 10.0, radius: float = 20.0,
               delta_bl: float = 0.05, jitter: float = 0.0, seed: int = 0) -> CGrid:
    """Build a C-grid of ni x nj cells (vertex arrays (nj+1) x (ni+1)).

    ``jitter`` > 0 moves every vertex off the wall, cut and outer boundary by a
    seeded random fraction of its local spacing (used by tests that need a
    strongly curvilinear grid).
    """
    if n_wake is None:
        n_wake = ni // 8
    nw = n_wake
    nsurf = ni - 2 * nw
    if nsurf <= 0 or nsurf % 2:
        raise ValueError("ni - 2*n_wake must be positive and even")
    nside = nsurf // 2
    x = np.zeros((nj + 1, ni + 1))
    y = np.zeros((nj + 1, ni + 1))

    # inner curve j = 0
    k = np.arange(nside + 1)
    xl = 0.5 * (1.0 + np.cos(np.pi * k / nside))          # TE -> LE
    xu = 0.5 * (1.0 - np.cos(np.pi * k / nside))          # LE -> TE
    x[0, nw:nw + nside + 1] = xl
    y[0, nw:nw + nside + 1] = -naca_thickness(xl, thickness)
    x[0, nw + nside:ni - nw + 1] = xu
    y[0, nw + nside:ni - nw + 1] = naca_thickness(xu, thickness)
    y[0, nw] = 0.0
    y[0, ni - nw] = 0.0
    x[0, nw] = 1.0
    x[0, ni - nw] = 1.0
    y[0, ni // 2] = 0.0
    if nw > 0:
        h0 = 0.5 * (1.0 - np.cos(np.pi / nside))
        if nw == 1 or h0 * nw >= wake_length:
            dwk = np.linspace(0.0, wake_length, nw + 1)
        else:
            rw = _geometric_ratio(h0, nw, wake_length)
            kk = np.arange(nw + 1)
            dwk = h0 * (rw**kk - 1.0) / (rw - 1.0)
        dwk[-1] = wake_length
        for kq in range(nw + 1):
            x[0, nw - kq] = 1.0 + dwk[kq]
            y[0, nw - kq] = 0.0
        for i in range(nw + 1):                           # coincident cut vertices
            x[0, ni - i] = x[0, i]
            y[0, ni - i] = y[0, i]

    # Line directions: straight lines leave the inner curve along a direction
    # field that rotates monotonically along i (so lines never cross): the
    # discrete outward normal on the airfoil, the analytic trailing-edge normal
    # at the trailing edge, and a lean that grows linearly downstream on the wake.
    p0 = np.stack([x[0], y[0]], axis=1)
    tang = np.zeros_like(p0)
    tang[1:-1] = p0[2:] - p0[:-2]
    tang[0] = p0[1] - p0[0]
    tang[-1] = p0[-1] - p0[-2]
    m = np.stack([-tang[:, 1], tang[:, 0]], axis=1)
    nrm = np.linalg.norm(m, axis=1, keepdims=True)
    m = m / np.where(nrm > 0, nrm, 1.0)
    m[ni // 2] = (-1.0, 0.0)                                  # leading edge
    xs = 1.0
    slope_te = 5.0 * thickness * (0.2969 / (2.0 * np.sqrt(xs)) - 0.1260 - 2 * 0.3516 * xs
                                  + 3 * 0.2843 * xs**2 - 4 * 0.1036 * xs**3)
    th_te = float(np.arctan(-slope_te))                       # aft lean of the TE normal
    lean_max = max(0.3, th_te + 0.05)
    for i in range(nw + 1):
        xi = x[0, i] - 1.0
        lean = th_te + (lean_max - th_te) * (xi / wake_length if wake_length > 0 else 0.0)
        m[i] = (np.sin(lean), -np.cos(lean))                  # lower wake / lower TE
        m[ni - i] = (np.sin(lean), np.cos(lean))              # upper wake / upper TE

    for i in range(ni + 1):
        P0 = p0[i]
        d = _line_distribution(nj, wall_spacing, delta_bl, radius)
        for j in range(1, nj + 1):
            x[j, i] = P0[0] + d[j] * m[i, 0]
            y[j, i] = P0[1] + d[j] * m[i, 1]

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        for j in range(1, nj):
            for i in range(1, ni):
                hx = min(abs(x[j, i + 1] - x[j, i]) + abs(y[j, i + 1] - y[j, i]),
                         abs(x[j, i] - x[j, i - 1]) + abs(y[j, i] - y[j, i - 1]))
                hy = min(abs(x[j + 1, i] - x[j, i]) + abs(y[j + 1, i] - y[j, i]),
                         abs(x[j, i] - x[j - 1, i]) + abs(y[j, i] - y[j - 1, i]))
                h = min(hx, hy)
                x[j, i] += jitter * h * rng.uniform(-1, 1)
                y[j, i] += jitter * h * rng.uniform(-1, 1)

    g = CGrid(ni, nj, nw, x, y, dict(thickness=thickness, wall_spacing=wall_spacing,
                                      wake_length=wake_length, radius=radius, delta_bl=delta_bl,
                                      jitter=jitter, seed=seed))
    check_cgrid(g)
    return g


def make_rect_grid(ni: int, nj: int, lx: float = 1.0, ly: float = 1.0, jitter: float = 0.0,
                   seed: int = 0) -> CGrid:
    """Cartesian ni x nj grid on [0,lx] x [0,ly] with no wake cut (n_wake = 0)."""
    xs = np.linspace(0.0, lx, ni + 1)
    ys = np.linspace(0.0, ly, nj + 1)
    x, y = np.meshgrid(xs, ys)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx, hy = lx / ni, ly / nj
        x[1:-1, 1:-1] += jitter * hx * rng.uniform(-1, 1, size=(nj - 1, ni - 1))
        y[1:-1, 1:-1] += jitter * hy * rng.uniform(-1, 1, size=(nj - 1, ni - 1))
    g = CGrid(ni, nj, 0, np.ascontiguousarray(x), np.ascontiguousarray(y),
              dict(rect=True, lx=lx, ly=ly, jitter=jitter))
    check_cgrid(g)
    return g


def check_cgrid(g: CGrid) -> None:
    """Reject folded grids: no quad corner may turn right (straight corners are
    allowed, e.g. at the leading edge of a zero-thickness plate) and every quad
    must enclose a positive area."""
    x, y = g.x, g.y
    P = [(x[:-1, :-1], y[:-1, :-1]), (x[:-1, 1:], y[:-1, 1:]),
         (x[1:, 1:], y[1:, 1:]), (x[1:, :-1], y[1:, :-1])]
    for k in range(4):
        a, b, c = P[k - 1], P[k], P[(k + 1) % 4]
        cr = (b[0] - a[0]) * (c[1] - b[1]) - (b[1] - a[1]) * (c[0] - b[0])
        if not np.all(cr >= 0.0):
            bad = np.argwhere(~(cr >= 0.0))
            raise ValueError(f"grid has inverted cells, first at (j,i)={bad[0]}")
    area2 = ((P[2][0] - P[0][0]) * (P[3][1] - P[1][1]) - (P[2][1] - P[0][1]) * (P[3][0] - P[1][0]))
    if not np.all(area2 > 0.0):
        raise ValueError("grid has cells of zero area")
    if g.n_wake > 0:
        for i in range(g.n_wake + 1):
            if x[0, i] != x[0, g.ni - i] or y[0, i] != y[0, g.ni - i]:
                raise ValueError("wake-cut vertices do not coincide")
