"""Named synthetic workloads (grid sizes, flow conditions, seeds).

Cell counts are even multiples of 2^(levels-1) so that every multigrid level
is a 2x2 agglomeration.  The workload sizes quoted as 129x33 ... 1025x257 are
vertex counts; the cell counts are one less in each direction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .cgrid import CGrid, make_cgrid


@dataclass
class FlowCase:
    name: str
    ni: int
    nj: int
    thickness: float
    wall_spacing: float
    mach: float
    alpha_deg: float
    reynolds: float = 0.0          # 0 => Euler
    levels: int = 3
    extra: dict = field(default_factory=dict)
    n_wake: int | None = None      # None => ni // 8

    def grid(self) -> CGrid:
        return make_cgrid(self.ni, self.nj, thickness=self.thickness,
                          wall_spacing=self.wall_spacing, n_wake=self.n_wake)


def config_c1(alpha_deg: float = 1.25) -> FlowCase:
    """Steady Euler, 128x32 cells, M=0.8, 3-level V-cycle, 40 cycles."""
    return FlowCase("euler_128x32", 128, 32, 0.10, 2e-3, 0.8, alpha_deg, 0.0, 3,
                    dict(cycles=40))


def config_c2() -> FlowCase:
    """Steady thin-layer RANS, 256x64 cells, wall spacing 1e-5, M=0.5, Re=1e7, 4 levels."""
    return FlowCase("rans_256x64", 256, 64, 0.10, 1e-5, 0.5, 0.0, 1e7, 4,
                    dict(drop=1e-6))


def config_c3() -> FlowCase:
    """Unsteady pitching RANS, 512x128 cells, M=0.8, Re=1e6, k=0.2, 64 steps/period."""
    k = 0.2
    omega = 2.0 * k
    period = 2.0 * np.pi / omega
    return FlowCase("pitch_512x128", 512, 128, 0.10, 1e-5, 0.8, 0.0, 1e6, 4,
                    dict(amplitude_deg=2.0, omega=omega, steps_per_period=64,
                         dt=period / 64, drop=1e-11))


def config_c4_cases(n: int = 64, seed: int = 1710) -> list[FlowCase]:
    """Batched steady Euler cases of uneven size drawn from a seeded generator.

    Up to 4 multigrid levels, fewer where the coarsest grid would have fewer than 8 cells
    across the j direction; the wake-cut length is a multiple of 8 cells so that every level
    agglomerates it exactly."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        ni = 32 * int(rng.integers(4, 17))
        nj = ni // 4
        mach = float(rng.uniform(0.5, 0.85))
        alpha = float(rng.uniform(-2.0, 4.0))
        t = float(rng.uniform(0.08, 0.12))
        levels = 1
        while levels < 4 and nj // (2 ** levels) >= 8:
            levels += 1
        n_wake = 8 * max(1, round(ni / 64))
        out.append(FlowCase(f"batch{c:02d}_{ni}x{nj}", ni, nj, t, 2e-3, mach, alpha, 0.0, levels,
                            n_wake=n_wake))
    return out


def config_c5() -> FlowCase:
    """Steady RANS for shape sensitivities, 1024x256 cells, M=0.75, Re=6.5e6, 5 levels."""
    return FlowCase("adjoint_1024x256", 1024, 256, 0.10, 1e-5, 0.75, 0.0, 6.5e6, 5,
                    dict(n_bumps=16))
