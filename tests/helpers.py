"""Shared test helpers: matched oracle / CUDA-library solver pairs on the same seeded input."""
from __future__ import annotations

import numpy as np

import oracle as O


def pair_params(scheme="AW3", nlevels=3, gamma_cycle=1, nu1=1, viscous=0, turb=0, sensor=None,
                mach=0.8, alpha_deg=1.25, re=1e6, pr=0.75, prt=0.9, eta=0.8, d_cut=0.5, cfl=1e4,
                cfl_ramp=20.0, ramp_cycles=2, s_coarse=0.25, norm_all=0, precision="fp64", flux="jst"):
    sensor = (1 if viscous else 0) if sensor is None else sensor
    po = O.make_params(scheme, nlevels=nlevels, gamma_cycle=gamma_cycle, nu1=nu1, viscous=viscous, turb=turb,
                       sensor=sensor, mach=mach, alpha_deg=alpha_deg, re=re, pr=pr, prt=prt, eta=eta,
                       d_cut=d_cut, cfl=cfl, cfl_ramp=cfl_ramp, ramp_cycles=ramp_cycles, s_coarse=s_coarse,
                       norm_all=norm_all, flux=flux)
    import paper_1710_04875_gb300 as P
    pg = P.default_params(scheme=scheme, nlevels=nlevels, gamma_cycle=gamma_cycle, nu1=nu1, viscous=viscous,
                          turb=turb, sensor=sensor, mach=mach, alpha_deg=alpha_deg, re=re, pr=pr, prt=prt,
                          eta=eta, d_cut=d_cut, cfl=cfl, cfl_ramp=cfl_ramp, ramp_cycles=ramp_cycles,
                          s_coarse=s_coarse, norm_all=norm_all, precision=precision, flux=flux)
    return po, pg


def make_pair(grid, **kw):
    import paper_1710_04875_gb300 as P
    po, pg = pair_params(**kw)
    return O.Oracle(grid, po), P.Solver(grid, pg)


def perturbed_state(mach, alpha_deg, nj, ni, amp=0.03, seed=0):
    w = O.free_stream(mach, alpha_deg)
    rng = np.random.default_rng(seed)
    # smooth-ish perturbation: random field plus a low mode, keeps density and pressure positive
    jj, ii = np.meshgrid(np.arange(nj), np.arange(ni), indexing="ij")
    low = np.sin(2 * np.pi * ii / max(ni, 1)) * np.cos(np.pi * jj / max(nj, 1))
    u = w[:, None, None] * (1.0 + amp * rng.standard_normal((4, nj, ni)) + amp * low[None])
    return np.ascontiguousarray(u)


def rel_err(a, b):
    """max |a - b| over max |b| (per array)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
