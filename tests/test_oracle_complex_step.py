"""The oracle's complex-step derivative of the residual (the residual's own formulas evaluated in
complex arithmetic at u + i h v): its real part is the residual to rounding (complex division,
square root and power round differently from their real forms), and its imaginary
part / h is the directional derivative, pinned against central differences of the residual
(truncation O(eps^2)) and against linearity.  It is the exact reference for the GPU's
forward-mode linearization.  CPU only."""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid
from tests.helpers import perturbed_state, rel_err

CASES = {
    "euler": dict(mach=0.7, alpha_deg=1.5),
    "laminar": dict(viscous=1, turb=0, mach=0.5, alpha_deg=1.0, re=1e4),
    "rans": dict(viscous=1, turb=1, mach=0.6, alpha_deg=2.0, re=1e6),
    "fvs": dict(mach=0.7, alpha_deg=1.5, flux="fvs"),
}


def _setup(kind, ni=32, nj=8, nw=4, seed=5):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=seed, wall_spacing=2e-3)
    kw = dict(CASES[kind])
    p = O.make_params("AW3", nlevels=1, cfl=50.0, d_cut=0.4, **kw)
    o = O.Oracle(g, p)
    u = perturbed_state(kw["mach"], kw["alpha_deg"], nj, ni, amp=0.02, seed=seed)
    o.set_state(u)
    if kind == "rans":
        o.compute_mut()
    return o, u


@pytest.mark.parametrize("kind", list(CASES))
def test_real_part_is_the_residual(kind):
    o, u = _setup(kind)
    v = np.random.default_rng(1).standard_normal(u.shape)
    F, dF = o.residual_complex_step(v)
    assert rel_err(F, o.residual()[0]) < 1e-12


@pytest.mark.parametrize("kind", list(CASES))
def test_derivative_equals_central_differences(kind):
    o, u = _setup(kind)
    v = np.random.default_rng(2).standard_normal(u.shape) * np.abs(u)
    _, dF = o.residual_complex_step(v)
    mut = o.get_mut().copy() if kind == "rans" else None
    eps = 1e-6
    o.set_state(u + eps * v)
    if mut is not None:
        o.set_mut(mut)
    Fp = o.residual()[0]
    o.set_state(u - eps * v)
    if mut is not None:
        o.set_mut(mut)
    Fm = o.residual()[0]
    o.set_state(u)
    assert rel_err(dF, (Fp - Fm) / (2 * eps)) < 1e-7


def test_derivative_is_linear_in_the_direction():
    o, u = _setup("laminar")
    rng = np.random.default_rng(3)
    v, w = rng.standard_normal(u.shape), rng.standard_normal(u.shape)
    _, dv = o.residual_complex_step(v)
    _, dw = o.residual_complex_step(w)
    _, dvw = o.residual_complex_step(2.0 * v - 3.0 * w)
    assert rel_err(dvw, 2.0 * dv - 3.0 * dw) < 1e-13


def test_step_size_independence():
    """No subtractive cancellation: the derivative does not change with the step over many
    decades."""
    o, u = _setup("euler")
    v = np.random.default_rng(4).standard_normal(u.shape)
    _, d1 = o.residual_complex_step(v, h=1e-30)
    _, d2 = o.residual_complex_step(v, h=1e-12)
    assert rel_err(d1, d2) < 1e-14
