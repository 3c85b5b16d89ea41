"""The forward-mode linearization of the residual (kernels_tangent.cu; fasw_tangent_residual and
the default Jacobian assembly of the adjoint).

Checks, each against something independent of the tangent code: (1) its value part reproduces
the residual kernels' F (the same discrete operator); (2) its tangent equals central differences
of the GPU residual kernels along the same direction (to the differences' truncation); (3) the
assembled Jacobian times a vector equals the matrix-free tangent (colouring and extraction), and
the dot-product identity <w, J v> = <J^T w, v> holds between the matrix-free tangent and the
assembled transpose; (4) the assembled Jacobian agrees with the coloured central-difference
assembly of the library and with the oracle's sparse Jacobian (built by its own differences of
the C++ residual)."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from synth.cgrid import make_cgrid
from tests.helpers import make_pair, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "euler": dict(viscous=0, turb=0, mach=0.7, alpha_deg=1.5),
    "laminar": dict(viscous=1, turb=0, mach=0.5, alpha_deg=1.0, re=1e4),
    "fvs": dict(viscous=0, turb=0, mach=0.7, alpha_deg=1.5, flux="fvs"),
}


def _setup(kind, ni=48, nj=12, nw=6, seed=3):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=seed, wall_spacing=2e-3)
    o, s = make_pair(g, nlevels=1, d_cut=0.4, **CASES[kind])
    kw = CASES[kind]
    u = perturbed_state(kw["mach"], kw["alpha_deg"], nj, ni, amp=0.02, seed=seed)
    o.set_state(u); s.set_state(u)
    return g, o, s, u


@pytest.mark.parametrize("kind", list(CASES))
def test_value_part_is_the_residual(kind):
    g, o, s, u = _setup(kind)
    v = np.random.default_rng(1).standard_normal(u.shape)
    dF, F = s.tangent_residual(v, with_value=True)
    Fk, _, _ = s.residual()
    assert rel_err(F, Fk) < 1e-13
    assert rel_err(F, o.residual()[0]) < 1e-11


@pytest.mark.parametrize("kind", list(CASES))
def test_tangent_equals_differences_of_the_residual_kernels(kind):
    g, o, s, u = _setup(kind)
    v = np.random.default_rng(2).standard_normal(u.shape) * np.abs(u)
    dF = s.tangent_residual(v)
    eps = 1e-6
    s.set_state(np.ascontiguousarray(u + eps * v)); Fp = s.residual()[0]
    s.set_state(np.ascontiguousarray(u - eps * v)); Fm = s.residual()[0]
    s.set_state(u)
    fd = (Fp - Fm) / (2 * eps)
    assert rel_err(dF, fd) < 1e-6


@pytest.mark.parametrize("kind", list(CASES))
def test_assembled_jacobian_is_the_tangent(kind):
    g, o, s, u = _setup(kind)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(u.shape)
    w = rng.standard_normal(u.shape)
    s.adjoint_jacobian(1e-6)                      # forward-mode assembly (the default)
    Jv = s.adjoint_apply(v)
    dF = s.tangent_residual(v)
    assert rel_err(Jv, dF) < 1e-12
    JTw = s.adjoint_apply(w, transpose=True)
    lhs, rhs = float(np.sum(w * dF)), float(np.sum(JTw * v))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(w * dF).sum() + np.abs(JTw * v).sum())
    # against the coloured central-difference assembly of the same residual kernels
    s.adjoint_set_jacobian("differences")
    s.adjoint_jacobian(1e-6)
    Jv_fd = s.adjoint_apply(v)
    assert rel_err(Jv_fd, Jv) < 1e-6
    # and the objective gradients
    s.adjoint_set_jacobian("tangent")
    s.adjoint_jacobian(1e-6)
    g_t = s.adjoint_objective_gradient(1)
    s.adjoint_set_jacobian("differences")
    s.adjoint_jacobian(1e-6)
    g_fd = s.adjoint_objective_gradient(1)
    assert rel_err(g_t, g_fd) < 1e-6


@pytest.mark.parametrize("kind", ["euler", "laminar"])
def test_tangent_against_the_oracles_jacobian(kind):
    g, o, s, u = _setup(kind, ni=32, nj=8, nw=4, seed=5)
    J, gL, gD = OA.jacobian(o, CASES[kind]["alpha_deg"], 1e-6)
    v = np.random.default_rng(6).standard_normal(u.shape)
    dF = s.tangent_residual(v)
    assert rel_err(dF.ravel(), J @ v.ravel()) < 1e-6
    s.adjoint_jacobian(1e-6)
    assert rel_err(s.adjoint_objective_gradient(1).ravel(), gD) < 1e-6
