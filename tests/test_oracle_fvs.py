"""Pins of the oracle's first-order flux-vector-split residual and of the exact preconditioner
(the discretization that section 4.4 linearizes to build the preconditioner, eqs. steadylinearized
and form1, and the "exact" preconditioner of section 5.4's tables).

The FVS face flux is h = A+(u_bar) u_L + A-(u_bar) u_R.  Pinned by: (1) free-stream
preservation on curvilinear grids, every level; (2) discrete conservation (interior fluxes
telescope, so the volume-weighted sum of the residual is the sum of boundary fluxes); (3) the
residual is exactly the preconditioner's own block operator applied to the state: for the ARK
blocks (scale 1/Omega, no time term) F_i = [(D + L + U) u]_i in every cell whose faces all have
an interior cell or the wake-cut mirror on the other side -- two independent code paths of the
oracle (the flux loop and the block assembly with its neighbour sets) agreeing; (4) the exact
preconditioner's banded elimination solves (D + L + U) z = r, checked against numpy's dense solve
of the operator assembled column by column."""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid, make_rect_grid
from tests.helpers import perturbed_state, rel_err


def _oracle(g, scheme="ARK3J", **kw):
    p = O.make_params(scheme, nlevels=kw.pop("nlevels", 1), mach=0.7, alpha_deg=1.5, flux="fvs", **kw)
    return O.Oracle(g, p)


def _uniform(w, nj, ni):
    return np.ascontiguousarray(np.broadcast_to(w[:, None, None], (4, nj, ni)))


def test_fvs_residual_preserves_the_free_stream_on_a_jittered_grid():
    """Uniform flow tangent to a flat slip wall on a randomly jittered grid: F = 0 to roundoff."""
    g = make_rect_grid(12, 8, lx=2.0, ly=1.0, jitter=0.3, seed=1)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=0.0, flux="fvs"))
    o.set_state(_uniform(O.free_stream(0.8, 0.0), 8, 12))
    F, Fc, Fv = o.residual()
    assert np.abs(F).max() < 1e-12 and np.abs(Fv).max() < 1e-12


def test_fvs_residual_preserves_the_free_stream_on_every_level():
    """Zero-thickness plate C-grid at alpha = 0 (wall tangent, cut interior): F = 0 on every level."""
    g = make_cgrid(32, 8, thickness=0.0)
    o = O.Oracle(g, O.make_params(nlevels=3, mach=0.8, alpha_deg=0.0, flux="fvs"))
    w = O.free_stream(0.8, 0.0)
    for l in range(3):
        ni, nj, _ = o.dims(l)
        o.set_state(_uniform(w, nj, ni), l)
        F, _, _ = o.residual(l)
        assert np.abs(F).max() < 1e-11, l


@pytest.mark.parametrize("cell", [(10, 6), (16, 5), (2, 0), (29, 0), (3, 0), (28, 0)])
def test_fvs_residual_is_conservative(cell):
    """Interior and wake-cut face fluxes telescope: sum(Omega F) depends only on boundary fluxes,
    so perturbing a cell with no wall, outflow or far-field face (the FVS stencil is one cell
    wide) leaves it unchanged; a cell on the wall (control) changes it."""
    ni, nj = 32, 12
    g = make_cgrid(ni, nj, n_wake=4, jitter=0.1, seed=2)
    o = O.Oracle(g, O.make_params(nlevels=1, mach=0.8, alpha_deg=1.0, flux="fvs"))
    vol = o.metrics(0)[4]
    u = perturbed_state(0.8, 1.0, nj, ni, amp=0.05, seed=0)
    o.set_state(u)
    F, _, _ = o.residual()
    s0 = (F * vol).sum(axis=(1, 2))
    i, j = cell
    u2 = u.copy()
    u2[:, j, i] *= 1.03
    o.set_state(u2)
    F2, _, _ = o.residual()
    s1 = (F2 * vol).sum(axis=(1, 2))
    scale = np.abs(F * vol).sum()
    assert np.abs(s1 - s0).max() < 1e-13 * scale
    u3 = u.copy()
    u3[:, 0, ni // 2] *= 1.03              # a wall cell: the wall flux changes
    o.set_state(u3)
    F3, _, _ = o.residual()
    assert np.abs((F3 * vol).sum(axis=(1, 2)) - s0).max() > 1e-6 * scale


@pytest.mark.parametrize("jitter,nw", [(0.0, 4), (0.06, 6)])
def test_fvs_residual_is_the_block_operator(jitter, nw):
    ni, nj = 36, 10
    g = make_cgrid(ni, nj, n_wake=nw, jitter=jitter, seed=7)
    o = _oracle(g, d_cut=0.3)
    u = perturbed_state(0.7, 1.5, nj, ni, amp=0.03, seed=4)
    o.set_state(u)
    F = o.residual()[0]
    Au = o.block_apply(u, 1.0)
    mask = np.zeros((nj, ni), bool)
    mask[1:nj - 1, 1:ni - 1] = True
    mask[0, :nw] = True                     # wake-cut cells: the mirror is a block neighbour
    mask[0, ni - nw:] = True
    mask[0, 0] = mask[0, ni - 1] = False     # i-boundary (outflow) faces have ghosts
    err = np.abs(F - Au)[:, mask].max() / np.abs(F).max()
    assert err < 1e-12
    # and the identity fails for the JST residual (the blocks are not its Jacobian)
    pj = O.make_params("ARK3J", nlevels=1, mach=0.7, alpha_deg=1.5, d_cut=0.3)
    oj = O.Oracle(g, pj)
    oj.set_state(u)
    assert np.abs(oj.residual()[0] - Au)[:, mask].max() / np.abs(F).max() > 1e-4


@pytest.mark.parametrize("scheme", ["AW3", "ARK3J"])
def test_exact_preconditioner_solves_the_block_system(scheme):
    ni, nj, nw = 12, 4, 2
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=9)
    o = _oracle(g, scheme=scheme, d_cut=0.5)
    u = perturbed_state(0.7, 1.5, nj, ni, amp=0.03, seed=2)
    o.set_state(u)
    cfl = 50.0
    N = 4 * ni * nj
    A = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        A[:, k] = o.block_apply(e.reshape(4, nj, ni), cfl).ravel()
    r = np.random.default_rng(3).standard_normal((4, nj, ni))
    z, _ = o.precond_apply(r, cfl, dense="exact")
    assert rel_err(z.ravel(), np.linalg.solve(A, r.ravel())) < 1e-11
    assert rel_err(o.block_apply(z, cfl), r) < 1e-11
    # the SGS factorization is a different operator: it does not solve the same system
    zs, _ = o.precond_apply(r, cfl)
    assert rel_err(zs, z) > 1e-6
