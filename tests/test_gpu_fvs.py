"""GPU parity of the first-order flux-vector-split residual option (the discretization that
section 4.4 linearizes for the preconditioner) with the oracle, on every level and inside the
smoother and the FAS cycle, and the wall force it implies."""
import numpy as np
import pytest

from synth.cgrid import make_cgrid
from tests.helpers import make_pair, perturbed_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("viscous", [0, 1])
@pytest.mark.parametrize("ni,nj,nw", [(128, 32, 16), (72, 20, 8)])
def test_fvs_residual_parity(viscous, ni, nj, nw):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=ni, wall_spacing=1e-3)
    o, s = make_pair(g, nlevels=2, viscous=viscous, mach=0.7, alpha_deg=1.0, re=1e5, flux="fvs", d_cut=0.3)
    for l in (1, 0):
        ni_l, nj_l, _ = o.dims(l)
        u = perturbed_state(0.7, 1.0, nj_l, ni_l, amp=0.05, seed=3)
        o.set_state(u, l); s.set_state(u, l)
        Fo, Fco, Fvo = o.residual(l)
        Fg, Fcg, Fvg = s.residual(l)
        assert rel_err(Fg, Fo) < 1e-11
        assert rel_err(Fcg, Fco) < 1e-11 and rel_err(Fvg, Fvo) < 1e-11
    o.set_state(u, 0)


def test_fvs_cycle_history_and_force():
    g = make_cgrid(128, 32)
    o, s = make_pair(g, nlevels=3, mach=0.8, alpha_deg=1.25, flux="fvs", cfl=100.0)
    ho = np.array([o.fas_cycle(k) for k in range(15)])
    hg = np.array([s.fas_cycle(k) for k in range(15)])
    assert np.all(np.abs(hg - ho) <= 1e-8 * ho)
    assert rel_err(s.get_state(), o.get_state()) < 1e-12
    from oracle import adjoint as A
    cl_o, cd_o = A.force_coefficients(*o.wall_force(), 1.25)
    cl, cd = s.force_coefficients()
    assert abs(cl - cl_o) <= 1e-10 * abs(cl_o) and abs(cd - cd_o) <= 1e-10 * abs(cd_o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["AW3", "ARK3J"])
def test_exact_preconditioner_converges_to_the_oracles_direct_solve(precision, scheme):
    """The GPU's block Gauss-Seidel corrections toward (D+L+U)^-1 approach the oracle's banded
    direct solve geometrically: with the AW blocks (I + eta dt* J) the SGS factor is close to the
    whole operator and 60 corrections reach the direct solve to 1e-9 (FP64) / FP32 accuracy; the
    ARK blocks (J alone) are far less diagonally dominant (measured contraction about 0.93 per
    correction on this grid), so they take 400."""
    g = make_cgrid(48, 12, n_wake=6, jitter=0.03, seed=5)
    o, s = make_pair(g, scheme=scheme, nlevels=1, d_cut=0.5, precision=precision)
    u = perturbed_state(0.8, 1.25, 12, 48, amp=0.05, seed=6)
    o.set_state(u); s.set_state(u)
    r = np.random.default_rng(8).standard_normal((4, 12, 48))
    ze, _ = o.precond_apply(r, 50.0, dense="exact")
    errs = []
    for k in (2, 8, 60 if scheme == "AW3" else 400):
        s.set_exact_preconditioner(k)
        errs.append(rel_err(s.precond_apply(r, 50.0), ze))
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-12
    assert errs[2] < (1e-9 if precision == "fp64" else 1e-4), errs
    s.set_exact_preconditioner(0)
    zs = s.precond_apply(r, 50.0)
    zo, _ = o.precond_apply(r, 50.0)
    assert rel_err(zs, zo) < (1e-11 if precision == "fp64" else 1e-3)


def test_exact_preconditioner_in_the_smoother():
    """AW3 with the exact preconditioner inside the stage loop: the GPU's smoothing steps follow
    the oracle's (precond exact, direct solve) to the accuracy of 200 corrections."""
    g = make_cgrid(32, 8, n_wake=4)
    from tests.helpers import pair_params
    import oracle as O
    import paper_1710_04875_gb300 as P
    po, pg = pair_params(nlevels=1, mach=0.8, alpha_deg=1.25, cfl=200.0)
    po.precond = 1
    o, s = O.Oracle(g, po), P.Solver(g, pg)
    s.set_exact_preconditioner(200)
    u = perturbed_state(0.8, 1.25, 8, 32, amp=0.02, seed=9)
    o.set_state(u); s.set_state(u)
    for _ in range(3):
        o.smooth(1, 200.0)
        s.smooth(1, 200.0)
    assert rel_err(s.get_state() - u, o.get_state() - u) < 1e-8
