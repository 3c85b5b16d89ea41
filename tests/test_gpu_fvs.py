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
