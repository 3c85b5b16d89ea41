"""Parity of the CUDA library (through its C ABI) with the FP64 oracle on identical seeded
inputs.  Tolerances follow the stated targets: the residual after one cycle to 1e-11
relative and convergence histories to 1e-8 relative (FP64 path)."""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid, make_rect_grid
from tests.helpers import make_pair, pair_params, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

# grids spanning several residual tiles (32 x 4 cells) with ragged tails
GRIDS = [(128, 32, 16), (40, 12, 4), (72, 20, 8), (8, 4, 1)]


@pytest.mark.parametrize("ni,nj,nw", GRIDS)
@pytest.mark.parametrize("finest", [True, False])
def test_residual_parity_euler(ni, nj, nw, finest):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=ni)
    nlev = 2 if (ni % 2 == 0 and nj % 2 == 0 and nw % 2 == 0 and ni >= 16) else 1
    o, s = make_pair(g, nlevels=nlev, mach=0.8, alpha_deg=1.25)
    l = nlev - 1 if finest else 0
    ni_l, nj_l, _ = o.dims(l)
    u = perturbed_state(0.8, 1.25, nj_l, ni_l, amp=0.05, seed=1)
    forcing = 0.1 * np.random.default_rng(2).standard_normal((4, nj_l, ni_l))
    o.set_state(u, l); s.set_state(u, l)
    if not finest:
        o.set_forcing(forcing, l); s.set_forcing(forcing, l)
    Fo, Fco, Fvo = o.residual(l)
    Fg, Fcg, Fvg, ng = s.residual(l, want_norm=True)
    assert rel_err(Fg, Fo) < 1e-11
    assert rel_err(Fcg, Fco) < 1e-11
    assert rel_err(Fvg, Fvo) < 1e-11
    assert abs(ng - np.sqrt(np.mean(Fo[0] ** 2))) < 1e-11 * abs(ng)


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
@pytest.mark.parametrize("ni,nj,nw", [(128, 32, 16), (72, 20, 8)])
def test_residual_parity_every_tile_height(rows, ni, nj, nw):
    """The residual kernel with each tile height the autotuner may pick (tiles of 31 x rows
    cells, ragged in both directions here): the same F as the oracle."""
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=ni, wall_spacing=1e-3)
    o, s = make_pair(g, nlevels=1, viscous=1, mach=0.7, alpha_deg=1.0, re=1e5)
    s.set_residual_tile(rows)
    u = perturbed_state(0.7, 1.0, nj, ni, amp=0.05, seed=4)
    o.set_state(u); s.set_state(u)
    Fo, _, _ = o.residual()
    Fg, _, _, ng = s.residual(want_norm=True)
    assert rel_err(Fg, Fo) < 1e-11
    assert abs(ng - np.sqrt(np.mean(Fo[0] ** 2))) < 1e-11 * abs(ng)


@pytest.mark.parametrize("sensor", [0, 1])
def test_residual_parity_thin_layer_with_eddy_viscosity(sensor):
    ni, nj, nw = 64, 16, 8
    g = make_cgrid(ni, nj, n_wake=nw, wall_spacing=1e-4)
    o, s = make_pair(g, nlevels=1, viscous=1, turb=1, sensor=sensor, mach=0.5, alpha_deg=1.0, re=1e5)
    u = perturbed_state(0.5, 1.0, nj, ni, amp=0.05, seed=3)
    o.set_state(u); s.set_state(u)
    mut = 1e-4 * np.random.default_rng(4).random((nj, ni))
    o.set_mut(mut)
    # the library computes mu_t itself; compare Baldwin-Lomax first, then feed it to the oracle
    mg = s.get_mut()
    mo = o.compute_mut()
    assert rel_err(mg, mo) < 1e-10
    Fo, _, _ = o.residual()
    Fg, _, _ = s.residual()
    assert rel_err(Fg, Fo) < 1e-11


@pytest.mark.parametrize("h", [1.3e-3, 6e-5])
def test_baldwin_lomax_on_closed_form_states(h):
    """The library's Baldwin-Lomax on the linear-shear plate states whose eddy viscosity has a
    closed form (both branches of F_wake, density varying through the layer): element by
    element against the oracle, and on the plate lines against the closed form itself."""
    from tests.test_oracle_baldwin_lomax import _plate_grid, _state, _wall_line_closed_form
    ni, nj, nw = 64, 32, 8
    g = _plate_grid(ni, nj, nw, h)
    a, re = 100.0, 1e6
    yc = np.abs(0.25 * (g.y[:-1, :-1] + g.y[:-1, 1:] + g.y[1:, 1:] + g.y[1:, :-1]))
    rho_of = lambda y: 0.7 + 0.3 * y / (y + 4.0 * h)
    u = _state(rho_of(yc), a * yc, np.zeros((nj, ni)), np.full((nj, ni), 100.0))
    o, s = make_pair(g, nlevels=1, viscous=1, turb=1, mach=0.5, re=re)
    o.set_state(u); s.set_state(u)
    mg = s.get_mut()
    assert rel_err(mg, o.compute_mut()) < 1e-12
    expect, _, _ = _wall_line_closed_form(a, h, rho_of((np.arange(nj) + 0.5) * h), 1.0 / re, nj)
    for i in [i for i in range(nw, ni - nw) if i not in (ni // 2 - 1, ni // 2)]:
        assert np.allclose(mg[:, i], expect, rtol=1e-11, atol=0.0), i
    s.close()


@pytest.mark.parametrize("cfl", [3.0, 1e4])
def test_pseudo_dt_and_face_blocks(cfl):
    ni, nj, nw = 72, 20, 8
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=7)
    o, s = make_pair(g, nlevels=1, d_cut=0.3)
    u = perturbed_state(0.8, 1.25, nj, ni, amp=0.05, seed=5)
    o.set_state(u); s.set_state(u)
    assert rel_err(s.pseudo_dt(cfl), o.pseudo_dt(cfl)) < 1e-13
    bo = o.face_blocks()
    bg = s.face_blocks()
    for a, b in zip(bg, bo):
        assert rel_err(a, b) < 1e-12


@pytest.mark.parametrize("scheme", ["AW3", "ARK3J"])
@pytest.mark.parametrize("ni,nj,nw", [(128, 32, 16), (40, 12, 4), (8, 4, 1)])
def test_preconditioner_apply_parity(scheme, ni, nj, nw):
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=11)
    o, s = make_pair(g, scheme=scheme, nlevels=1, d_cut=0.5)
    u = perturbed_state(0.8, 1.25, nj, ni, amp=0.05, seed=6)
    o.set_state(u); s.set_state(u)
    r = np.random.default_rng(8).standard_normal((4, nj, ni))
    zo, _ = o.precond_apply(r, 50.0)
    zg = s.precond_apply(r, 50.0)
    assert rel_err(zg, zo) < 1e-11


@pytest.mark.parametrize("scheme", ["AW3", "ARK3J", "AW5J", "AW51", "AW52", "ARK5J", "ARK51", "ARK52"])
def test_smoothing_step_parity(scheme):
    ni, nj, nw = 64, 16, 8
    g = make_cgrid(ni, nj, n_wake=nw)
    cfl = 1e4 if scheme.startswith("AW") else 1.0
    o, s = make_pair(g, scheme=scheme, nlevels=1, mach=0.8, alpha_deg=1.25)
    u = perturbed_state(0.8, 1.25, nj, ni, amp=0.02, seed=9)
    o.set_state(u); s.set_state(u)
    for _ in range(3):
        o.smooth(1, cfl)
        s.smooth(1, cfl)
    uo, ug = o.get_state(), s.get_state()
    assert rel_err(ug - u, uo - u) < 1e-10


@pytest.mark.parametrize("gamma", [1, 2])
def test_one_cycle_residual_parity(gamma):
    """Spec target: the residual after one FAS cycle matches to 1e-11 relative."""
    g = make_cgrid(128, 32)
    o, s = make_pair(g, nlevels=3, gamma_cycle=gamma, mach=0.8, alpha_deg=1.25)
    no = o.fas_cycle(0)
    ng = s.fas_cycle(0)
    assert abs(ng - no) <= 1e-12 * abs(no)
    Fo, _, _ = o.residual()
    Fg, _, _ = s.residual()
    assert rel_err(Fg, Fo) < 1e-11


def test_convergence_history_parity_c1():
    """Spec target: 40-cycle history on the 128x32 Euler case matches to 1e-8 relative
    (while above 1e-12 of the initial residual)."""
    g = make_cgrid(128, 32)
    o, s = make_pair(g, nlevels=3, mach=0.8, alpha_deg=1.25)
    ho = np.array([o.fas_cycle(k) for k in range(40)])
    hg = np.array([s.fas_cycle(k) for k in range(40)])
    mask = ho > 1e-12 * ho[0]
    assert np.all(np.abs(hg - ho)[mask] <= 1e-8 * ho[mask])
    assert ho[-1] < 1e-2 * ho[0]


def test_rans_cycle_parity_full_size():
    """The 256x64 thin-layer RANS workload (4 levels, Baldwin-Lomax): three cycles."""
    g = make_cgrid(256, 64, wall_spacing=1e-5)
    o, s = make_pair(g, nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=0.5, alpha_deg=0.0, re=1e7, cfl=100.0)
    for k in range(3):
        no = o.fas_cycle(k)
        ng = s.fas_cycle(k)
        assert abs(ng - no) <= 1e-12 * abs(no), k
    Fo, _, _ = o.residual()
    Fg, _, _ = s.residual()
    assert rel_err(Fg, Fo) < 1e-11


@pytest.mark.parametrize("precision,tol_norm,tol_f", [("fp64", 1e-12, 1e-11), ("mixed", 1e-3, 1e-2)])
def test_pitching_grid_cycle_parity_full_size(precision, tol_norm, tol_f):
    """The 512x128 C-grid of the pitching case (thin-layer RANS, Baldwin-Lomax, M 0.8, Re 1e6,
    4-level W-cycles) in the launch configuration the benchmark times: two cycles from the free
    stream against the FP64 oracle.  The mixed form differs from FP64 only through its FP32
    preconditioner, so its residual follows the oracle's to FP32 accuracy."""
    from synth.cases import config_c3
    c = config_c3()
    g = c.grid()
    po, _ = pair_params(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=c.mach, alpha_deg=0.0, re=c.reynolds,
                        cfl=100.0)
    _, pg = pair_params(nlevels=4, gamma_cycle=2, viscous=1, turb=1, mach=c.mach, alpha_deg=0.0, re=c.reynolds,
                        cfl=100.0, precision=precision)
    import paper_1710_04875_gb300 as P
    o, s = O.Oracle(g, po), P.Solver(g, pg)
    for k in range(2):
        no = o.fas_cycle(k)
        ng = s.fas_cycle(k)
        assert abs(ng - no) <= tol_norm * abs(no), k
    Fo, _, _ = o.residual()
    Fg, _, _ = s.residual()
    assert rel_err(Fg, Fo) < tol_f


@pytest.mark.parametrize("precision,tol_norm,tol_f", [("fp64", 1e-12, 1e-11), ("mixed", 1e-3, 1e-2)])
def test_largest_grid_cycle_parity(precision, tol_norm, tol_f):
    """The 1024x256 C-grid of the sensitivity case (thin-layer RANS, Baldwin-Lomax, M 0.75,
    Re 6.5e6, 5-level W-cycles): two cycles from the free stream against the FP64 oracle."""
    g = make_cgrid(1024, 256, n_wake=128, wall_spacing=1e-5)
    kw = dict(nlevels=5, gamma_cycle=2, viscous=1, turb=1, mach=0.75, alpha_deg=0.0, re=6.5e6, cfl=100.0)
    po, _ = pair_params(**kw)
    _, pg = pair_params(precision=precision, **kw)
    import paper_1710_04875_gb300 as P
    o, s = O.Oracle(g, po), P.Solver(g, pg)
    for k in range(2):
        no = o.fas_cycle(k)
        ng = s.fas_cycle(k)
        assert abs(ng - no) <= tol_norm * abs(no), k
    Fo, _, _ = o.residual()
    Fg, _, _ = s.residual()
    assert rel_err(Fg, Fo) < tol_f


@pytest.mark.parametrize("sweep", ["auto", "staged", "cta"])
def test_mixed_precision_reaches_the_fp64_fixed_point(sweep):
    """FP32 preconditioner only changes the iteration, not the converged answer (every FP32
    sweep kernel)."""
    g = make_cgrid(64, 16)
    import paper_1710_04875_gb300 as P
    from tests.helpers import pair_params
    _, p64 = pair_params(nlevels=2, mach=0.5, alpha_deg=1.0)
    _, p32 = pair_params(nlevels=2, mach=0.5, alpha_deg=1.0, precision="mixed")
    a, b = P.Solver(g, p64), P.Solver(g, p32)
    b.set_sweep(sweep)
    ca, na, ha = a.solve(1e-10, 400)
    cb, nb, hb = b.solve(1e-10, 400)
    assert ca == 0 and cb == 0
    ua, ub = a.get_state(), b.get_state()
    assert rel_err(ub, ua) < 1e-8


@pytest.mark.parametrize("sweep", ["staged", "cta"])
def test_mixed_ark_stage_update_tracks_fp64(sweep):
    """ARK stage updates (u0 - alpha dt* z) through the FP32 sweeps: the cycle history follows
    the FP64 one to FP32 accuracy."""
    g = make_cgrid(64, 16)
    import paper_1710_04875_gb300 as P
    from tests.helpers import pair_params
    kw = dict(scheme="ARK3J", nlevels=2, mach=0.5, alpha_deg=1.0, cfl=2.0, cfl_ramp=2.0)
    _, p64 = pair_params(**kw)
    _, p32 = pair_params(precision="mixed", **kw)
    a, b = P.Solver(g, p64), P.Solver(g, p32)
    b.set_sweep(sweep)
    ha = np.array([a.fas_cycle(k) for k in range(15)])
    hb = np.array([b.fas_cycle(k) for k in range(15)])
    assert np.all(np.abs(hb - ha) <= 1e-4 * ha)


def test_graph_replayed_cycles_equal_eager_cycles():
    """Cycles captured into CUDA graphs (non-default stream) give the same history as eager launches."""
    import torch
    import paper_1710_04875_gb300 as P
    from tests.helpers import pair_params
    g = make_cgrid(64, 16)
    _, p = pair_params(nlevels=2, mach=0.8, alpha_deg=1.25)
    st = torch.cuda.Stream()
    a = P.Solver(g, p, stream=st.cuda_stream)
    b = P.Solver(g, p, stream=st.cuda_stream)
    b.use_graphs(False)
    ha = [a.fas_cycle(k) for k in range(6)]
    hb = [b.fas_cycle(k) for k in range(6)]
    assert ha == hb
    assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("kind", ["reference", "cta", "strips", "strips16", "strips4", "warp", "warp8"])
@pytest.mark.parametrize("scheme", ["AW3", "ARK3J"])
@pytest.mark.parametrize("ni,nj,nw", [(128, 32, 16), (72, 20, 8), (40, 12, 4), (256, 64, 32), (16, 6, 2),
                                      (64, 100, 8), (48, 33, 4)])
def test_sweep_kinds_match_the_oracle(kind, scheme, ni, nj, nw):
    """Every sweep kernel (one thread per cell, one CTA with transfer blocks, pipelined strips
    with a partial last strip) applies the same (D+L) D^-1 (D+U) inverse."""
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=ni + nj, wall_spacing=2e-3 if nj < 64 else 1e-4)
    o, s = make_pair(g, scheme=scheme, nlevels=1, d_cut=0.5)
    s.set_sweep(kind)
    u = perturbed_state(0.8, 1.25, nj, ni, amp=0.05, seed=6)
    o.set_state(u); s.set_state(u)
    r = np.random.default_rng(8).standard_normal((4, nj, ni))
    zo, _ = o.precond_apply(r, 50.0)
    zg = s.precond_apply(r, 50.0)
    assert rel_err(zg, zo) < 1e-11


@pytest.mark.parametrize("kind", ["staged", "staged4", "staged8", "cta", "strips", "warp", "warp8"])
@pytest.mark.parametrize("ni,nj,nw", [(128, 32, 16), (72, 20, 8), (16, 6, 2), (256, 64, 32), (128, 128, 16),
                                      (256, 256, 32), (192, 200, 24)])
def test_mixed_sweep_is_the_fp32_preconditioner(kind, ni, nj, nw):
    """Mixed precision: every FP32 sweep kernel applies the oracle's operator to FP32 accuracy,
    including partial 8-row groups (nj = 20, 6, 200) and the 128- and 256-row staged variants
    (one CTA of up to 1024 threads)."""
    g = make_cgrid(ni, nj, n_wake=nw, jitter=0.03, seed=ni + nj, wall_spacing=2e-3 if nj < 64 else 1e-4)
    o, s = make_pair(g, nlevels=1, d_cut=0.5, precision="mixed")
    s.set_sweep(kind)
    u = perturbed_state(0.8, 1.25, nj, ni, amp=0.05, seed=6)
    o.set_state(u); s.set_state(u)
    r = np.random.default_rng(8).standard_normal((4, nj, ni))
    zo, _ = o.precond_apply(r, 50.0)
    zg = s.precond_apply(r, 50.0)
    assert rel_err(zg, zo) < 1e-3


def test_staged_and_cta_fp32_sweeps_agree():
    """The two single-CTA FP32 sweeps differ only by FP32 rounding."""
    g = make_cgrid(256, 64, n_wake=32, jitter=0.03, seed=5, wall_spacing=1e-4)
    _, s = make_pair(g, nlevels=1, d_cut=0.5, precision="mixed")
    u = perturbed_state(0.8, 1.25, 64, 256, amp=0.05, seed=6)
    s.set_state(u)
    r = np.random.default_rng(8).standard_normal((4, 64, 256))
    s.set_sweep("staged")
    za = s.precond_apply(r, 50.0)
    s.set_sweep("cta")
    zb = s.precond_apply(r, 50.0)
    assert rel_err(za, zb) < 1e-4


@pytest.mark.parametrize("kind", ["cta", "strips", "strips16", "warp", "warp8"])
def test_cycle_history_with_fast_sweeps(kind):
    """Full FAS cycles with the transfer-block sweeps keep the 1e-8 history parity."""
    g = make_cgrid(128, 32)
    o, s = make_pair(g, nlevels=3, mach=0.8, alpha_deg=1.25)
    s.set_sweep(kind)
    ho = np.array([o.fas_cycle(k) for k in range(25)])
    hg = np.array([s.fas_cycle(k) for k in range(25)])
    mask = ho > 1e-12 * ho[0]
    assert np.all(np.abs(hg - ho)[mask] <= 1e-8 * ho[mask])
