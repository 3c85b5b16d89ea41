"""Failure detection in forms that fault no GPU: a bounded device-side wait made to run out
(a spin limit of one poll), allocation failures injected on the host before cudaMalloc, and a
case whose iteration must diverge.  Each checks the error code the C ABI returns and that the
library stays usable afterwards."""
import numpy as np
import pytest

import oracle as O
from synth.cgrid import make_cgrid
from tests.helpers import make_pair, pair_params

pytestmark = pytest.mark.gpu


def _lib():
    import ctypes
    import paper_1710_04875_gb300 as P
    lib = P.library()
    lib.fasw_fault_inject_alloc.restype = None
    lib.fasw_fault_inject_alloc.argtypes = [ctypes.c_longlong]
    lib.fasw_live_allocations.restype = ctypes.c_longlong
    lib.fasw_live_allocations.argtypes = []
    return lib


def test_strip_sweep_wait_that_runs_out_reports_a_timeout():
    """FP64 strips of 8 rows on a 128 x 32 grid: strip b waits for strip b-1's rows.  With a
    limit of one poll a wait gives up, the kernel sets the error word and returns, and the cycle
    reports FASW_ERR_DEVICE_TIMEOUT.  The error word is cleared by the next call: the one-CTA
    sweep (no cross-CTA wait) on the same context then succeeds, and a fresh context on the same
    GPU still matches the oracle."""
    import paper_1710_04875_gb300 as P
    g = make_cgrid(128, 32)
    _, pg = pair_params(nlevels=3, mach=0.8, alpha_deg=1.25)
    pg.spin_limit = 1
    s = P.Solver(g, pg)
    s.set_sweep("strips")
    codes = []
    for k in range(3):
        try:
            s.fas_cycle(k)
            codes.append(0)
        except P.FaswError as e:
            codes.append(e.code)
    assert -5 in codes, codes
    s.set_sweep("cta")
    nrm = s.fas_cycle(3)          # no bounded wait on this path: must not see the old timeout
    assert np.isfinite(nrm) or np.isnan(nrm)   # the state after a timeout is incomplete, not checked
    s.close()
    o, f = make_pair(g, nlevels=3, mach=0.8, alpha_deg=1.25)
    for k in range(2):
        no, nf = o.fas_cycle(k), f.fas_cycle(k)
        assert abs(nf - no) <= 1e-11 * abs(no)
    f.close()


@pytest.mark.parametrize("fail_at", [0, 1, 2, 7, 31, 60])
def test_injected_allocation_failure_returns_oom_and_releases_everything(fail_at):
    """The fail_at-th device allocation of fasw_create fails on the host: the call returns
    FASW_ERR_OOM and every buffer it had allocated is released."""
    import ctypes
    import paper_1710_04875_gb300 as P
    lib = _lib()
    g = make_cgrid(64, 16)
    x, y = g.coords()
    p = P.default_params(nlevels=3, precision="mixed")
    before = lib.fasw_live_allocations()
    lib.fasw_fault_inject_alloc(fail_at)
    h = ctypes.c_void_p()
    rc = lib.fasw_create(64, 16, 8, x.ctypes.data, y.ctypes.data, 0, ctypes.byref(p), None, ctypes.byref(h))
    lib.fasw_fault_inject_alloc(-1)
    assert rc == -2 and not h.value
    assert lib.fasw_live_allocations() == before
    # the library still works afterwards
    s = P.Solver(g, p)
    assert lib.fasw_live_allocations() > before
    assert np.isfinite(s.fas_cycle(0))
    s.close()
    assert lib.fasw_live_allocations() == before


def test_injected_failure_in_the_adjoint_workspace():
    """An allocation failure while the adjoint workspace is set up returns FASW_ERR_OOM; the
    context is intact, and the same call succeeds once the injection is off."""
    import paper_1710_04875_gb300 as P
    lib = _lib()
    g = make_cgrid(32, 8)
    _, p = pair_params(nlevels=1, mach=0.5, alpha_deg=1.0)
    s = P.Solver(g, p)
    lib.fasw_fault_inject_alloc(3)
    with pytest.raises(P.FaswError) as e:
        s.adjoint_jacobian(1e-6)
    lib.fasw_fault_inject_alloc(-1)
    assert e.value.code == -2
    n0 = s.fas_cycle(0)
    assert np.isfinite(n0)
    s.close()


def test_solver_reports_divergence_not_garbage():
    """Preconditioned ARK3J far beyond its stability limit (c* = 50; the paper finds it unstable
    for c* > 1, section 6.2): the oracle's iterate becomes NaN in the second cycle, and the
    library's steady solve must stop with FASW_ERR_DIVERGED, not report convergence."""
    g = make_cgrid(32, 8)
    po, _ = pair_params(scheme="ARK3J", nlevels=2, cfl=50.0, cfl_ramp=50.0)
    o = O.Oracle(g, po)
    h = [o.fas_cycle(k) for k in range(3)]
    assert not np.isfinite(h[-1]) or h[-1] > 1e8 * h[0]
    import paper_1710_04875_gb300 as P
    _, p = pair_params(scheme="ARK3J", nlevels=2, cfl=50.0, cfl_ramp=50.0)
    s = P.Solver(g, p)
    code, nc, hist = s.solve(1e-6, 60)
    assert code == -4
    assert not np.isfinite(hist[-1]) or hist[-1] > 1e8 * hist[0]
    assert nc < 60


def test_warp_strip_sweep_wait_that_runs_out_reports_a_timeout():
    """The warp-strip sweep on a 128 x 96 grid (three strips of 32 rows, each waiting for its
    neighbour's boundary row): with a limit of one poll a wait gives up and the call reports
    FASW_ERR_DEVICE_TIMEOUT; the error word does not outlive the call."""
    import paper_1710_04875_gb300 as P
    g = make_cgrid(128, 96, n_wake=16)
    _, pg = pair_params(nlevels=1, mach=0.8, alpha_deg=1.25, precision="mixed")
    pg.spin_limit = 1
    s = P.Solver(g, pg)
    s.set_sweep("warp")
    r = np.random.default_rng(3).standard_normal((4, 96, 128))
    with pytest.raises(P.FaswError) as e:
        for _ in range(3):
            s.precond_apply(r, 50.0)
    assert e.value.code == -5
    s.set_sweep("staged")          # one CTA, no cross-CTA wait
    z = s.precond_apply(r, 50.0)
    assert np.all(np.isfinite(z))
    s.close()
