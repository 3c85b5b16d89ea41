"""The residual entry point that allocates nothing (fasw_residual_noalloc).

It exists for callers that cannot call cudaMalloc where they need a residual (an
application that owns all device memory, or a loop that must not pay for allocation).
This file is collected last so that, if it fails, a run that stops at the first failure
has already run every other test.  It must pass alone in a fresh process and after the
rest of the suite (the fixed scratch array keeps the previous call's contents).
"""
import ctypes

import numpy as np
import pytest

from synth.cgrid import make_cgrid
from tests.helpers import pair_params, perturbed_state

pytestmark = pytest.mark.gpu


def _noalloc_residual(lib, g, params, u_dev, torch):
    x, y = g.coords()
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    F = torch.full((4 * g.ni * g.nj,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.fasw_residual_noalloc(g.ni, g.nj, g.n_wake, xd.data_ptr(), yd.data_ptr(), u_dev.data_ptr(),
                                   F.data_ptr(), ctypes.byref(params), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, F.cpu().numpy().reshape(4, g.nj, g.ni)


@pytest.mark.parametrize("viscous", [0, 1])
def test_noalloc_residual_matches_the_context_residual_twice(viscous):
    torch = pytest.importorskip("torch")
    import paper_1710_04875_gb300 as P
    lib = P.library()
    cases = [(128, 32, 16, 1.25, 0), (72, 20, 8, -0.5, 1)]  # two calls in a row, different grids
    for ni, nj, nw, alpha, seed in cases:
        g = make_cgrid(ni, nj, n_wake=nw, jitter=0.05, seed=seed, wall_spacing=1e-3)
        _, params = pair_params(nlevels=1, viscous=viscous, turb=0, mach=0.7, alpha_deg=alpha, re=1e5)
        u = perturbed_state(0.7, alpha, nj, ni, amp=0.03, seed=seed + 10)
        s = P.Solver(g, params)
        s.set_state(u)
        F_ref, _, _ = s.residual()
        s.close()
        u_dev = torch.from_numpy(np.ascontiguousarray(u).ravel()).cuda()
        rc, F = _noalloc_residual(lib, g, params, u_dev, torch)
        assert rc == 0, rc
        assert np.all(np.isfinite(F))
        err = np.abs(F - F_ref).max() / np.abs(F_ref).max()
        assert err < 1e-12, err


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    import paper_1710_04875_gb300 as P
    lib = P.library()
    g = make_cgrid(512, 128, wall_spacing=1e-5)
    _, params = pair_params(nlevels=1)
    u_dev = torch.zeros(4 * g.ni * g.nj, dtype=torch.float64, device="cuda")
    rc, _ = _noalloc_residual(lib, g, params, u_dev, torch)
    assert rc == -7
