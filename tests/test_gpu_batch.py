"""Batched cases (one captured CUDA graph per cycle, one branch per case): every case of
uneven size follows exactly the history of its own single-case solve, and the autotuner's
choice does not change the results beyond rounding."""
import numpy as np
import pytest

import paper_1710_04875_gb300 as P
from synth.cgrid import make_cgrid
from tests.helpers import pair_params, rel_err

pytestmark = pytest.mark.gpu

CASES = [(128, 32, 0.8, 1.25, 0.10), (96, 24, 0.7, -1.0, 0.08), (160, 40, 0.6, 3.0, 0.12), (128, 48, 0.75, 0.5, 0.10)]


def _case(ni, nj, mach, alpha, t, precision="fp64"):
    g = make_cgrid(ni, nj, thickness=t)
    _, p = pair_params(nlevels=3, mach=mach, alpha_deg=alpha, cfl=100.0, precision=precision)
    return g, p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_case_runs(precision):
    gs, ps = zip(*[_case(*c, precision=precision) for c in CASES])
    b = P.fasw.Batch(list(gs), list(ps))
    singles = [P.Solver(g, p) for g, p in zip(gs, ps)]
    for k in range(8):
        nb = b.cycle(k)
        ns = np.array([s.fas_cycle(k) for s in singles])
        np.testing.assert_allclose(nb, ns, rtol=1e-13, atol=0)
    for q, s in enumerate(singles):
        assert rel_err(b.get_state(q), s.get_state()) < 1e-13


def test_batch_solve_and_autotune():
    gs, ps = zip(*[_case(*c) for c in CASES])
    b = P.fasw.Batch(list(gs), list(ps))
    choice = b.autotune()
    assert all(c in (2, 5) for c in choice)
    code, cycles, drops, ncy = b.solve(1e-3, 120)
    assert code == 0 and np.all(cycles > 0) and np.all(drops <= 1e-3)
    ref = P.Solver(gs[0], ps[0])
    c0, n0, h0 = ref.solve(1e-3, 120)
    assert abs(n0 - cycles[0]) <= 1
