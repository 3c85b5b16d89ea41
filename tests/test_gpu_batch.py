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
    tuned = b.autotune(with_tiles=True)
    assert all(c in (2, 9, 10) for c, _ in tuned)        # FP64 cases: one CTA or the warp strips
    assert all(t in (0, 1, 2, 4, 8) for _, t in tuned)
    code, cycles, drops, ncy = b.solve(1e-3, 120)
    assert code == 0 and np.all(cycles > 0) and np.all(drops <= 1e-3)
    ref = P.Solver(gs[0], ps[0])
    c0, n0, h0 = ref.solve(1e-3, 120)
    assert abs(n0 - cycles[0]) <= 1


def test_autotune_choices_are_cached_per_shape():
    """A second batch with the same grid shapes takes the cached choices without timing, and
    cases of one shape share one choice."""
    import time
    gs, ps = zip(*[_case(*c) for c in CASES])
    b1 = P.fasw.Batch(list(gs), list(ps))
    c1 = b1.autotune()
    b2 = P.fasw.Batch(list(gs), list(ps))
    t0 = time.perf_counter()
    c2 = b2.autotune()
    assert list(c1) == list(c2)
    assert time.perf_counter() - t0 < 1.0
    shapes = {}
    for g, c in zip(gs, c1):
        shapes.setdefault((g.ni, g.nj), set()).add(c)
    assert all(len(v) == 1 for v in shapes.values())


def test_mixed_batch_autotune_candidates_and_results():
    """Mixed-precision batch: the tuner picks among the co-scheduled sweep kinds and a residual
    tile height, and the tuned batch still converges like the single-case run."""
    gs, ps = zip(*[_case(*c, precision="mixed") for c in CASES])
    b = P.fasw.Batch(list(gs), list(ps))
    tuned = b.autotune(with_tiles=True)
    assert all(c in (2, 5, 6, 7, 9) for c, _ in tuned)
    code, cycles, drops, ncy = b.solve(1e-3, 120)
    assert code == 0 and np.all(cycles > 0)
