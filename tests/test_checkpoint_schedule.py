"""Host logic of the unsteady adjoint's reverse sweep: the binomial checkpoint schedule the
library plans (no GPU needed).

- every schedule is executable and delivers the time levels N, ..., 1 once each, in order,
  never holding more than `snapshots` stored levels besides the initial state;
- its count of physical steps equals the optimum found by a shortest-path search over all
  action sequences on small cases;
- and equals the closed form of binomial checkpointing (Griewank and Walther, "Algorithm 799:
  revolve", ACM TOMS 2000): t(l, s) = r l - C(s + r, r - 1) with r the least integer such that
  C(s + r, s) >= l, taken at l = N + 1 steps and s + 1 snapshots (the initial state is an extra
  stored level, and a level is consumed as the output of its step rather than the input).
"""
import heapq
from math import comb

import pytest

import paper_1710_04875_gb300 as P

ADVANCE, STORE, RESTORE, CONSUME, FREE = range(5)


def simulate(nsteps, snapshots, actions):
    pos, stored, consumed, steps = 0, set(), [], 0
    for op, arg in actions:
        if op == ADVANCE:
            assert arg > pos
            steps += arg - pos
            pos = arg
        elif op == STORE:
            assert arg == pos and arg not in stored and arg > 0
            stored.add(arg)
            assert len(stored) <= snapshots
        elif op == RESTORE:
            assert arg == 0 or arg in stored
            pos = arg
        elif op == CONSUME:
            assert arg == pos
            consumed.append(arg)
        elif op == FREE:
            stored.remove(arg)
        else:
            raise AssertionError(op)
    assert consumed == list(range(nsteps, 0, -1))
    return steps


def optimum(nsteps, snapshots):
    """Fewest physical steps over every action sequence (Dijkstra on (pos, stored, next))."""
    start = (0, frozenset(), nsteps)
    dist = {start: 0}
    heap = [(0, 0, frozenset(), nsteps)]
    while heap:
        d, pos, st, k = heapq.heappop(heap)
        if k == 0:
            return d
        if dist.get((pos, st, k), 1 << 60) < d:
            continue
        moves = []
        if pos < k:
            moves.append((1, (pos + 1, st, k)))
        if pos == k:
            moves.append((0, (pos, st, k - 1)))
        if pos > 0 and pos not in st and len(st) < snapshots:
            moves.append((0, (pos, st | {pos}, k)))
        for x in list(st) + [0]:
            if x <= k:
                moves.append((0, (x, st, k)))
        for x in st:
            moves.append((0, (pos, st - {x}, k)))
        for c, nxt in moves:
            nd = d + c
            if nd < dist.get(nxt, 1 << 60):
                dist[nxt] = nd
                heapq.heappush(heap, (nd, *nxt))
    raise AssertionError("unreachable")


def binomial_closed_form(l, s):
    r = 0
    while comb(s + r, s) < l:
        r += 1
    return r * l - comb(s + r, r - 1)


@pytest.mark.parametrize("nsteps", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("snapshots", [0, 1, 2, 3])
def test_schedule_is_valid_and_optimal_on_small_cases(nsteps, snapshots):
    acts, fs = P.checkpoint_schedule(nsteps, snapshots)
    assert simulate(nsteps, snapshots, acts) == fs
    assert fs == optimum(nsteps, snapshots)


@pytest.mark.parametrize("nsteps,snapshots", [(10, 2), (50, 3), (128, 4), (128, 8), (300, 5), (1000, 10)])
def test_schedule_cost_is_the_binomial_optimum(nsteps, snapshots):
    acts, fs = P.checkpoint_schedule(nsteps, snapshots)
    assert simulate(nsteps, snapshots, acts) == fs
    assert fs == binomial_closed_form(nsteps + 1, snapshots + 1)


def test_enough_snapshots_store_every_level_once():
    for n in (1, 4, 64):
        acts, fs = P.checkpoint_schedule(n, n)
        assert fs == n and simulate(n, n, acts) == n
        acts2, fs2 = P.checkpoint_schedule(n, max(n - 1, 0))
        assert acts2 == acts


def test_schedule_rejects_bad_arguments():
    with pytest.raises(P.FaswError):
        P.checkpoint_schedule(0, 2)
    with pytest.raises(P.FaswError):
        P.checkpoint_schedule(4, -1)
