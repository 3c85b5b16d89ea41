// Binomial checkpointing for the reverse sweep of the unsteady adjoint (host code only).
//
// The adjoint of dual time stepping visits the time levels backwards, n = N, ..., 1, and at
// level n needs the converged primal state u^n.  Holding every u^n costs N states; with s
// stored levels besides the initial state the states are recomputed from the nearest stored
// level instead, and the schedule below recomputes as few physical steps as possible: the
// binomial checkpointing of Griewank and Walther ("Algorithm 799: revolve", ACM TOMS 2000),
// derived here as a dynamic programme.
//
// Let C(l, s) be the fewest physical steps that deliver the levels a + l, ..., a + 1 (in that
// order) when level a is stored and s further slots are free.  With no slot, every level is
// recomputed from a: C(l, 0) = l (l + 1) / 2.  Otherwise the first advance goes k steps to
// m = a + k and stores m; the levels above m are then delivered with s - 1 free slots, m
// itself from its slot, and the levels below m (slot freed) with s slots:
//   C(l, s) = min over 1 <= k <= l of  k + C(l - k, s - 1) + C(k - 1, s).
// The initial forward sweep that evaluates the objective is the first chain of advances of
// this schedule, so C(N, s) counts every physical step of the whole adjoint run (C(N, s) = N
// when s >= N - 1: every level is stored once).  A level stored in a slot holds u^m and
// u^(m-1), the two states a BDF2 step starts from.
#include <vector>

#include "../../include/fasw.h"
#include "fasw_checkpoint.cuh"

namespace fasw {

namespace {

struct Planner {
  int N = 0, S = 0;
  std::vector<long long> cost;  // (N + 1) x (S + 1)
  std::vector<int> split;
  std::vector<CkAction>* out = nullptr;
  int pos = 0;  // the level the working state holds

  long long& C(int l, int s) { return cost[(size_t)l * (S + 1) + s]; }
  int& K(int l, int s) { return split[(size_t)l * (S + 1) + s]; }

  void table() {
    cost.assign((size_t)(N + 1) * (S + 1), 0);
    split.assign((size_t)(N + 1) * (S + 1), 0);
    for (int l = 1; l <= N; ++l) C(l, 0) = (long long)l * (l + 1) / 2;
    for (int s = 1; s <= S; ++s)
      for (int l = 1; l <= N; ++l) {
        long long best = -1;
        int arg = 1;
        for (int k = 1; k <= l; ++k) {
          const long long v = k + C(l - k, s - 1) + C(k - 1, s);
          if (best < 0 || v < best) {
            best = v;
            arg = k;
          }
        }
        C(l, s) = best;
        K(l, s) = arg;
      }
  }

  void emit(int op, int arg) { out->push_back({op, arg}); }
  void restore(int a) {
    if (pos != a) emit(CK_RESTORE, a);
    pos = a;
  }
  void advance(int m) {
    emit(CK_ADVANCE, m);
    pos = m;
  }

  // deliver levels b, ..., a + 1 with level a stored and s slots free
  void reverse(int a, int b, int s) {
    while (b > a) {
      const int l = b - a;
      if (s == 0 || l == 1) {
        restore(a);
        advance(b);
        emit(CK_CONSUME, b);
        --b;
        continue;
      }
      const int m = a + K(l, s);
      restore(a);
      advance(m);
      if (m < b) {
        emit(CK_STORE, m);
        reverse(m, b, s - 1);
        restore(m);
        emit(CK_CONSUME, m);
        emit(CK_FREE, m);
      } else {
        emit(CK_CONSUME, m);
      }
      b = m - 1;
    }
  }
};

}  // namespace

int checkpoint_schedule(int nsteps, int snapshots, std::vector<CkAction>& out, long long* forward_steps) {
  if (nsteps < 1 || nsteps > CK_MAX_STEPS || snapshots < 0) return FASW_ERR_ARG;
  Planner p;
  p.N = nsteps;
  p.S = snapshots < nsteps - 1 ? snapshots : nsteps - 1;  // more slots than that are never used
  if ((double)p.N * p.N * p.S > 4.0e9) return FASW_ERR_ARG;  // planning would take minutes
  p.table();
  out.clear();
  p.out = &out;
  p.pos = 0;
  p.reverse(0, nsteps, p.S);
  long long steps = 0, pos = 0;
  for (const CkAction& a : out) {
    if (a.op == CK_ADVANCE) {
      steps += a.arg - pos;
      pos = a.arg;
    } else if (a.op == CK_RESTORE) {
      pos = a.arg;
    }
  }
  if (forward_steps) *forward_steps = steps;
  return FASW_OK;
}

}  // namespace fasw

extern "C" int fasw_checkpoint_schedule(int nsteps, int snapshots, int* ops, int* args, int capacity, int* nactions,
                                        long long* forward_steps) {
  if (!nactions || capacity < 0 || (capacity > 0 && (!ops || !args))) return FASW_ERR_ARG;
  std::vector<fasw::CkAction> acts;
  const int r = fasw::checkpoint_schedule(nsteps, snapshots, acts, forward_steps);
  if (r) return r;
  *nactions = (int)acts.size();
  if ((int)acts.size() > capacity) return capacity == 0 ? FASW_OK : FASW_ERR_ARG;
  for (size_t k = 0; k < acts.size(); ++k) {
    ops[k] = acts[k].op;
    args[k] = acts[k].arg;
  }
  return FASW_OK;
}
