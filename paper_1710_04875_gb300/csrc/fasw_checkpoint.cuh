// Binomial checkpoint schedule for the reverse sweep of the unsteady adjoint
// (checkpoint_schedule.cu).  Host code only.
#pragma once
#include <vector>

namespace fasw {

// Actions on a machine whose working state holds one time level (u^p, u^(p-1)); level 0 (the
// initial state) is always stored.
enum CkOp {
  CK_ADVANCE = 0,  // physical steps from the current level up to level arg
  CK_STORE = 1,    // store the current level (arg) in a free slot
  CK_RESTORE = 2,  // make the stored level arg current
  CK_CONSUME = 3,  // adjoint step of level arg (the current level)
  CK_FREE = 4      // release the slot of level arg
};

struct CkAction {
  int op;
  int arg;
};

constexpr int CK_MAX_STEPS = 1 << 16;

// Actions of the fewest-recomputation schedule for nsteps levels with `snapshots` slots;
// *forward_steps = the physical steps it runs (the initial sweep included).
int checkpoint_schedule(int nsteps, int snapshots, std::vector<CkAction>& out, long long* forward_steps);

}  // namespace fasw
