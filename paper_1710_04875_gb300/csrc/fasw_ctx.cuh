// Host-side context of the C ABI, shared by the translation units that implement it:
// fasw_api.cu (levels, stage loop, FAS cycle, steady and dual-time solves), fasw_adjoint_api.cu
// (discrete adjoint, unsteady adjoint, shape and vertex gradients) and fasw_batch.cu (batches
// and the per-shape sweep autotuner).
#pragma once
#include <string>
#include <vector>

#include "../../include/fasw.h"
#include "fasw_internal.cuh"
#include "fasw_sweep.cuh"
#include "fasw_adjoint.cuh"

namespace fasw {
extern thread_local std::string g_last_cuda_error;
int cuda_fail(cudaError_t e);
}  // namespace fasw

#define CKR(expr)                                       \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return fasw::cuda_fail(e_);  \
  } while (0)

struct fasw_ctx {
  fasw_params prm{};
  fasw::PhysParams ph{};
  fasw::SchemeParams sc{};
  std::vector<fasw::LevelDev> lev;
  std::vector<void*> allocs;
  cudaStream_t st = nullptr;
  int mixed = 0;
  double* d_norm = nullptr;
  double* h_norm = nullptr;    // pinned
  double* d_tmp = nullptr;     // 4 * n_finest scratch for host copies
  double* d_tmp2 = nullptr;
  double* d_tmp3 = nullptr;
  long long launches = 0;
  // optional per-kernel-class timing with CUDA events on the context's stream
  int profiling = 0;
  struct Pending { int id; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  long long prof_count[FASW_NKERNELS] = {};
  double prof_ms[FASW_NKERNELS] = {};
  // captured FAS cycles, one per pseudo CFL value (ramp and full)
  struct CycleGraph { double cfl; cudaGraphExec_t exec; long long kernels; };
  std::vector<CycleGraph> graphs;
  int use_graphs = 1;
  int sweep_kind = fasw::SWEEP_AUTO;
  int in_batch = 0;             // a case of a batch: its kernels run beside other cases' kernels
  bool mut_frozen = false;       // eddy viscosity held at a value set by fasw_freeze_mut
  int exact_iters = 0;          // > 0: the preconditioner iterates toward the exact (D+L+U)^-1
  long long spin_limit = 1LL << 22;
  long long* d_prog = nullptr;  // strip progress flags
  int* d_err = nullptr;         // device error word (bounded waits)
  int* h_err = nullptr;         // pinned copy
  double* d_x0 = nullptr;       // reference vertices (the grid at rest)
  double* d_y0 = nullptr;
  double* d_un = nullptr;       // dual-time history of the finest level (4 x n)
  double* d_unm1 = nullptr;
  int steps_done = 0;
  fasw::AdjointDev adj;               // discrete adjoint of the steady finest level (built on demand)
  int L() const { return (int)lev.size() - 1; }
};

namespace fasw {
// driver steps (fasw_api.cu)
int level_sweep_kind(const fasw_ctx* c, const LevelDev& L);
void run_sweep(fasw_ctx* c, const LevelDev& L, int do_update, double alpha, const double* rhs);
void bc_aux(fasw_ctx* c, int l, double cfl, int want_dts);
void smooth_step(fasw_ctx* c, int l, double cfl, bool record_norm);
void fas_cycle_rec(fasw_ctx* c, int l, double cfl, bool record_norm);
void enqueue_cycle(fasw_ctx* c, double cfl);
void drop_graphs(fasw_ctx* c);
int check_level(fasw_ctx* c, int l);
int copy_in(fasw_ctx* c, double* dst, const double* src, size_t count, int on_device);
int copy_out(fasw_ctx* c, double* dst, const double* src, size_t count, int on_device);
int sync(fasw_ctx* c);
// device error word of the bounded waits: cleared on the stream at the start of a call that runs
// sweeps, read (with a stream synchronize) at its end
void err_clear(fasw_ctx* c);
int err_read(fasw_ctx* c);
}  // namespace fasw
