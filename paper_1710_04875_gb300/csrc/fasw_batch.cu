// C ABI of batches: many independent cases advanced together in one captured CUDA graph per
// cycle, and the per-shape autotuner of their sweep variant.
#include <cmath>
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "fasw_ctx.cuh"

using namespace fasw;

extern "C" {

// Many independent cases (own grids, sizes and flow conditions) advanced together: every
// case is a context on its own stream, and one FAS cycle of all cases is captured into a
// single CUDA graph as parallel branches (fork on the batch stream, join back), so the GPU
// runs the cases' kernels concurrently.  The per-case sweep variant is chosen by timing.
struct fasw_batch {
  std::vector<fasw_ctx*> cases;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t st = nullptr;
  int own_stream = 0;
  struct G { int phase; cudaGraphExec_t exec; long long kernels; };
  std::vector<G> graphs;
  long long launches = 0;
};

static void batch_drop_graphs(fasw_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

int fasw_batch_create(int ncases, const int* ni, const int* nj, const int* n_wake, const double* const* x,
                      const double* const* y, int coords_on_device, const fasw_params* params, void* stream,
                      fasw_batch** out) {
  if (!out || ncases < 1 || !ni || !nj || !n_wake || !x || !y || !params) return FASW_ERR_ARG;
  *out = nullptr;
  fasw_batch* b = new (std::nothrow) fasw_batch();
  if (!b) return FASW_ERR_OOM;
  b->st = static_cast<cudaStream_t>(stream);
  if (!b->st) {  // graph capture needs a non-default stream
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return FASW_ERR_CUDA;
    }
    b->own_stream = 1;
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < ncases; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      fasw_batch_destroy(b);
      return FASW_ERR_CUDA;
    }
    b->streams.push_back(s);
    b->joins.push_back(e);
    fasw_ctx* c = nullptr;
    const int r = fasw_create(ni[k], nj[k], n_wake[k], x[k], y[k], coords_on_device, &params[k], s, &c);
    if (r != FASW_OK) {
      fasw_batch_destroy(b);
      return r;
    }
    c->in_batch = 1;
    c->sweep_kind = SWEEP_WS;  // as a single case: the warp strips in both precisions
    b->cases.push_back(c);
  }
  *out = b;
  return FASW_OK;
}

void fasw_batch_destroy(fasw_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_drop_graphs(b);
  for (fasw_ctx* c : b->cases) fasw_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b;
}

fasw_ctx* fasw_batch_case(fasw_batch* b, int k) {
  return (b && k >= 0 && k < (int)b->cases.size()) ? b->cases[k] : nullptr;
}

static double case_cfl(const fasw_ctx* c, int cycle_index) {
  return cycle_index < c->prm.ramp_cycles ? std::fmin(c->prm.cfl, c->prm.cfl_ramp) : c->prm.cfl;
}

int fasw_batch_cycle(fasw_batch* b, int cycle_index, double* norms) {
  if (!b) return FASW_ERR_ARG;
  // the cycle's launch sequence depends on each case's c*, i.e. on whether it is still ramped
  int phase = 0;
  for (size_t k = 0; k < b->cases.size(); ++k)
    if (cycle_index < b->cases[k]->prm.ramp_cycles) phase |= 1;
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b->graphs)
    if (g.phase == phase) {
      exec = g.exec;
      b->launches += g.kernels;
    }
  if (!exec) {
    long long before = 0;
    for (fasw_ctx* c : b->cases) before += c->launches;
    CKR(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(b->fork, b->st);
    for (size_t k = 0; k < b->cases.size(); ++k) {
      fasw_ctx* c = b->cases[k];
      cudaStreamWaitEvent(c->st, b->fork, 0);
      enqueue_cycle(c, case_cfl(c, cycle_index));
      cudaEventRecord(b->joins[k], c->st);
      cudaStreamWaitEvent(b->st, b->joins[k], 0);
    }
    cudaGraph_t graph = nullptr;
    CKR(cudaStreamEndCapture(b->st, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    long long after = 0;
    for (fasw_ctx* c : b->cases) after += c->launches;
    b->graphs.push_back({phase, exec, after - before});
    b->launches += after - before;
  }
  CKR(cudaGraphLaunch(exec, b->st));
  CKR(cudaStreamSynchronize(b->st));
  CKR(cudaGetLastError());
  for (size_t k = 0; k < b->cases.size(); ++k) {
    if (*b->cases[k]->h_err) return FASW_ERR_DEVICE_TIMEOUT;
    if (norms) norms[k] = *b->cases[k]->h_norm;
  }
  return FASW_OK;
}

int fasw_batch_solve(fasw_batch* b, double drop, int max_cycles, int* cycles, double* final_drop, int* ncycles) {
  if (!b || max_cycles < 1) return FASW_ERR_ARG;
  const size_t nc = b->cases.size();
  std::vector<double> n0(nc, 0.0), nk(nc, 0.0);
  std::vector<int> done(nc, 0);  // 1 converged, 2 diverged (its cycles[] is -2)
  int diverged = 0;
  for (int k = 0; k < max_cycles; ++k) {
    int r = fasw_batch_cycle(b, k, nk.data());
    if (r) return r;
    if (ncycles) *ncycles = k + 1;
    size_t ndone = 0;
    for (size_t q = 0; q < nc; ++q) {
      if (k == 0) n0[q] = nk[q];
      if (!done[q]) {
        if (final_drop) final_drop[q] = nk[q] / n0[q];
        if (!std::isfinite(nk[q]) || (k > 0 && nk[q] > 1e8 * n0[q])) {
          done[q] = 2;
          diverged = 1;
          if (cycles) cycles[q] = -2;
        } else if (k > 0 && nk[q] <= drop * n0[q]) {
          done[q] = 1;
          if (cycles) cycles[q] = k + 1;
        }
      }
      ndone += done[q] != 0;
    }
    if (ndone == nc) return diverged ? FASW_ERR_DIVERGED : FASW_OK;
  }
  for (size_t q = 0; q < nc; ++q)
    if (!done[q] && cycles) cycles[q] = -1;
  return diverged ? FASW_ERR_DIVERGED : FASW_ERR_NOT_CONVERGED;
}

// Autotuner.  Candidates are the sweep variants whose CTAs never wait on one another (strip
// sweeps are not candidates: their CTAs wait on each other, which is safe only while all CTAs
// of one sweep are resident, and concurrent branches of a batch graph do not guarantee that):
// the hyperplane-staged FP32 sweep with a ring of 8 or 4 steps and the one-CTA sweep.  Which
// wins depends on the grid shape and on how full the GPU is, so the tuner times whole batch
// cycles (all cases concurrently, CUDA events, states saved and restored) and improves the
// choice one grid shape (ni, nj) at a time, keeping a change only when the batch gets faster.
// Results are cached per (ni, nj, precision) for the process: a later batch whose shapes are
// all cached takes them without timing.
namespace {
struct TuneKey {
  int ni, nj, mixed;
  bool operator<(const TuneKey& o) const {
    return ni != o.ni ? ni < o.ni : nj != o.nj ? nj < o.nj : mixed < o.mixed;
  }
};
std::map<TuneKey, std::pair<int, int>> g_tune_cache;  // (sweep kind, residual tile height)
std::mutex g_tune_mutex;

TuneKey key_of(fasw_ctx* c) {
  const LevelDev& F = c->lev[c->L()];
  return TuneKey{F.ni, F.nj, c->mixed};
}
}  // namespace

static void set_tile(fasw_ctx* c, int rows) {
  for (auto& L : c->lev) L.res_ty = rows;
}

// Times `reps` batch cycles with sweep kinds[k] and residual tile height tys[k] on case k (after
// one capturing cycle); states restored.
static int batch_time(fasw_batch* b, const std::vector<int>& kinds, const std::vector<int>& tys,
                      const std::vector<double*>& saved, int reps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  for (size_t k = 0; k < b->cases.size(); ++k) {
    b->cases[k]->sweep_kind = kinds[k];
    set_tile(b->cases[k], tys[k]);
    drop_graphs(b->cases[k]);
  }
  batch_drop_graphs(b);
  int r = fasw_batch_cycle(b, 0, nullptr);  // capture + warm-up
  if (r) return r;
  CKR(cudaEventRecord(e0, b->st));
  for (int rep = 0; rep < reps; ++rep)
    if ((r = fasw_batch_cycle(b, 0, nullptr))) return r;
  CKR(cudaEventRecord(e1, b->st));
  CKR(cudaEventSynchronize(e1));
  CKR(cudaEventElapsedTime(ms, e0, e1));
  for (size_t k = 0; k < b->cases.size(); ++k) {  // restore the states
    fasw_ctx* c = b->cases[k];
    launch_pack(c->lev[c->L()], saved[k], 1, nullptr, c->st);
    launch_bc(c->lev[c->L()], c->ph, c->st);
    CKR(cudaStreamSynchronize(c->st));
  }
  return FASW_OK;
}

// choice (nullable, ncases): the kind used for case k.
int fasw_batch_autotune(fasw_batch* b, int* choice) {
  if (!b) return FASW_ERR_ARG;
  const size_t nc = b->cases.size();
  std::vector<int> kinds(nc), tys(nc, 0);
  for (size_t k = 0; k < nc; ++k) kinds[k] = SWEEP_WS;
  std::map<TuneKey, std::vector<size_t>> groups;
  for (size_t k = 0; k < nc; ++k) groups[key_of(b->cases[k])].push_back(k);
  bool all_cached = true;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (auto& gk : groups) {
      auto it = g_tune_cache.find(gk.first);
      if (it == g_tune_cache.end()) {
        all_cached = false;
        continue;
      }
      for (size_t k : gk.second) {
        kinds[k] = it->second.first;
        tys[k] = it->second.second;
      }
    }
  }
  if (!all_cached) {
    std::vector<double*> saved(nc, nullptr);
    for (size_t k = 0; k < nc; ++k) {
      fasw_ctx* c = b->cases[k];
      saved[k] = c->d_tmp2;  // 4 x n of the finest level
      launch_pack(c->lev[c->L()], nullptr, 0, saved[k], c->st);
      CKR(cudaStreamSynchronize(c->st));
    }
    cudaEvent_t e0, e1;
    CKR(cudaEventCreate(&e0));
    CKR(cudaEventCreate(&e1));
    const int reps = 3;
    int r = FASW_OK;
    // the faster of two timings of the same kinds, so that one noisy timing decides nothing
    auto timed = [&](float* out) {
      float a = 0.f, c2 = 0.f;
      if ((r = batch_time(b, kinds, tys, saved, reps, e0, e1, &a))) return;
      if ((r = batch_time(b, kinds, tys, saved, reps, e0, e1, &c2))) return;
      *out = std::min(a, c2);
    };
    // sweep variants whose CTAs never wait on a CTA that may not be resident (one CTA, or the
    // warp strips launched as one cluster); the FP32 staged kinds only in mixed precision
    const int cand_mixed[5] = {SWEEP_HP8, SWEEP_HP4, SWEEP_CTA, SWEEP_WS, SWEEP_WS8};
    const int cand_fp64[3] = {SWEEP_WS, SWEEP_WS8, SWEEP_CTA};
    const int tile_cand[5] = {0, 1, 2, 4, 8};
    // larger shapes first: they dominate the batch time
    std::vector<std::pair<TuneKey, std::vector<size_t>>> order(groups.begin(), groups.end());
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) {
      return (long long)x.first.ni * x.first.nj * x.second.size() > (long long)y.first.ni * y.first.nj * y.second.size();
    });
    // each candidate against the incumbent timed right beside it; a switch must gain 2 %
    for (size_t gi = 0; gi < order.size() && r == FASW_OK; ++gi) {
      const std::vector<size_t>& members = order[gi].second;
      const bool mixed = order[gi].first.mixed != 0;
      const int* cand = mixed ? cand_mixed : cand_fp64;
      const int ncand = mixed ? 5 : 3;
      // sweep variant first (it dominates), then the residual tile height with it
      int keep = kinds[members[0]];
      for (int ci = 0; ci < ncand; ++ci) {
        const int k = cand[ci];
        if (k == keep || r) continue;
        float t_keep = 0.f, t_k = 0.f;
        timed(&t_keep);
        for (size_t m : members) kinds[m] = k;
        if (r == FASW_OK) timed(&t_k);
        if (r == FASW_OK && t_k < 0.98f * t_keep) keep = k;
        for (size_t m : members) kinds[m] = keep;
      }
      int keep_ty = tys[members[0]];
      for (int ty : tile_cand) {
        if (ty == keep_ty || r) continue;
        float t_keep = 0.f, t_k = 0.f;
        timed(&t_keep);
        for (size_t m : members) tys[m] = ty;
        if (r == FASW_OK) timed(&t_k);
        if (r == FASW_OK && t_k < 0.98f * t_keep) keep_ty = ty;
        for (size_t m : members) tys[m] = keep_ty;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (auto& gk : groups) g_tune_cache[gk.first] = {kinds[gk.second[0]], tys[gk.second[0]]};
  }
  for (size_t k = 0; k < nc; ++k) {
    b->cases[k]->sweep_kind = kinds[k];
    set_tile(b->cases[k], tys[k]);
    drop_graphs(b->cases[k]);
    if (choice) choice[k] = kinds[k] | (tys[k] << 8);
  }
  batch_drop_graphs(b);
  return FASW_OK;
}

long long fasw_batch_launch_count(fasw_batch* b) { return b ? b->launches : -1; }

}  // extern "C"
