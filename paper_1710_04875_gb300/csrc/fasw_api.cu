// C ABI and host-side driver: level allocation, the AW / ARK stage loop (sections 4.1-4.2
// of arXiv 1710.04875), the FAS V/W cycle (section 3) and the steady solve loop.
// Every arithmetic step runs in the kernels of the other translation units.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/fasw.h"
#include "fasw_internal.cuh"
#include "fasw_sweep.cuh"
#include "fasw_adjoint.cuh"
#include "fasw_transfer.cuh"
#include "fasw_checkpoint.cuh"

using namespace fasw;

namespace {

thread_local std::string g_last_cuda_error;

// Table "RK smoothers" (section 4.1); the W methods use the same coefficients, the
// 5-stage ARK51/ARK52 alphas take the ARK5J betas, and the ARK5J beta row is read as
// (1, 0, 0.56, 0, 0.44).
struct Coef { int s; double a[5], b[5]; };
const Coef kCoef[4] = {
    {3, {0.1481, 2.0 / 5.0, 1.0, 0, 0}, {1.0, 0.5, 0.5, 0, 0}},
    {5, {1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0}, {1.0, 0.0, 0.56, 0.0, 0.44}},
    {5, {0.0533, 0.1263, 0.2375, 0.4414, 1.0}, {1.0, 0.0, 0.56, 0.0, 0.44}},
    {5, {0.0695, 0.1602, 0.2898, 0.5060, 1.0}, {1.0, 0.0, 0.56, 0.0, 0.44}},
};

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return FASW_ERR_CUDA;
}

#define CKR(expr)                             \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

}  // namespace

struct fasw_ctx {
  fasw_params prm{};
  PhysParams ph{};
  SchemeParams sc{};
  std::vector<LevelDev> lev;
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
  int sweep_kind = SWEEP_AUTO;
  long long spin_limit = 1LL << 22;
  long long* d_prog = nullptr;  // strip progress flags
  int* d_err = nullptr;         // device error word (bounded waits)
  int* h_err = nullptr;         // pinned copy
  double* d_x0 = nullptr;       // reference vertices (the grid at rest)
  double* d_y0 = nullptr;
  double* d_un = nullptr;       // dual-time history of the finest level (4 x n)
  double* d_unm1 = nullptr;
  int steps_done = 0;
  AdjointDev adj;               // discrete adjoint of the steady finest level (built on demand)
  int L() const { return (int)lev.size() - 1; }
};

namespace {

template <typename T>
int dalloc(fasw_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    g_last_cuda_error = cudaGetErrorString(e);
    return FASW_ERR_OOM;
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return FASW_OK;
}

cudaEvent_t pool_get(fasw_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch with events when profiling is on.
struct Prof {
  fasw_ctx* c;
  int id;
  cudaEvent_t a = nullptr;
  Prof(fasw_ctx* cc, int k) : c(cc), id(k) {
    if (c->profiling) {
      a = pool_get(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~Prof() {
    if (a) {
      cudaEvent_t b = pool_get(c);
      cudaEventRecord(b, c->st);
      c->pending.push_back({id, a, b});
    }
  }
};

void prof_resolve(fasw_ctx* c) {
  for (auto& q : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      c->prof_ms[q.id] += ms;
      c->prof_count[q.id] += 1;
    }
    c->event_pool.push_back(q.a);
    c->event_pool.push_back(q.b);
  }
  c->pending.clear();
}

int alloc_level(fasw_ctx* c, LevelDev& L) {
  int r = FASW_OK;
  const size_t n = L.n, G = L.Gn, nfx = L.nfx, nfe = L.nfe;
#define A(ptr, cnt) if ((r = dalloc(c, &(ptr), (cnt))) != FASW_OK) return r
  A(L.u, 4 * G);
  A(L.u0, 4 * n);
  A(L.fvc, 4 * n);
  A(L.rhs, 4 * n);
  A(L.s, 4 * n);
  A(L.ut, 4 * n);
  A(L.src, 4 * n);
  A(L.p, G);
  A(L.q, G);
  A(L.rinv, G);
  A(L.rt, 2 * n);
  A(L.dts, n);
  A(L.sxi, 2 * nfx);
  A(L.seta, 2 * nfe);
  A(L.vol, n);
  A(L.mut, n);
  A(L.wdist, n);
  A(L.omega, n);
  A(L.coef, n);
  A(L.blk64, 32 * (nfx + nfe));
  A(L.dlu64, 16 * n);
  A(L.yz64, 4 * n);
  A(L.blk32, 32 * (nfx + nfe));
  A(L.dlu32, 16 * n);
  A(L.yz32, 4 * n);
  A(L.norm_part, (size_t)residual_blocks(L));
  A(L.tb, 80 * n);
  A(L.vfx, nfx);
  A(L.vfe, nfe);
  A(L.wvx, (size_t)L.ni);
  A(L.wvy, (size_t)L.ni);
  if (c->mixed && hp_fits(L.ni, L.nj, L.nw)) {
    const size_t h = hp_floats(L.ni, L.nj);
    A(L.hpF, 32 * h);
    A(L.hpB, 32 * h);
    A(L.hpC, 4 * h);
    A(L.hpY, 4 * h);
  }
#undef A
  CKR(cudaMemsetAsync(L.vfx, 0, nfx * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.vfe, 0, nfe * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.wvx, 0, (size_t)L.ni * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.wvy, 0, (size_t)L.ni * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.s, 0, 4 * n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.src, 0, 4 * n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.mut, 0, n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.fvc, 0, 4 * n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.rhs, 0, 4 * n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.ut, 0, 4 * n * sizeof(double), c->st));
  CKR(cudaMemsetAsync(L.wdist, 0, n * sizeof(double), c->st));
  return FASW_OK;
}

void free_stream(double mach, double alpha_deg, double w[4]) {
  const double al = alpha_deg * M_PI / 180.0;
  const double p = 1.0 / (GAM * mach * mach);
  const double u = std::cos(al), v = std::sin(al);
  w[0] = 1.0;
  w[1] = u;
  w[2] = v;
  w[3] = p / (GAM - 1.0) + 0.5 * (u * u + v * v);
}

// ---- driver steps
// Sweep kind used on a level: automatic = hyperplane-staged FP32 sweep where the level fits
// (mixed), else one CTA (mixed) or strips (FP64); a requested kind that does not apply to the
// level or precision falls back the same way.
int level_sweep_kind(const fasw_ctx* c, const LevelDev& L) {
  int k = c->sweep_kind;
  if (k == SWEEP_AUTO || (is_hp(k) && !(c->mixed && L.hpF)))
    k = c->mixed ? (L.hpF ? SWEEP_HP : SWEEP_CTA) : SWEEP_STRIPS;
  return k;
}

void run_sweep(fasw_ctx* c, const LevelDev& L, int do_update, double alpha, const double* rhs) {
  if (c->sweep_kind == SWEEP_LEGACY) {
    launch_sgs(L, c->sc, c->mixed, do_update, alpha, rhs, nullptr, c->st);
    ++c->launches;
    return;
  }
  c->launches += launch_sweep(L, c->mixed, level_sweep_kind(c, L), do_update, c->sc.aw, alpha, rhs, c->d_prog,
                              c->d_err, c->spin_limit, c->st);
}

void bc_aux(fasw_ctx* c, int l, double cfl, int want_dts) {
  Prof p(c, FASW_K_CELL_AUX);
  launch_bc_aux(c->lev[l], c->ph, cfl, want_dts, c->st);
  ++c->launches;
}

// One smoothing step on level l: dt* and the preconditioner frozen at u^(0) (reading G19),
// then the s-stage low-storage loop; AW applies W^-1 to (dt* r), ARK applies dt* P^-1 r.
void smooth_step(fasw_ctx* c, int l, double cfl, bool record_norm) {
  LevelDev& L = c->lev[l];
  const SchemeParams& sc = c->sc;
  bc_aux(c, l, cfl, 1);
  { Prof p(c, FASW_K_FACE_BLOCKS); launch_face_blocks(L, c->ph, sc, c->mixed, c->st); }
  { Prof p(c, FASW_K_DIAG_BLOCKS); launch_diag_blocks(L, sc, c->mixed, c->st); }  // also saves u^(0)
  c->launches += 2;
  if (c->sweep_kind != SWEEP_LEGACY) {
    Prof p(c, FASW_K_DIAG_BLOCKS);
    launch_sgs_prep(L, c->mixed, level_sweep_kind(c, L), c->st);
    ++c->launches;
  }
  for (int i = 1; i <= sc.nstages; ++i) {
    if (i > 1) bc_aux(c, l, cfl, 0);
    ResArgs a{};
    a.mode = RES_STAGE;
    a.stage = i;
    a.beta = sc.beta[i - 1];
    a.aw = sc.aw;
    a.want_norm = (record_norm && i == 1) ? 1 : 0;
    a.norm_all = c->prm.norm_all;
    { Prof p(c, FASW_K_RESIDUAL); launch_residual(L, c->ph, a, c->st); }
    if (a.want_norm) {
      Prof p(c, FASW_K_NORM);
      launch_norm_final(L, residual_blocks(L), L.n * (c->prm.norm_all ? 4 : 1), c->d_norm, c->st);
      ++c->launches;
    }
    { Prof p(c, FASW_K_SGS); run_sweep(c, L, 1, sc.alpha[i - 1], L.rhs); }
    ++c->launches;  // the residual
  }
  // no ghost refill here: every consumer of the ghosts starts with its own fill (bc_aux)
}

void fas_cycle_rec(fasw_ctx* c, int l, double cfl, bool record_norm) {
  for (int k = 0; k < c->prm.nu1; ++k) smooth_step(c, l, cfl, record_norm && k == 0);
  if (l == 0) return;
  LevelDev& F = c->lev[l];
  LevelDev& C = c->lev[l - 1];
  bc_aux(c, l, cfl, 0);
  ResArgs a{};
  a.mode = RES_FASRES;
  { Prof p(c, FASW_K_RESIDUAL); launch_residual(F, c->ph, a, c->st); }
  { Prof p(c, FASW_K_RESTRICT); launch_restrict(F, C, c->prm.turb, c->st); }
  c->launches += 2;
  bc_aux(c, l - 1, cfl, 0);
  ResArgs b{};
  b.mode = RES_FORCING;
  { Prof p(c, FASW_K_RESIDUAL); launch_residual(C, c->ph, b, c->st); }
  ++c->launches;
  for (int g = 0; g < c->prm.gamma_cycle; ++g) fas_cycle_rec(c, l - 1, cfl, false);
  { Prof p(c, FASW_K_PROLONG); launch_prolong(F, C, c->st); }
  ++c->launches;
}

void drop_graphs(fasw_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

int check_level(fasw_ctx* c, int l) { return (c && l >= 0 && l < (int)c->lev.size()) ? FASW_OK : FASW_ERR_ARG; }

int copy_in(fasw_ctx* c, double* dst, const double* src, size_t count, int on_device) {
  CKR(cudaMemcpyAsync(dst, src, count * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      c->st));
  return FASW_OK;
}

int copy_out(fasw_ctx* c, double* dst, const double* src, size_t count, int on_device) {
  CKR(cudaMemcpyAsync(dst, src, count * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      c->st));
  return FASW_OK;
}

int sync(fasw_ctx* c) {
  CKR(cudaGetLastError());
  CKR(cudaStreamSynchronize(c->st));
  if (!c->pending.empty()) prof_resolve(c);
  return FASW_OK;
}

}  // namespace

extern "C" {

void fasw_default_params(fasw_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->scheme = FASW_AW3;
  p->nlevels = 3;
  p->gamma_cycle = 1;
  p->nu1 = 1;
  p->viscous = 0;
  p->turb = 0;
  p->sensor = 0;
  p->mach = 0.8;
  p->alpha_deg = 0.0;
  p->re = 1e6;
  p->pr = 0.75;
  p->prt = 0.9;
  p->eta = 0.8;
  p->d_cut = 0.5;
  p->cfl = 1e4;
  p->cfl_ramp = 20.0;
  p->ramp_cycles = 2;
  p->s_coarse = 0.25;
  p->precision = FASW_FP64;
  p->norm_all = 0;
  p->spin_limit = 0;
}

int fasw_create(int ni, int nj, int n_wake, const double* x, const double* y, int coords_on_device,
                const fasw_params* p, void* stream, fasw_ctx** out) {
  if (!out || !x || !y || !p) return FASW_ERR_ARG;
  *out = nullptr;
  if (ni < 4 || nj < 2 || n_wake < 0 || 2 * n_wake >= ni || p->nlevels < 1 || p->nlevels > 12) return FASW_ERR_ARG;
  if (p->scheme < 0 || p->scheme > 7 || p->gamma_cycle < 1 || p->gamma_cycle > 2 || p->nu1 < 1) return FASW_ERR_ARG;
  const int f = 1 << (p->nlevels - 1);
  if (ni % f || nj % f || n_wake % f || ni / f < 4 || nj / f < 2) return FASW_ERR_ARG;
  if (!(p->mach > 0.0) || (p->viscous && !(p->re > 0.0))) return FASW_ERR_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  fasw_ctx* c = new (std::nothrow) fasw_ctx();
  if (!c) return FASW_ERR_OOM;
  c->prm = *p;
  c->st = static_cast<cudaStream_t>(stream);
  c->mixed = p->precision == FASW_MIXED ? 1 : 0;
  c->ph.mach = p->mach;
  c->ph.alpha_deg = p->alpha_deg;
  c->ph.re = p->re;
  c->ph.pr = p->pr;
  c->ph.prt = p->prt;
  c->ph.inv_re = p->re > 0.0 ? 1.0 / p->re : 0.0;
  c->ph.inv_pr = p->pr > 0.0 ? 1.0 / p->pr : 0.0;
  c->ph.inv_prt = p->prt > 0.0 ? 1.0 / p->prt : 0.0;
  c->ph.s_coarse = p->s_coarse;
  c->ph.viscous = p->viscous;
  c->ph.turb = p->turb;
  c->ph.sensor = p->sensor;
  free_stream(p->mach, p->alpha_deg, c->ph.uinf);
  const Coef& cf = kCoef[p->scheme % 4];
  c->sc.aw = p->scheme < 4 ? 1 : 0;
  c->sc.nstages = cf.s;
  for (int k = 0; k < 5; ++k) {
    c->sc.alpha[k] = cf.a[k];
    c->sc.beta[k] = cf.b[k];
  }
  c->sc.eta = p->eta;
  c->sc.d_cut = p->d_cut;
  const int nl = p->nlevels;
  c->lev.resize(nl);
  for (int l = nl - 1; l >= 0; --l) {
    LevelDev& L = c->lev[l];
    std::memset(&L, 0, sizeof(L));
    const int s = 1 << (nl - 1 - l);
    L.ni = ni / s;
    L.nj = nj / s;
    L.nw = n_wake / s;
    L.P = L.ni + 4;
    L.Gn = L.P * (L.nj + 4);
    L.n = L.ni * L.nj;
    L.nfx = (L.ni + 1) * L.nj;
    L.nfe = L.ni * (L.nj + 1);
    L.finest = l == nl - 1 ? 1 : 0;
    L.a_t = 0.0;
    int r = alloc_level(c, L);
    if (r != FASW_OK) {
      fasw_destroy(c);
      return r;
    }
  }
  int r = FASW_OK;
  if ((r = dalloc(c, &c->d_norm, 1)) != FASW_OK || (r = dalloc(c, &c->d_tmp, 4 * (size_t)ni * nj)) != FASW_OK ||
      (r = dalloc(c, &c->d_tmp2, 4 * (size_t)ni * nj)) != FASW_OK ||
      (r = dalloc(c, &c->d_tmp3, 32 * (size_t)(ni + 1) * (nj + 1))) != FASW_OK) {
    fasw_destroy(c);
    return r;
  }
  e = cudaMallocHost(&c->h_norm, sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(int));
  if (e != cudaSuccess) {
    fasw_destroy(c);
    return cuda_fail(e);
  }
  *c->h_err = 0;
  if (p->spin_limit > 0) c->spin_limit = p->spin_limit;
  {
    const int nstrips = (nj + 3) / 4 + 1;  // strips of 4 rows at most
    if ((r = dalloc(c, &c->d_prog, 2 * (size_t)nstrips)) != FASW_OK || (r = dalloc(c, &c->d_err, 1)) != FASW_OK) {
      fasw_destroy(c);
      return r;
    }
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    cudaMemsetAsync(c->d_prog, 0, 2 * (size_t)nstrips * sizeof(long long), c->st);
  }
  // metrics on the finest level from the vertices, coarse levels by agglomeration
  const size_t nv = (size_t)(ni + 1) * (nj + 1);
  double *dx = nullptr, *dy = nullptr;
  if ((r = dalloc(c, &dx, nv)) != FASW_OK || (r = dalloc(c, &dy, nv)) != FASW_OK ||
      (r = dalloc(c, &c->d_un, 4 * (size_t)ni * nj)) != FASW_OK ||
      (r = dalloc(c, &c->d_unm1, 4 * (size_t)ni * nj)) != FASW_OK) {
    fasw_destroy(c);
    return r;
  }
  const cudaMemcpyKind kind = coords_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(dx, x, nv * sizeof(double), kind, c->st);
  cudaMemcpyAsync(dy, y, nv * sizeof(double), kind, c->st);
  c->d_x0 = dx;
  c->d_y0 = dy;
  launch_metrics_fine(c->lev[nl - 1], dx, dy, c->st);
  for (int l = nl - 2; l >= 0; --l) launch_agglomerate(c->lev[l + 1], c->lev[l], c->st);
  for (int l = 0; l < nl; ++l) launch_fill_state(c->lev[l], c->ph.uinf, c->st);
  c->launches += 2 * nl;
  if ((r = sync(c)) != FASW_OK) {
    fasw_destroy(c);
    return r;
  }
  *out = c;
  return FASW_OK;
}

void fasw_destroy(fasw_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  drop_graphs(c);
  for (auto& q : c->pending) {
    c->event_pool.push_back(q.a);
    c->event_pool.push_back(q.b);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  for (void* q : c->allocs) cudaFree(q);
  if (c->h_norm) cudaFreeHost(c->h_norm);
  if (c->h_err) cudaFreeHost(c->h_err);
  adj_release(c->adj);
  delete c;
}

int fasw_level_dims(fasw_ctx* c, int l, int* ni, int* nj, int* nw) {
  if (check_level(c, l)) return FASW_ERR_ARG;
  if (ni) *ni = c->lev[l].ni;
  if (nj) *nj = c->lev[l].nj;
  if (nw) *nw = c->lev[l].nw;
  return FASW_OK;
}

int fasw_set_state(fasw_ctx* c, int l, const double* u, int on_device) {
  if (check_level(c, l) || !u) return FASW_ERR_ARG;
  LevelDev& L = c->lev[l];
  int r = copy_in(c, c->d_tmp, u, 4 * (size_t)L.n, on_device);
  if (r) return r;
  launch_pack(L, c->d_tmp, 1, nullptr, c->st);
  launch_bc(L, c->ph, c->st);
  c->launches += 2;
  return sync(c);
}

int fasw_get_state(fasw_ctx* c, int l, double* u, int on_device) {
  if (check_level(c, l) || !u) return FASW_ERR_ARG;
  LevelDev& L = c->lev[l];
  launch_pack(L, nullptr, 0, c->d_tmp, c->st);
  ++c->launches;
  int r = copy_out(c, u, c->d_tmp, 4 * (size_t)L.n, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_set_forcing(fasw_ctx* c, int l, const double* s, int on_device) {
  if (check_level(c, l) || !s) return FASW_ERR_ARG;
  int r = copy_in(c, c->lev[l].s, s, 4 * (size_t)c->lev[l].n, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_get_forcing(fasw_ctx* c, int l, double* s, int on_device) {
  if (check_level(c, l) || !s) return FASW_ERR_ARG;
  int r = copy_out(c, s, c->lev[l].s, 4 * (size_t)c->lev[l].n, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_residual(fasw_ctx* c, int l, double* F, double* Fc, double* Fv, int on_device, double* norm) {
  if (check_level(c, l)) return FASW_ERR_ARG;
  LevelDev& L = c->lev[l];
  const size_t m = 4 * (size_t)L.n;
  bc_aux(c, l, 1.0, 0);
  ResArgs a{};
  a.mode = RES_FULL;
  a.want_norm = norm ? 1 : 0;
  a.norm_all = c->prm.norm_all;
  a.F = F ? (on_device ? F : c->d_tmp) : nullptr;
  a.Fc = Fc ? (on_device ? Fc : c->d_tmp2) : nullptr;
  a.Fv = Fv ? (on_device ? Fv : L.rhs) : nullptr;
  launch_residual(L, c->ph, a, c->st);
  ++c->launches;
  if (norm) {
    launch_norm_final(L, residual_blocks(L), L.n * (c->prm.norm_all ? 4 : 1), c->d_norm, c->st);
    ++c->launches;
    CKR(cudaMemcpyAsync(c->h_norm, c->d_norm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  if (!on_device) {
    if (F) CKR(cudaMemcpyAsync(F, c->d_tmp, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (Fc) CKR(cudaMemcpyAsync(Fc, c->d_tmp2, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (Fv) CKR(cudaMemcpyAsync(Fv, L.rhs, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  int r = sync(c);
  if (r) return r;
  if (norm) *norm = *c->h_norm;
  return FASW_OK;
}

int fasw_pseudo_dt(fasw_ctx* c, int l, double cfl, double* dts, int on_device) {
  if (check_level(c, l) || !dts) return FASW_ERR_ARG;
  bc_aux(c, l, cfl, 1);
  int r = copy_out(c, dts, c->lev[l].dts, (size_t)c->lev[l].n, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_precond_apply(fasw_ctx* c, int l, double cfl, const double* rin, double* z, int on_device) {
  if (check_level(c, l) || !rin || !z) return FASW_ERR_ARG;
  LevelDev& L = c->lev[l];
  const size_t m = 4 * (size_t)L.n;
  bc_aux(c, l, cfl, 1);
  launch_face_blocks(L, c->ph, c->sc, c->mixed, c->st);
  launch_diag_blocks(L, c->sc, c->mixed, c->st);
  c->launches += 2;
  int r = copy_in(c, c->d_tmp2, rin, m, on_device);
  if (r) return r;
  if (c->sweep_kind != SWEEP_LEGACY) {
    launch_sgs_prep(L, c->mixed, level_sweep_kind(c, L), c->st);
    ++c->launches;
  }
  run_sweep(c, L, 0, 0.0, c->d_tmp2);
  const double* zsrc = L.yz64;
  if (c->mixed) {
    launch_f2d(L.yz32, c->d_tmp, (int)m, c->st);
    ++c->launches;
    zsrc = c->d_tmp;
  }
  r = copy_out(c, z, zsrc, m, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_face_blocks(fasw_ctx* c, int l, double* axp, double* axm, double* aep, double* aem, int on_device) {
  if (check_level(c, l)) return FASW_ERR_ARG;
  LevelDev& L = c->lev[l];
  bc_aux(c, l, 1.0, 1);
  launch_face_blocks(L, c->ph, c->sc, 0, c->st);
  ++c->launches;
  double* outs[4] = {axp, axm, aep, aem};
  const size_t offs[4] = {0, 16 * (size_t)L.nfx, 32 * (size_t)L.nfx, 32 * (size_t)L.nfx + 16 * (size_t)L.nfe};
  const int nfs[4] = {L.nfx, L.nfx, L.nfe, L.nfe};
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    launch_blocks_transpose(L.blk64 + offs[k], c->d_tmp3, nfs[k], c->st);
    ++c->launches;
    int r = copy_out(c, outs[k], c->d_tmp3, 16 * (size_t)nfs[k], on_device);
    if (r) return r;
    if ((r = sync(c)) != FASW_OK) return r;
  }
  return sync(c);
}

int fasw_smooth(fasw_ctx* c, int l, int nsteps, double cfl) {
  if (check_level(c, l) || nsteps < 0) return FASW_ERR_ARG;
  for (int k = 0; k < nsteps; ++k) smooth_step(c, l, cfl, false);
  return sync(c);
}

static void enqueue_cycle(fasw_ctx* c, double cfl) {
  const int Lf = c->L();
  if (c->prm.turb) {
    bc_aux(c, Lf, cfl, 0);
    { Prof p(c, FASW_K_BL); launch_bl(c->lev[Lf], c->ph, c->st); }
    c->launches += 2;
  }
  fas_cycle_rec(c, Lf, cfl, true);
  cudaMemcpyAsync(c->h_norm, c->d_norm, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
}

// The launch sequence of a cycle depends only on c*, so each distinct c* is captured once
// into a CUDA graph and replayed (no per-kernel launch overhead).  Not used while profiling
// or on the legacy default stream, where capture is not possible.
static int run_cycle(fasw_ctx* c, double cfl) {
  if (!c->use_graphs || c->profiling || c->st == nullptr) {
    enqueue_cycle(c, cfl);
    return FASW_OK;
  }
  for (auto& g : c->graphs)
    if (g.cfl == cfl) {
      CKR(cudaGraphLaunch(g.exec, c->st));
      c->launches += g.kernels;
      return FASW_OK;
    }
  const long long before = c->launches;
  CKR(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  enqueue_cycle(c, cfl);
  cudaGraph_t graph = nullptr;
  CKR(cudaStreamEndCapture(c->st, &graph));
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  const long long k = c->launches - before;
  c->graphs.push_back({cfl, exec, k});
  CKR(cudaGraphLaunch(exec, c->st));
  return FASW_OK;
}

int fasw_fas_cycle(fasw_ctx* c, int cycle_index, double* res_norm) {
  if (!c) return FASW_ERR_ARG;
  const double cfl = cycle_index < c->prm.ramp_cycles ? std::fmin(c->prm.cfl, c->prm.cfl_ramp) : c->prm.cfl;
  int r = run_cycle(c, cfl);
  if (r) return r;
  r = sync(c);
  if (r) return r;
  if (*c->h_err) return FASW_ERR_DEVICE_TIMEOUT;
  if (res_norm) *res_norm = *c->h_norm;
  return FASW_OK;
}

// ---- discrete adjoint (steady finest level, eddy viscosity frozen)
static int adj_ready(fasw_ctx* c) {
  if (c->adj.n) return FASW_OK;
  const LevelDev& F = c->lev[c->L()];
  c->adj.fp32 = c->mixed != 0;
  c->adj.prog = c->d_prog;
  c->adj.err = c->d_err;
  c->adj.spin_limit = c->spin_limit;
  return adj_setup(c->adj, F.ni, F.nj, F.nw, c->allocs, c->st);
}

// The finest level's Jacobian and, for the transposed FAS cycle, those of the coarse levels at
// the restricted state.
static int adj_assemble_all(fasw_ctx* c, double h_rel) {
  int r = adj_assemble(c->adj, c->lev[c->L()], c->ph, h_rel, c->st, c->launches);
  if (r) return r;
  const int kind = c->adj.precond_kind;
  if ((kind == ADJ_FAS_CYCLE_T || kind == ADJ_FAS_VCYCLE_T) && c->L() > 0) {
    const int gamma = kind == ADJ_FAS_VCYCLE_T ? 1 : c->prm.gamma_cycle;
    if ((r = adj_mg_setup(c->adj, c->lev, gamma, c->prm.nu1, c->allocs, c->st))) return r;
    if ((r = adj_mg_assemble(c->adj, c->lev, c->ph, c->prm.turb, h_rel, c->st, c->launches))) return r;
  }
  return FASW_OK;
}

// FASW_ERR_DEVICE_TIMEOUT when a bounded wait of the sweeps ran out (device error word set).
static int adj_err_check(fasw_ctx* c) {
  CKR(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CKR(cudaStreamSynchronize(c->st));
  return *c->h_err ? FASW_ERR_DEVICE_TIMEOUT : FASW_OK;
}

int fasw_force_coefficients(fasw_ctx* c, double* cl, double* cd) {
  if (!c || !cl || !cd) return FASW_ERR_ARG;
  int r = adj_ready(c);
  if (r) return r;
  return adj_force_coefficients(c->adj, c->lev[c->L()], c->ph, c->st, cl, cd, c->launches);
}

int fasw_adjoint_jacobian(fasw_ctx* c, double h_rel) {
  if (!c || !(h_rel > 0.0) || c->ph.moving || c->lev[c->L()].a_t != 0.0) return FASW_ERR_ARG;
  int r = adj_ready(c);
  if (r) return r;
  r = adj_assemble_all(c, h_rel);
  if (r) return r;
  return sync(c);
}

int fasw_adjoint_apply(fasw_ctx* c, const double* v, double* out, int transpose, int on_device) {
  if (!c || !v || !out || !c->adj.built) return FASW_ERR_ARG;
  const size_t m = 4 * (size_t)c->adj.n;
  int r = copy_in(c, c->d_tmp, v, m, on_device);
  if (r) return r;
  adj_apply(c->adj, c->d_tmp, c->d_tmp2, transpose, c->st);
  ++c->launches;
  r = copy_out(c, out, c->d_tmp2, m, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_adjoint_objective_gradient(fasw_ctx* c, int which, double* g, int on_device) {
  if (!c || !g || which < 0 || which > 1 || !c->adj.built) return FASW_ERR_ARG;
  const size_t m = 4 * (size_t)c->adj.n;
  int r = copy_out(c, g, c->adj.g + which * m, m, on_device);
  if (r) return r;
  return sync(c);
}

int fasw_adjoint_precond_apply(fasw_ctx* c, double cfl, int steps, const double* r, double* z, int on_device) {
  if (!c || !r || !z || !(cfl > 0.0) || steps < 0 || c->ph.moving) return FASW_ERR_ARG;
  if (steps > 0 && !c->adj.built) return FASW_ERR_ARG;
  int e = adj_ready(c);
  if (e) return e;
  const size_t m = 4 * (size_t)c->adj.n;
  if ((e = copy_in(c, c->d_tmp, r, m, on_device))) return e;
  adj_build_precond(c->adj, c->lev[c->L()], c->ph, c->sc, cfl, c->st, c->launches);
  adj_steps_apply(c->adj, steps, c->d_tmp, c->d_tmp2, c->st);
  c->launches += 2;
  if ((e = adj_err_check(c))) return e;
  if ((e = copy_out(c, z, c->d_tmp2, m, on_device))) return e;
  return sync(c);
}

int fasw_adjoint_set_precond_steps(fasw_ctx* c, int steps) {
  if (!c || steps < 1 || steps > 16) return FASW_ERR_ARG;
  c->adj.smooth_steps = steps;
  return FASW_OK;
}

int fasw_adjoint_set_precond(fasw_ctx* c, int kind) {
  if (!c || kind < ADJ_STAGE_LOOP || kind > ADJ_FAS_VCYCLE_T) return FASW_ERR_ARG;
  if (kind != c->adj.precond_kind) c->adj.built = false;  // the cycle needs the coarse Jacobians
  c->adj.precond_kind = kind;
  return FASW_OK;
}

int fasw_adjoint_cycle_apply(fasw_ctx* c, double cfl, int kind, int transpose, const double* r, double* z,
                             int on_device) {
  if (!c || !r || !z || !(cfl > 0.0) || (kind != 1 && kind != 2) || !c->adj.built) return FASW_ERR_ARG;
  if (kind == 2 && c->L() > 0 && !c->adj.mg) return FASW_ERR_ARG;
  const size_t m = 4 * (size_t)c->adj.n;
  int e = copy_in(c, c->d_tmp, r, m, on_device);
  if (e) return e;
  adj_build_precond(c->adj, c->lev[c->L()], c->ph, c->sc, cfl, c->st, c->launches);
  if (kind == 2) {
    adj_mg_build_precond(c->adj, c->lev, c->ph, c->sc, cfl, c->st, c->launches);
    adj_mg_apply(c->adj, transpose, c->d_tmp, c->d_tmp2, c->st);
  } else {
    adj_smoother_apply(c->adj, c->adj.smooth_steps, transpose, c->d_tmp, c->d_tmp2, c->st);
  }
  ++c->launches;
  if ((e = adj_err_check(c))) return e;
  if ((e = copy_out(c, z, c->d_tmp2, m, on_device))) return e;
  return sync(c);
}

int fasw_adjoint_solve(fasw_ctx* c, int which, const double* g, double* lam, double tol, int max_iters, int restart,
                       double cfl, int* iters, double* rel_res, int on_device) {
  if (!c || !lam || !iters || !rel_res || !c->adj.built || !(tol > 0.0) || max_iters < 1) return FASW_ERR_ARG;
  if (!g && (which < 0 || which > 1)) return FASW_ERR_ARG;
  const size_t m = 4 * (size_t)c->adj.n;
  const double* rhs = c->adj.g + (which < 0 ? 0 : which) * m;
  if (g) {
    int r = copy_in(c, c->d_tmp, g, m, on_device);
    if (r) return r;
    rhs = c->d_tmp;
  }
  const double pcfl = cfl > 0.0 ? cfl : c->prm.cfl;
  const int code = adj_solve(c->adj, c->lev, c->ph, c->sc, pcfl, rhs, c->d_tmp2, tol, max_iters, restart,
                             c->allocs, c->st, iters, rel_res, c->launches);
  if (code != FASW_OK && code != FASW_ERR_NOT_CONVERGED) return code;
  int r = adj_err_check(c);
  if (r) return r;
  r = copy_out(c, lam, c->d_tmp2, m, on_device);
  if (r) return r;
  r = sync(c);
  return r ? r : code;
}

}  // extern "C"

namespace {

// For one vertex field vk (device, (nj+1) x (ni+1) y-displacements of the grid at rest):
// *dC = C(X + h vk) - C(X - h vk) of objective `which` and *dot = lam . (F(X + h vk) - F(X - h vk))
// at the current state, the grid rotated by (phi, phidot) about (xc, yc) when rotate != 0.
// F leaves out the time term (it does not depend on X).  The caller restores the metrics.
int shape_term(fasw_ctx* c, int which, const double* d_lam, const double* vk, double h_x, int rotate, double phi,
               double phidot, double xc, double yc, double* dC, double* dot) {
  LevelDev F = c->lev[c->L()];
  F.a_t = 0.0;
  const size_t m = 4 * (size_t)F.n, nv = (size_t)(F.ni + 1) * (F.nj + 1);
  double* ytmp = c->d_tmp3;
  ResArgs a{};
  a.mode = RES_FULL;
  double cl[2], cd[2];
  for (int sgn = 0; sgn < 2; ++sgn) {
    adj_lincomb((int)nv, c->d_y0, sgn == 0 ? h_x : -h_x, vk, ytmp, c->st);
    launch_metrics_fine(F, c->d_x0, ytmp, c->st, rotate, phi, phidot, xc, yc);
    launch_bc_aux(F, c->ph, 1.0, 0, c->st);
    a.F = sgn == 0 ? c->adj.Fp : c->adj.Fm;
    launch_residual(F, c->ph, a, c->st);
    c->launches += 4;
    int r = adj_force_coefficients(c->adj, F, c->ph, c->st, &cl[sgn], &cd[sgn], c->launches);
    if (r) return r;
  }
  adj_lincomb((int)m, c->adj.Fp, -1.0, c->adj.Fm, c->d_tmp2, c->st);  // F+ - F-
  *dC = which == 0 ? cl[0] - cl[1] : cd[0] - cd[1];
  return adj_dot(c->adj, d_lam, c->d_tmp2, (int)m, c->st, dot);
}

}  // namespace

extern "C" {

int fasw_adjoint_shape_gradient(fasw_ctx* c, int which, const double* lam, int nparam, const double* vy, double h_x,
                                double* grad, int on_device) {
  if (!c || !lam || !vy || !grad || nparam < 1 || which < 0 || which > 1 || !(h_x > 0.0) || c->ph.moving)
    return FASW_ERR_ARG;
  int r = adj_ready(c);
  if (r) return r;
  LevelDev& F = c->lev[c->L()];
  const size_t m = 4 * (size_t)F.n, nv = (size_t)(F.ni + 1) * (F.nj + 1);
  if ((r = copy_in(c, c->d_tmp, lam, m, on_device))) return r;
  double* vk = c->d_tmp3 + nv;
  for (int k = 0; k < nparam; ++k) {
    if ((r = copy_in(c, vk, vy + (size_t)k * nv, nv, on_device))) return r;
    double dJ = 0.0, dot = 0.0;
    if ((r = shape_term(c, which, c->d_tmp, vk, h_x, 0, 0.0, 0.0, 0.0, 0.0, &dJ, &dot))) return r;
    grad[k] = (dJ - dot) / (2.0 * h_x);
  }
  launch_metrics_fine(F, c->d_x0, c->d_y0, c->st);
  launch_bc_aux(F, c->ph, 1.0, 0, c->st);
  c->launches += 2;
  return sync(c);
}

}  // extern "C"

namespace {

// (a_n, b_n, c_n) of F^n = R/vol + a_n u^n + b_n u^(n-1) + c_n u^(n-2): implicit Euler for
// the first step, BDF2 after (section 6), as fasw_dual_time_step takes them.
void time_coefficients(int n, double dt, int bdf_order, double* a, double* b, double* cc) {
  if (n <= 1 || bdf_order == 1) {
    *a = 1.0 / dt, *b = -1.0 / dt, *cc = 0.0;
  } else {
    *a = 1.5 / dt, *b = -2.0 / dt, *cc = 0.5 / dt;
  }
}

// Device buffers of one unsteady adjoint run, freed on every return.
struct RunBuffers {
  std::vector<void*> mem;
  ~RunBuffers() {
    for (void* p : mem) cudaFree(p);
  }
  int get(double** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(double));
    if (e != cudaSuccess) {
      g_last_cuda_error = cudaGetErrorString(e);
      return FASW_ERR_OOM;
    }
    mem.push_back(q);
    *p = static_cast<double*>(q);
    return FASW_OK;
  }
};

// Puts the context back to u0 on the grid at rest with no time term.
void unsteady_reset(fasw_ctx* c, const double* u0) {
  LevelDev& F = c->lev[c->L()];
  if (c->ph.moving) drop_graphs(c);
  c->ph.moving = 0;
  const int nl = (int)c->lev.size();
  launch_metrics_fine(F, c->d_x0, c->d_y0, c->st);
  for (int l = nl - 2; l >= 0; --l) launch_agglomerate(c->lev[l + 1], c->lev[l], c->st);
  if (F.a_t != 0.0) drop_graphs(c);
  for (auto& L : c->lev) L.a_t = 0.0;
  cudaMemsetAsync(F.src, 0, 4 * (size_t)F.n * sizeof(double), c->st);
  if (u0) {
    launch_pack(F, u0, 1, nullptr, c->st);
    launch_bc(F, c->ph, c->st);
  }
  c->launches += nl + (u0 ? 2 : 0);
  c->steps_done = 0;
  c->adj.built = false;
}

}  // namespace

extern "C" {

int fasw_unsteady_adjoint(fasw_ctx* c, double amp, double omega, double xc, double yc, double dt, int nsteps,
                          int bdf_order, double drop, int max_cycles, int snapshots, int which, int nparam,
                          const double* vy, double h_rel, double h_x, double tol, int max_iters, int restart,
                          double cfl, double* objective, double* grad, double* g0, int on_device, double* stats) {
  if (!c || !objective || !(dt > 0.0) || nsteps < 1 || (bdf_order != 1 && bdf_order != 2) || max_cycles < 1 ||
      snapshots < 0 || which < 0 || which > 1 || nparam < 0 || (nparam > 0 && (!vy || !grad)) || !(h_rel > 0.0) ||
      !(h_x > 0.0) || !(tol > 0.0) || max_iters < 1 || restart < 1 || c->ph.moving || c->steps_done != 0 ||
      c->lev[c->L()].a_t != 0.0)
    return FASW_ERR_ARG;
  std::vector<CkAction> plan;
  long long fsteps = 0;
  int r = checkpoint_schedule(nsteps, snapshots, plan, &fsteps);
  if (r) return r;
  if ((r = adj_ready(c))) return r;
  if ((r = sync(c))) return r;
  LevelDev& F = c->lev[c->L()];
  const size_t m = 4 * (size_t)F.n, nv = (size_t)(F.ni + 1) * (F.nj + 1);
  const int S = std::min(snapshots, nsteps - 1);
  RunBuffers buf;
  double *u0 = nullptr, *slots = nullptr, *lam = nullptr, *rhs = nullptr, *V = nullptr;
  if ((r = buf.get(&u0, m)) || (r = buf.get(&slots, 2 * m * (size_t)std::max(S, 1))) || (r = buf.get(&lam, 3 * m)) ||
      (r = buf.get(&rhs, m)) || (r = buf.get(&V, nv * (size_t)std::max(nparam, 1))))
    return r;
  if (nparam > 0 && (r = copy_in(c, V, vy, nv * (size_t)nparam, on_device))) return r;
  launch_pack(F, nullptr, 0, u0, c->st);
  cudaMemsetAsync(lam, 0, 3 * m * sizeof(double), c->st);
  ++c->launches;
  double* lam1 = lam;          // lam^(n+1)
  double* lam2 = lam + m;      // lam^(n+2)
  double* lamn = lam + 2 * m;  // lam^n
  std::vector<int> slot_of(nsteps + 1, -1);
  std::vector<int> free_slots;
  for (int k = S - 1; k >= 0; --k) free_slots.push_back(k);
  const double w = 1.0 / nsteps;
  const double pcfl = cfl > 0.0 ? cfl : c->prm.cfl;
  std::vector<double> gacc(nparam, 0.0);
  double J = 0.0, worst = 0.0;
  long long gm_iters = 0, cycles = 0;
  int pos = 0, reached = 0;
  bool soft = false;
  auto motion = [&](int n) {
    const double t = n * dt;
    return fasw_set_motion(c, -amp * std::sin(omega * t), -amp * omega * std::cos(omega * t), xc, yc);
  };
  auto fail = [&](int code) {
    unsteady_reset(c, u0);
    sync(c);
    return code;
  };
  for (const CkAction& act : plan) {
    if (act.op == CK_ADVANCE) {
      for (int n = pos + 1; n <= act.arg; ++n) {
        if ((r = motion(n))) return fail(r);
        int nc = 0;
        r = fasw_dual_time_step(c, dt, bdf_order, drop, max_cycles, nullptr, &nc);
        cycles += nc;
        if (r == FASW_ERR_NOT_CONVERGED) soft = true;
        else if (r) return fail(r);
        if (n > reached) {  // the first sweep: the objective
          double cl = 0.0, cd = 0.0;
          if ((r = adj_force_coefficients(c->adj, F, c->ph, c->st, &cl, &cd, c->launches))) return fail(r);
          J += w * (which == 0 ? cl : cd);
          reached = n;
        }
      }
      pos = act.arg;
    } else if (act.op == CK_STORE) {
      if (free_slots.empty() || act.arg < 1 || act.arg > nsteps) return fail(FASW_ERR_ARG);  // not a valid plan
      const int k = free_slots.back();
      free_slots.pop_back();
      slot_of[act.arg] = k;
      double* s = slots + 2 * m * (size_t)k;
      cudaMemcpyAsync(s, c->d_un, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(s + m, c->d_unm1, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    } else if (act.op == CK_FREE) {
      if (act.arg < 1 || act.arg > nsteps || slot_of[act.arg] < 0) return fail(FASW_ERR_ARG);
      free_slots.push_back(slot_of[act.arg]);
      slot_of[act.arg] = -1;
    } else if (act.op == CK_RESTORE) {
      if (act.arg == 0) {
        launch_pack(F, u0, 1, nullptr, c->st);
        c->steps_done = 0;
      } else {
        if (act.arg < 1 || act.arg > nsteps || slot_of[act.arg] < 0) return fail(FASW_ERR_ARG);
        const double* s = slots + 2 * m * (size_t)slot_of[act.arg];
        launch_pack(F, s, 1, nullptr, c->st);
        cudaMemcpyAsync(c->d_un, s, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->d_unm1, s + m, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        c->steps_done = act.arg;
      }
      launch_bc(F, c->ph, c->st);
      c->launches += 2;
      pos = act.arg;
    } else {  // CK_CONSUME: adjoint step of level n = pos
      const int n = act.arg;
      if (n != pos || n < 1) return fail(FASW_ERR_ARG);
      double a_n, b_n, c_n, a1, b1, c1, a2, b2, c2;
      time_coefficients(n, dt, bdf_order, &a_n, &b_n, &c_n);
      time_coefficients(n + 1, dt, bdf_order, &a1, &b1, &c1);
      time_coefficients(n + 2, dt, bdf_order, &a2, &b2, &c2);
      if ((r = motion(n))) return fail(r);
      if (F.a_t != a_n) {
        drop_graphs(c);
        for (auto& L : c->lev) L.a_t = a_n;
      }
      cudaMemsetAsync(F.src, 0, m * sizeof(double), c->st);
      if (c->prm.turb) {  // eddy viscosity frozen at its value for u^n
        launch_bc_aux(F, c->ph, 1.0, 0, c->st);
        launch_bl(F, c->ph, c->st);
        c->launches += 2;
      }
      if ((r = adj_assemble_all(c, h_rel))) return fail(r);
      cudaMemsetAsync(rhs, 0, m * sizeof(double), c->st);
      adj_axpby((int)m, w, c->adj.g + (size_t)which * m, 1.0, rhs, c->st);
      if (n + 1 <= nsteps) adj_axpby((int)m, -b1, lam1, 1.0, rhs, c->st);
      if (n + 2 <= nsteps) adj_axpby((int)m, -c2, lam2, 1.0, rhs, c->st);
      c->launches += 1 + (n + 1 <= nsteps) + (n + 2 <= nsteps);
      int it = 0;
      double rr = 0.0;
      r = adj_solve(c->adj, c->lev, c->ph, c->sc, pcfl, rhs, lamn, tol, max_iters, restart, c->allocs, c->st, &it, &rr,
                    c->launches);
      if (r == FASW_ERR_NOT_CONVERGED) soft = true;
      else if (r) return fail(r);
      if ((r = adj_err_check(c))) return fail(r);
      gm_iters += it;
      worst = std::max(worst, rr);
      const double t = n * dt;
      const double phi = -amp * std::sin(omega * t), phidot = -amp * omega * std::cos(omega * t);
      for (int k = 0; k < nparam; ++k) {
        double dC = 0.0, dot = 0.0;
        if ((r = shape_term(c, which, lamn, V + nv * (size_t)k, h_x, 1, phi, phidot, xc, yc, &dC, &dot)))
          return fail(r);
        gacc[k] += (w * dC - dot) / (2.0 * h_x);
      }
      launch_metrics_fine(F, c->d_x0, c->d_y0, c->st, 1, phi, phidot, xc, yc);
      ++c->launches;
      // rotate: lam^(n+2) <- lam^(n+1) <- lam^n
      double* old2 = lam2;
      lam2 = lam1;
      lam1 = lamn;
      lamn = old2;
    }
  }
  // dJ/du^0 = -(b_1 lam^1 + c_2 lam^2): lam1 holds lam^1, lam2 holds lam^2 (zero when N = 1)
  double a_1, b_1, c_1, a_2, b_2, c_2;
  time_coefficients(1, dt, bdf_order, &a_1, &b_1, &c_1);
  time_coefficients(2, dt, bdf_order, &a_2, &b_2, &c_2);
  cudaMemsetAsync(rhs, 0, m * sizeof(double), c->st);
  adj_axpby((int)m, -b_1, lam1, 1.0, rhs, c->st);
  if (nsteps >= 2) adj_axpby((int)m, -c_2, lam2, 1.0, rhs, c->st);
  c->launches += 1 + (nsteps >= 2);
  if (g0 && (r = copy_out(c, g0, rhs, m, on_device))) return fail(r);
  unsteady_reset(c, u0);
  if ((r = sync(c))) return r;
  *objective = J;
  for (int k = 0; k < nparam; ++k) grad[k] = gacc[k];
  if (stats) {
    stats[0] = (double)fsteps;
    stats[1] = (double)(fsteps - nsteps);
    stats[2] = (double)gm_iters;
    stats[3] = (double)cycles;
    stats[4] = worst;
  }
  return soft ? FASW_ERR_NOT_CONVERGED : FASW_OK;
}

}  // extern "C"

extern "C" {

int fasw_adjoint_vertex_gradient(fasw_ctx* c, int which, const double* lam, double h_x, double* gx, double* gy,
                                 int on_device) {
  if (!c || !lam || !gx || !gy || which < 0 || which > 1 || !(h_x > 0.0) || c->ph.moving) return FASW_ERR_ARG;
  int r = adj_ready(c);
  if (r) return r;
  LevelDev& F = c->lev[c->L()];
  AdjointDev& A = c->adj;
  if ((r = adj_vertex_setup(A, F.nw, c->allocs, c->st))) return r;
  adj_vertex_lengths(A, c->d_x0, c->d_y0, c->st);
  ++c->launches;
  const size_t m = 4 * (size_t)F.n, nv = (size_t)(F.ni + 1) * (F.nj + 1);
  if ((r = copy_in(c, c->d_tmp, lam, m, on_device))) return r;
  double* xo = A.vx;
  double* yo = A.vx + nv;
  double* g = c->d_tmp3;  // gx, then gy
  LevelDev Fz = F;
  Fz.a_t = 0.0;  // the time term does not depend on X
  ResArgs a{};
  a.mode = RES_FULL;
  const double al = c->ph.alpha_deg * M_PI / 180.0, sa = std::sin(al), ca = std::cos(al);
  for (int k = 0; k < A.nvcolours; ++k)
    for (int dir = 0; dir < 2; ++dir) {
      for (int sgn = 0; sgn < 2; ++sgn) {
        adj_vertex_perturb(A, k, dir, sgn == 0 ? h_x : -h_x, c->d_x0, c->d_y0, xo, yo, c->st);
        launch_metrics_fine(Fz, xo, yo, c->st);
        launch_bc_aux(Fz, c->ph, 1.0, 0, c->st);
        a.F = sgn == 0 ? A.Fp : A.Fm;
        launch_residual(Fz, c->ph, a, c->st);
        launch_wall_force(Fz, c->ph, A.fw + 2 * sgn * A.ni, A.fw + (2 * sgn + 1) * A.ni, c->st);
        c->launches += 5;
      }
      adj_vertex_accumulate(A, k, which, sa, ca, c->d_tmp, A.Fp, A.Fm, A.fw, h_x, g + dir * nv, c->st);
      ++c->launches;
    }
  launch_metrics_fine(F, c->d_x0, c->d_y0, c->st);
  launch_bc_aux(F, c->ph, 1.0, 0, c->st);
  c->launches += 2;
  if ((r = copy_out(c, gx, g, nv, on_device)) || (r = copy_out(c, gy, g + nv, nv, on_device))) return r;
  return sync(c);
}

int fasw_set_sweep(fasw_ctx* c, int kind) {
  if (!c || kind < SWEEP_AUTO || kind > SWEEP_STRIPS4) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  c->sweep_kind = kind;
  drop_graphs(c);
  return FASW_OK;
}

int fasw_use_graphs(fasw_ctx* c, int enable) {
  if (!c) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  c->use_graphs = enable ? 1 : 0;
  if (!enable) drop_graphs(c);
  return FASW_OK;
}

int fasw_solve_steady(fasw_ctx* c, double drop, int max_cycles, double* history, int* ncycles) {
  if (!c || max_cycles < 1) return FASW_ERR_ARG;
  double n0 = 0.0;
  for (int k = 0; k < max_cycles; ++k) {
    double nk = 0.0;
    int r = fasw_fas_cycle(c, k, &nk);
    if (r) return r;
    if (history) history[k] = nk;
    if (k == 0) n0 = nk;
    if (ncycles) *ncycles = k + 1;
    if (!std::isfinite(nk) || (k > 0 && nk > 1e8 * n0)) return FASW_ERR_DIVERGED;
    if (k > 0 && nk <= drop * n0) return FASW_OK;
  }
  return FASW_ERR_NOT_CONVERGED;
}

int fasw_get_mut(fasw_ctx* c, double* mut, int on_device) {
  if (!c || !mut) return FASW_ERR_ARG;
  const int Lf = c->L();
  bc_aux(c, Lf, 1.0, 0);
  launch_bl(c->lev[Lf], c->ph, c->st);
  c->launches += 2;
  int r = copy_out(c, mut, c->lev[Lf].mut, (size_t)c->lev[Lf].n, on_device);
  if (r) return r;
  if (!c->prm.turb)  // a laminar context's residual must not see the eddy viscosity
    CKR(cudaMemsetAsync(c->lev[Lf].mut, 0, (size_t)c->lev[Lf].n * sizeof(double), c->st));
  return sync(c);
}

int fasw_set_time_source(fasw_ctx* c, double a_t, const double* src, int on_device) {
  if (!c || a_t < 0.0) return FASW_ERR_ARG;
  int r0 = sync(c);
  if (r0) return r0;
  drop_graphs(c);  // a_t is a by-value kernel argument baked into the captured cycles
  for (auto& L : c->lev) L.a_t = a_t;
  LevelDev& F = c->lev[c->L()];
  const size_t m = 4 * (size_t)F.n;
  if (src) {
    int r = copy_in(c, F.src, src, m, on_device);
    if (r) return r;
  } else {
    CKR(cudaMemsetAsync(F.src, 0, m * sizeof(double), c->st));
  }
  return sync(c);
}

long long fasw_launch_count(fasw_ctx* c) { return c ? c->launches : -1; }

int fasw_set_motion(fasw_ctx* c, double phi, double phidot, double xc, double yc) {
  if (!c) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  if (!c->ph.moving) drop_graphs(c);  // the moving-wall flag is a by-value kernel argument
  c->ph.moving = 1;
  const int nl = (int)c->lev.size();
  launch_metrics_fine(c->lev[nl - 1], c->d_x0, c->d_y0, c->st, 1, phi, phidot, xc, yc);
  for (int l = nl - 2; l >= 0; --l) launch_agglomerate(c->lev[l + 1], c->lev[l], c->st);
  c->launches += nl;
  return sync(c);
}

int fasw_dual_time_step(fasw_ctx* c, double dt, int bdf_order, double drop, int max_cycles, double* history,
                        int* ncycles) {
  if (!c || !(dt > 0.0) || (bdf_order != 1 && bdf_order != 2) || max_cycles < 1) return FASW_ERR_ARG;
  LevelDev& F = c->lev[c->L()];
  const int m = 4 * F.n;
  if (c->steps_done == 0) {  // the current state is u^n
    launch_pack(F, nullptr, 0, c->d_un, c->st);
    ++c->launches;
  }
  const bool bdf2 = c->steps_done > 0 && bdf_order == 2;
  const double a_t = bdf2 ? 1.5 / dt : 1.0 / dt;
  int r = sync(c);
  if (r) return r;
  if (a_t != F.a_t) {
    drop_graphs(c);
    for (auto& L : c->lev) L.a_t = a_t;
  }
  if (bdf2)
    launch_time_source(F.src, c->d_un, c->d_unm1, -4.0 / (2.0 * dt), 1.0 / (2.0 * dt), m, c->st);
  else
    launch_time_source(F.src, c->d_un, nullptr, -1.0 / dt, 0.0, m, c->st);
  ++c->launches;
  r = fasw_solve_steady(c, drop, max_cycles, history, ncycles);
  if (r != FASW_OK && r != FASW_ERR_NOT_CONVERGED) return r;
  // shift the history: u^(n-1) <- u^n, u^n <- u
  CKR(cudaMemcpyAsync(c->d_unm1, c->d_un, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  launch_pack(F, nullptr, 0, c->d_un, c->st);
  ++c->launches;
  c->steps_done += 1;
  const int rs = sync(c);
  return rs ? rs : r;
}

int fasw_profile(fasw_ctx* c, int enable) {
  if (!c) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  c->profiling = enable ? 1 : 0;
  for (int k = 0; k < FASW_NKERNELS; ++k) {
    c->prof_count[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  return FASW_OK;
}

int fasw_kernel_time(fasw_ctx* c, int kernel, long long* count, double* total_ms) {
  if (!c || kernel < 0 || kernel >= FASW_NKERNELS) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  if (count) *count = c->prof_count[kernel];
  if (total_ms) *total_ms = c->prof_ms[kernel];
  return FASW_OK;
}

// ---------------------------------------------------------------- batched cases
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
std::map<TuneKey, int> g_tune_cache;
std::mutex g_tune_mutex;

TuneKey key_of(fasw_ctx* c) {
  const LevelDev& F = c->lev[c->L()];
  return TuneKey{F.ni, F.nj, c->mixed};
}
}  // namespace

// Times `reps` batch cycles with kinds[k] on case k (after one capturing cycle); states restored.
static int batch_time(fasw_batch* b, const std::vector<int>& kinds, const std::vector<double*>& saved, int reps,
                      cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  for (size_t k = 0; k < b->cases.size(); ++k) {
    b->cases[k]->sweep_kind = kinds[k];
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
  std::vector<int> kinds(nc, SWEEP_HP);
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
      for (size_t k : gk.second) kinds[k] = it->second;
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
      if ((r = batch_time(b, kinds, saved, reps, e0, e1, &a))) return;
      if ((r = batch_time(b, kinds, saved, reps, e0, e1, &c2))) return;
      *out = std::min(a, c2);
    };
    const int cand[3] = {SWEEP_HP8, SWEEP_HP4, SWEEP_CTA};
    // larger shapes first: they dominate the batch time
    std::vector<std::pair<TuneKey, std::vector<size_t>>> order(groups.begin(), groups.end());
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) {
      return (long long)x.first.ni * x.first.nj * x.second.size() > (long long)y.first.ni * y.first.nj * y.second.size();
    });
    // each candidate against the incumbent timed right beside it; a switch must gain 2 %
    for (size_t gi = 0; gi < order.size() && r == FASW_OK; ++gi) {
      const std::vector<size_t>& members = order[gi].second;
      int keep = kinds[members[0]];
      for (int k : cand) {
        if (k == keep || r) continue;
        float t_keep = 0.f, t_k = 0.f;
        timed(&t_keep);
        for (size_t m : members) kinds[m] = k;
        if (r == FASW_OK) timed(&t_k);
        if (r == FASW_OK && t_k < 0.98f * t_keep) keep = k;
        for (size_t m : members) kinds[m] = keep;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (auto& gk : groups) g_tune_cache[gk.first] = kinds[gk.second[0]];
  }
  for (size_t k = 0; k < nc; ++k) {
    b->cases[k]->sweep_kind = kinds[k];
    drop_graphs(b->cases[k]);
    if (choice) choice[k] = kinds[k];
  }
  batch_drop_graphs(b);
  return FASW_OK;
}

long long fasw_batch_launch_count(fasw_batch* b) { return b ? b->launches : -1; }

const char* fasw_strerror(int code) {
  switch (code) {
    case FASW_OK: return "ok";
    case FASW_ERR_ARG: return "invalid argument";
    case FASW_ERR_OOM: return "device allocation failed";
    case FASW_ERR_CUDA: return "CUDA runtime error";
    case FASW_ERR_DIVERGED: return "residual diverged";
    case FASW_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case FASW_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case FASW_ERR_TOO_LARGE: return "grid too large for the fixed no-allocation scratch";
    default: return "unknown error";
  }
}

const char* fasw_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

}  // extern "C"
