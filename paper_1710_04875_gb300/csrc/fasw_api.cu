// C ABI and host-side driver: level allocation, the AW / ARK stage loop (sections 4.1-4.2
// of arXiv 1710.04875), the FAS V/W cycle (section 3), the steady solve loop and dual time
// stepping (section 6).  Every arithmetic step runs in the kernels of the other translation
// units; the adjoint entry points are in fasw_adjoint_api.cu, batches in fasw_batch.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <atomic>
#include <vector>

#include "fasw_ctx.cuh"
#include "fasw_transfer.cuh"

using namespace fasw;

namespace fasw {
thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return FASW_ERR_CUDA;
}
}  // namespace fasw

namespace {

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

}  // namespace

namespace fasw {

// Host-side allocation-failure injection and a count of the library's live device
// allocations (fasw_fault_inject_alloc, fasw_live_allocations): a failure is made on the host,
// before cudaMalloc would be called, so no GPU fault is involved.
std::atomic<long long> g_fail_alloc_in{-1};
std::atomic<long long> g_live_allocs{0};

int device_alloc(void** q, size_t bytes) {
  long long k = g_fail_alloc_in.load();
  while (k >= 0 && !g_fail_alloc_in.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 0) {
    g_last_cuda_error = "allocation failure injected on the host";
    return FASW_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(q, bytes);
  if (e != cudaSuccess) {
    g_last_cuda_error = cudaGetErrorString(e);
    return FASW_ERR_OOM;
  }
  g_live_allocs.fetch_add(1);
  return FASW_OK;
}

void device_free(void* q) {
  if (!q) return;
  cudaFree(q);
  g_live_allocs.fetch_sub(1);
}

template <typename T>
int dalloc(fasw_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  const int r = device_alloc(&q, count * sizeof(T));
  if (r != FASW_OK) return r;
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return FASW_OK;
}

// The device error word records a bounded wait that ran out.  Each call that runs sweeps clears
// it first (on the stream, so a captured cycle clears it too) and reads it at its end, so a
// timeout is reported by the call in which it happened and later calls start clean.
void err_clear(fasw_ctx* c) { cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st); }

int err_read(fasw_ctx* c) {
  CKR(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CKR(cudaStreamSynchronize(c->st));
  return *c->h_err ? FASW_ERR_DEVICE_TIMEOUT : FASW_OK;
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
  A(L.norm_part, (size_t)residual_blocks_max(L));
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
  if (ws_fits(L.ni, L.nj, L.nw)) {
    const size_t wf = ws_floats(L.ni, L.nj), wv = ws_vec_floats(L.ni, L.nj);
    A(L.wsF, wf);
    A(L.wsB, wf);
    A(L.wsC, wv);
    A(L.wsY, wv);
    A(L.wsCut, 16 * (size_t)(L.nw > 0 ? L.nw : 1));
    A(L.wsZ, 2 * wv);
    A(L.wsT, 4 * n);
    A(L.wsX, 4 * n);
    // padding positions of the skewed arrays are never written: they must read as zero
    CKR(cudaMemsetAsync(L.wsF, 0, wf * sizeof(float), c->st));
    CKR(cudaMemsetAsync(L.wsB, 0, wf * sizeof(float), c->st));
    CKR(cudaMemsetAsync(L.wsC, 0, wv * sizeof(float), c->st));
    CKR(cudaMemsetAsync(L.wsY, 0, wv * sizeof(float), c->st));
    CKR(cudaMemsetAsync(L.wsZ, 0, 2 * wv * sizeof(float), c->st));
    CKR(cudaMemsetAsync(L.wsCut, 0, 16 * (size_t)(L.nw > 0 ? L.nw : 1) * sizeof(float), c->st));
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
  if (c->exact_iters > 0 && L.wsF) return SWEEP_WS;  // the exact-preconditioner iterations run on it
  int k = c->sweep_kind;
  if (k == SWEEP_AUTO) {
    // measured per level on GB300: the warp strips win on every level in both precisions (mixed,
    // one application: 64x16 28.6 against 32.3 us for the one-CTA hyperplane-staged sweep,
    // 128x32 41.9 against 58.3 us)
    if (L.wsF) return SWEEP_WS;
    return c->mixed ? (L.hpF ? SWEEP_HP : SWEEP_CTA) : SWEEP_STRIPS;
  }
  if (is_ws(k) && !L.wsF) k = c->mixed ? SWEEP_CTA : SWEEP_STRIPS;
  if (is_hp(k) && !(c->mixed && L.hpF)) k = c->mixed ? SWEEP_CTA : SWEEP_STRIPS;
  if (c->in_batch && (k == SWEEP_STRIPS || k == SWEEP_STRIPS16 || k == SWEEP_STRIPS4))
    k = L.wsF ? SWEEP_WS : SWEEP_CTA;  // concurrent cases: only sweeps whose CTAs are co-scheduled
  return k;
}

void run_sweep(fasw_ctx* c, const LevelDev& L, int do_update, double alpha, const double* rhs) {
  if (c->sweep_kind == SWEEP_LEGACY) {
    launch_sgs(L, c->sc, c->mixed, do_update, alpha, rhs, nullptr, c->st);
    ++c->launches;
    return;
  }
  c->launches += launch_sweep(L, c->mixed, level_sweep_kind(c, L), do_update, c->sc.aw, alpha, rhs, c->d_prog,
                              c->d_err, c->spin_limit, c->st, c->exact_iters);
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


void enqueue_cycle(fasw_ctx* c, double cfl) {
  const int Lf = c->L();
  err_clear(c);
  if (c->prm.turb && !c->mut_frozen) {
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
int run_cycle(fasw_ctx* c, double cfl) {
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

}  // namespace fasw


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
  if (p->flux < 0 || p->flux > 1) return FASW_ERR_ARG;
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
  c->ph.flux = p->flux;
  c->ph.d_cut = p->d_cut;
  free_stream(p->mach, p->alpha_deg, c->ph.uinf);
  set_free_stream_prims(c->ph);
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
  for (void* q : c->allocs) device_free(q);
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
  err_clear(c);
  run_sweep(c, L, 0, 0.0, c->d_tmp2);
  const double* zsrc = L.yz64;
  if (c->mixed) {
    launch_f2d(L.yz32, c->d_tmp, (int)m, c->st);
    ++c->launches;
    zsrc = c->d_tmp;
  }
  r = copy_out(c, z, zsrc, m, on_device);
  if (r) return r;
  r = sync(c);
  return r ? r : err_read(c);
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
  err_clear(c);
  for (int k = 0; k < nsteps; ++k) smooth_step(c, l, cfl, false);
  int r = sync(c);
  return r ? r : err_read(c);
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

int fasw_set_sweep(fasw_ctx* c, int kind) {
  if (!c || kind < SWEEP_AUTO || kind > SWEEP_WS8) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  c->sweep_kind = kind;
  drop_graphs(c);
  return FASW_OK;
}

int fasw_set_exact_preconditioner(fasw_ctx* c, int iters) {
  if (!c || iters < 0 || iters > 1000) return FASW_ERR_ARG;
  for (auto& L : c->lev)
    if (iters > 0 && !L.wsF) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  c->exact_iters = iters;
  drop_graphs(c);
  return FASW_OK;
}

int fasw_set_residual_tile(fasw_ctx* c, int rows) {
  if (!c || !(rows == 0 || rows == 1 || rows == 2 || rows == 4 || rows == 8)) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  for (auto& L : c->lev) L.res_ty = rows;
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
  if (!c->mut_frozen) {
    bc_aux(c, Lf, 1.0, 0);
    launch_bl(c->lev[Lf], c->ph, c->st);
    c->launches += 2;
  }
  int r = copy_out(c, mut, c->lev[Lf].mut, (size_t)c->lev[Lf].n, on_device);
  if (r) return r;
  if (!c->prm.turb)  // a laminar context's residual must not see the eddy viscosity
    CKR(cudaMemsetAsync(c->lev[Lf].mut, 0, (size_t)c->lev[Lf].n * sizeof(double), c->st));
  return sync(c);
}

int fasw_freeze_mut(fasw_ctx* c, const double* mut, int on_device) {
  if (!c) return FASW_ERR_ARG;
  if (mut && !c->prm.turb) return FASW_ERR_ARG;
  int r = sync(c);
  if (r) return r;
  drop_graphs(c);  // the captured cycles hold the Baldwin-Lomax launches, or not
  c->mut_frozen = mut != nullptr;
  if (mut) {
    LevelDev& F = c->lev[c->L()];
    if ((r = copy_in(c, F.mut, mut, (size_t)F.n, on_device))) return r;
  }
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

int fasw_check_math(int n, const double* a, const double* b, double* out, int on_device) {
  if (n < 0 || (n > 0 && (!a || !b || !out))) return FASW_ERR_ARG;
  if (n == 0) return FASW_OK;
  const size_t m = (size_t)n;
  if (on_device) {
    launch_check_math(n, a, b, out, 0);
    CKR(cudaGetLastError());
    CKR(cudaDeviceSynchronize());
    return FASW_OK;
  }
  double* d = nullptr;
  if (cudaMalloc(&d, 6 * m * sizeof(double)) != cudaSuccess) return FASW_ERR_OOM;
  cudaError_t e = cudaMemcpy(d, a, m * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + m, b, m * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_check_math(n, d, d + m, d + 2 * m, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * m, 4 * m * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? FASW_OK : cuda_fail(e);
}

void fasw_fault_inject_alloc(long long n) { g_fail_alloc_in.store(n < 0 ? -1 : n); }

long long fasw_live_allocations(void) { return g_live_allocs.load(); }

int fasw_scheme_coefficients(int scheme, int* nstages, double* alpha, double* beta) {
  if (scheme < 0 || scheme > 7 || !nstages) return FASW_ERR_ARG;
  const Coef& cf = kCoef[scheme % 4];
  *nstages = cf.s;
  for (int k = 0; k < cf.s; ++k) {
    if (alpha) alpha[k] = cf.a[k];
    if (beta) beta[k] = cf.b[k];
  }
  return FASW_OK;
}

// ---------------------------------------------------------------- batched cases
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
