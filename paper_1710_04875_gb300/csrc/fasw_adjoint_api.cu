// C ABI of the discrete adjoint (steady finest level with the eddy viscosity frozen, the
// unsteady adjoint of dual time stepping with binomial checkpointing, shape and vertex
// gradients); the adjoint kernels and the preconditioners are in kernels_adjoint.cu.
#include <cmath>
#include <algorithm>
#include <vector>

#include "fasw_ctx.cuh"
#include "fasw_transfer.cuh"
#include "fasw_checkpoint.cuh"

using namespace fasw;

extern "C" {

// ---- discrete adjoint (steady finest level, eddy viscosity frozen)
static int adj_ready(fasw_ctx* c) {
  if (c->adj.n) return FASW_OK;
  const LevelDev& F = c->lev[c->L()];
  if (!c->adj.tan.u) {  // tangent arrays first: the workspace is published only when complete
    void* mem = nullptr;
    const int r = device_alloc(&mem, tangent_doubles(F) * sizeof(double));
    if (r) return r;
    c->allocs.push_back(mem);
    tangent_carve(F, static_cast<double*>(mem), c->adj.tan);
  }
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

// FASW_ERR_DEVICE_TIMEOUT when a bounded wait of the sweeps ran out since the last err_clear.
static int adj_err_check(fasw_ctx* c) { return err_read(c); }

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
  err_clear(c);
  adj_build_precond(c->adj, c->lev[c->L()], c->ph, c->sc, cfl, c->st, c->launches);
  adj_steps_apply(c->adj, steps, c->d_tmp, c->d_tmp2, c->st);
  c->launches += 2;
  if ((e = adj_err_check(c))) return e;
  if ((e = copy_out(c, z, c->d_tmp2, m, on_device))) return e;
  return sync(c);
}

int fasw_adjoint_set_jacobian(fasw_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 1) return FASW_ERR_ARG;
  if (mode != c->adj.jac_mode) c->adj.built = false;
  c->adj.jac_mode = mode;
  return FASW_OK;
}

int fasw_tangent_residual(fasw_ctx* c, const double* v, double* dF, double* F, int on_device) {
  if (!c || !v || !dF || c->ph.moving) return FASW_ERR_ARG;
  int r = adj_ready(c);
  if (r) return r;
  LevelDev& L = c->lev[c->L()];
  const size_t m = 4 * (size_t)L.n;
  if ((r = copy_in(c, c->d_tmp, v, m, on_device))) return r;
  launch_bc_aux(L, c->ph, 1.0, 0, c->st);
  launch_tangent(L, c->adj.tan, c->ph, c->d_tmp, nullptr, 0, -1, 0.0, c->adj.Fp, nullptr, F ? c->adj.Fm : nullptr,
                 nullptr, nullptr, c->st);
  c->launches += 6;
  if ((r = copy_out(c, dF, c->adj.Fp, m, on_device))) return r;
  if (F && (r = copy_out(c, F, c->adj.Fm, m, on_device))) return r;
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
  err_clear(c);
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
  err_clear(c);
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
  *dC = which < 0 ? 0.0 : which == 0 ? cl[0] - cl[1] : cd[0] - cd[1];  // which -1: no explicit part
  return adj_dot(c->adj, d_lam, c->d_tmp2, (int)m, c->st, dot);
}

}  // namespace

extern "C" {

int fasw_adjoint_shape_gradient(fasw_ctx* c, int which, const double* lam, int nparam, const double* vy, double h_x,
                                double* grad, int on_device) {
  if (!c || !lam || !vy || !grad || nparam < 1 || which < -1 || which > 1 || !(h_x > 0.0) || c->ph.moving)
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

int fasw_pitching_objective(fasw_ctx* c, double amp, double omega, double xc, double yc, double dt, int nsteps,
                            int bdf_order, double drop, int max_cycles, int which, double* objective, int* cycles) {
  if (!c || !objective || nsteps < 1 || which < 0 || which > 1 || !(dt > 0.0)) return FASW_ERR_ARG;
  double J = 0.0;
  int total = 0, soft = 0;
  for (int n = 1; n <= nsteps; ++n) {
    const double t = n * dt;
    int r = fasw_set_motion(c, -amp * std::sin(omega * t), -amp * omega * std::cos(omega * t), xc, yc);
    if (r) return r;
    int nc = 0;
    r = fasw_dual_time_step(c, dt, bdf_order, drop, max_cycles, nullptr, &nc);
    total += nc;
    if (r == FASW_ERR_NOT_CONVERGED)
      soft = 1;
    else if (r)
      return r;
    double cl = 0.0, cd = 0.0;
    if ((r = fasw_force_coefficients(c, &cl, &cd))) return r;
    J += (which == 0 ? cl : cd) / nsteps;
  }
  *objective = J;
  if (cycles) *cycles = total;
  return soft ? FASW_ERR_NOT_CONVERGED : FASW_OK;
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
    for (void* p : mem) device_free(p);
  }
  int get(double** p, size_t count) {
    void* q = nullptr;
    const int r = device_alloc(&q, (count ? count : 1) * sizeof(double));
    if (r != FASW_OK) return r;
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
      if (c->prm.turb && !c->mut_frozen) {  // eddy viscosity frozen at its value for u^n
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
      err_clear(c);
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

}  // extern "C"
