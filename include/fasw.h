/*
 * fasw.h -- C ABI of the GB300 (sm_103a) library for preconditioned FAS smoothers
 * on 2D finite-volume Euler / thin-layer RANS on structured C-grids.
 *
 * Method: Birken, Bull & Jameson, "Preconditioned smoothers for the full
 * approximation scheme for the RANS equations" (arXiv 1710.04875):
 *   - JST residual, section 2 (eqs. e2, e4, spectralcorrection), steady system
 *     eq. (nonlin-eq-steady), BDF2 system eq. (nonlin-eq);
 *   - FAS cycle with agglomeration restriction and bilinear prolongation, section 3,
 *     coarse equation eq. (coarse-nonlin-eq);
 *   - additive W (AW) and preconditioned additive Runge-Kutta (ARK) low-storage
 *     stage loops, sections 4.1-4.2, coefficients of Table "RK smoothers";
 *   - block SGS preconditioner (D+L) D^-1 (D+U), eq. (sgs-precon), built from
 *     flux-vector-split Jacobians at face-averaged states with the parabolic
 *     eigenvalue cutoff, eqs. (cutoff), (d-l-u-matrices-J), (d-l-u-matrices-W).
 *
 * Conventions (all entry points):
 *   - Every call returns int: FASW_OK (0) or a negative FASW_ERR_* code.
 *   - Grid: vertex (i, j) of an ni x nj-cell C-grid at index j*(ni+1)+i; i runs
 *     along the C (lower wake outflow .. trailing edge .. lower surface .. leading
 *     edge .. upper surface .. trailing edge .. upper wake outflow), j from the
 *     wall / wake cut (j = 0) to the far field.  Cells (i,0) with i < n_wake or
 *     i >= ni - n_wake lie on the wake cut, whose vertices coincide pairwise
 *     (vertex i with vertex ni - i).
 *   - State / residual arrays: 4 x nj x ni doubles, component-major (rho, rho u,
 *     rho v, rho E), cell (i, j) at c*ni*nj + j*ni + i; nondimensional with
 *     rho_inf = 1, |v_inf| = 1, p_inf = 1/(gamma M^2), chord 1.
 *   - Caller buffers are borrowed for the duration of the call and never retained.
 *     Pointers flagged on_device are device pointers; otherwise host pointers.
 *   - All device work is enqueued on the stream given to fasw_create.  Calls that
 *     return host values (norms, histories, host copies) synchronize that stream.
 *   - A context is not thread-safe.  The library owns every device buffer it
 *     allocates (cudaMalloc at create, cudaFree at destroy).
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     touches the device returns FASW_ERR_CUDA.
 *   - Bounded device-side waits (the strip-pipelined sweeps, where one CTA waits for the
 *     rows of another) give up after spin_limit polls and set the context's device error
 *     word; the call that ran the sweep returns FASW_ERR_DEVICE_TIMEOUT (its results are
 *     then incomplete).  Every call that runs sweeps clears the word first, so a timeout is
 *     reported by the call in which it happened and does not poison later calls.
 */
#ifndef FASW_H
#define FASW_H

#ifdef __cplusplus
extern "C" {
#endif

#define FASW_OK 0
#define FASW_ERR_ARG (-1)            /* invalid argument or grid not coarsenable */
#define FASW_ERR_OOM (-2)            /* device allocation failed */
#define FASW_ERR_CUDA (-3)           /* CUDA runtime error (message via fasw_last_cuda_error) */
#define FASW_ERR_DIVERGED (-4)       /* residual norm became NaN/Inf or grew by > 1e8 */
#define FASW_ERR_DEVICE_TIMEOUT (-5) /* a bounded device-side wait ran out */
#define FASW_ERR_NOT_CONVERGED (-6)  /* soft: max_cycles reached; history is filled */
#define FASW_ERR_TOO_LARGE (-7)      /* grid needs more than the fixed no-allocation scratch */

/* Smoother schemes (Table "RK smoothers"; AW uses the same alpha/beta as ARK). */
enum fasw_scheme {
  FASW_AW3 = 0, FASW_AW5J = 1, FASW_AW51 = 2, FASW_AW52 = 3,
  FASW_ARK3J = 4, FASW_ARK5J = 5, FASW_ARK51 = 6, FASW_ARK52 = 7
};

/* Arithmetic of the preconditioner (blocks, LU and sweeps). */
enum fasw_precision { FASW_FP64 = 0, FASW_MIXED = 1 };

typedef struct fasw_params {
  int scheme;          /* enum fasw_scheme */
  int nlevels;         /* multigrid levels, >= 1; ni, nj, n_wake divisible by 2^(nlevels-1) */
  int gamma_cycle;     /* 1 = V-cycle, 2 = W-cycle (section 3) */
  int nu1;             /* presmoothing steps per level visit (>= 1) */
  int viscous;         /* 0 = Euler (slip wall), 1 = thin-layer Navier-Stokes (no-slip wall) */
  int turb;            /* 0 = laminar, 1 = Baldwin-Lomax eddy viscosity (finest level, once per cycle) */
  int sensor;          /* 0 = pressure sensor, 1 = entropy sensor p/rho^gamma */
  double mach, alpha_deg, re, pr, prt;
  double eta;          /* W-method parameter */
  double d_cut;        /* eigenvalue cutoff fraction d in [0,1], eq. (cutoff) */
  double cfl;          /* pseudo CFL number c* */
  double cfl_ramp;     /* cap on c* during the first ramp_cycles cycles (section 6: 20 for 2) */
  int ramp_cycles;
  double s_coarse;     /* constant sensor value of the first-order coarse-level JST */
  int precision;       /* enum fasw_precision */
  int norm_all;        /* 0: RMS of the density residual; 1: RMS over all 4 components */
  long long spin_limit;/* bound on device-side waits (iterations); <= 0 picks the default */
  int flux;            /* residual face flux: 0 = JST (section 2), 1 = first-order flux-vector splitting
                          A+(u_bar) u_L + A-(u_bar) u_R with the cutoff d_cut (the discretization of
                          eqs. steadylinearized / form1, section 4.4, whose linearization at frozen
                          face states the preconditioner's blocks are) */
} fasw_params;

typedef struct fasw_ctx fasw_ctx;

/* Fill *p with the defaults (robust mode: AW3, d = 0.5, eta = 0.8, c* = 1e4, ramp 20 for 2
 * cycles, 3-level V-cycle, M = 0.8, Euler, FP64). */
void fasw_default_params(fasw_params* p);

/* Create a solver for one grid.  x, y: (ni+1)*(nj+1) vertex coordinates (host, or device if
 * coords_on_device).  stream: a cudaStream_t (NULL = legacy default stream).  The state of
 * every level starts at the free stream.  Errors: FASW_ERR_ARG (sizes, NULL pointers,
 * levels), FASW_ERR_OOM, FASW_ERR_CUDA. */
int fasw_create(int ni, int nj, int n_wake, const double* x, const double* y, int coords_on_device,
                const fasw_params* p, void* stream, fasw_ctx** out);

/* Release every device buffer of the context.  NULL is ignored. */
void fasw_destroy(fasw_ctx* ctx);

/* Level l in the paper's numbering: 0 = coarsest, nlevels-1 = finest.  Dimensions of a level. */
int fasw_level_dims(fasw_ctx* ctx, int level, int* ni, int* nj, int* n_wake);

/* Copy the interior state of a level in / out (4 x nj x ni).  set_state refills the ghosts. */
int fasw_set_state(fasw_ctx* ctx, int level, const double* u, int on_device);
int fasw_get_state(fasw_ctx* ctx, int level, double* u, int on_device);

/* FAS forcing s_l of a level (4 x nj x ni); zero on the finest level of a steady solve. */
int fasw_set_forcing(fasw_ctx* ctx, int level, const double* s, int on_device);
int fasw_get_forcing(fasw_ctx* ctx, int level, double* s, int on_device);

/* Residual of level l at its current state, per unit volume, split as eq. (split-rhs):
 * F = F^c + F^v with F^c = Omega^-1 (central fluxes) + a_t u + src - s_l and
 * F^v = Omega^-1 (-(JST dissipation) - (viscous fluxes)).  Any output may be NULL.
 * norm (nullable): RMS of the density component of F (all components if norm_all). */
int fasw_residual(fasw_ctx* ctx, int level, double* F, double* Fc, double* Fv, int on_device, double* norm);

/* Local pseudo time step dt*_i = cfl Omega_i / (r_xi + r_eta) at the current state (n doubles). */
int fasw_pseudo_dt(fasw_ctx* ctx, int level, double cfl, double* dts, int on_device);

/* Build dt* (with cfl) and the preconditioner at the current state, then z = P^-1 r with
 * P = (D+L) D^-1 (D+U) (eq. sgs-precon); r, z: 4 x nj x ni.  AW blocks of eq.
 * (d-l-u-matrices-W) or ARK blocks of eq. (d-l-u-matrices-J) by the context's scheme. */
int fasw_precond_apply(fasw_ctx* ctx, int level, double cfl, const double* r, double* z, int on_device);

/* Split face Jacobians A+ and A- (times the face length) at the current state:
 * i-faces (nj x (ni+1) x 16 each) and j-faces ((nj+1) x ni x 16), row-major 4x4.
 * Always FP64 (independent of the precision setting).  Any output may be NULL. */
int fasw_face_blocks(fasw_ctx* ctx, int level, double* axp, double* axm, double* aep, double* aem, int on_device);

/* nsteps smoothing steps of the context's scheme on level l with pseudo CFL cfl
 * (dt* and the preconditioner frozen at the start of each step). */
int fasw_smooth(fasw_ctx* ctx, int level, int nsteps, double cfl);

/* One FAS cycle (V or W, section 3) from the finest level.  cycle_index selects the
 * c* ramp.  res_norm (nullable): residual norm at the start of the cycle. */
int fasw_fas_cycle(fasw_ctx* ctx, int cycle_index, double* res_norm);

/* Cycles until norm_k <= drop * norm_0 (k >= 1) or max_cycles.  history (nullable, max_cycles
 * doubles): norm at the start of each cycle.  *ncycles: cycles run.  Returns FASW_OK,
 * FASW_ERR_NOT_CONVERGED, or FASW_ERR_DIVERGED. */
int fasw_solve_steady(fasw_ctx* ctx, double drop, int max_cycles, double* history, int* ncycles);

/* enable != 0 (the default): each FAS cycle is captured once per pseudo CFL value into a CUDA
 * graph and replayed; 0 launches every kernel individually.  Capture needs a non-default
 * stream; with the legacy default stream (NULL) cycles are always launched individually. */
int fasw_use_graphs(fasw_ctx* ctx, int enable);

/* How the SGS sweeps run: 0 = automatic (warp strips, 9, in both precisions; a level the warp
 * strips do not fit -- more than 256 rows -- takes the strip-pipelined sweep in FP64 and the
 * hyperplane-staged sweep, else one CTA, in mixed precision), 1 = one
 * thread per cell
 * applying the LU blocks (reference kernel), 2 = one CTA with precomputed transfer blocks
 * (strips where a hyperplane exceeds 128 cells), 3 = strip-pipelined with 8 rows per strip,
 * 4 = with 16 rows per strip, 5 = hyperplane-staged (mixed precision only, nj <= 256: blocks
 * stored hyperplane-major and staged through shared memory by cp.async; elsewhere as 0), 6 / 7 =
 * hyperplane-staged with a staging ring of 4 / 8 steps, 8 = strip-pipelined with 4 rows per
 * strip, 9 = warp strips: one warp per strip of 32 rows, each lane a row holding all four
 * components of its cell, operands staged into shared memory by bulk asynchronous copies, the
 * strips of one sweep launched as one thread-block cluster, each strip storing its boundary row
 * straight into the shared memory of the strip that reads it; its recurrence runs in FP32, and in
 * FP64 contexts it is followed by one FP64 defect correction (the FP64 residual of the SGS system
 * at the FP32 result, solved by a second FP32 sweep and added), which brings the result to FP64
 * accuracy; 10 = as 9, with operand chunks of 8 steps instead of 16 staged in shared memory (half
 * the shared memory per strip, so that strips of different batch cases can share an SM).  All
 * give the same Gauss-Seidel result up to rounding.  Synchronizes the stream; drops captured
 * cycles. */
int fasw_set_sweep(fasw_ctx* ctx, int kind);

/* The "exact" preconditioner (the column of that name in section 5.4's tables): iters > 0 makes
 * every application of the preconditioner, in the smoother and in fasw_precond_apply, continue
 * the SGS solve by iters block Gauss-Seidel corrections x <- x + P^-1 (r - (D+L+U) x) (P the SGS
 * factorization, applied by the warp-strip sweep), which converge to (D+L+U)^-1 r, the inverse of
 * the whole first-order flux-vector-split operator the blocks form; 0 (the default) is the
 * paper's SGS preconditioner.  FASW_ERR_ARG for iters outside 0..1000 or a level the warp-strip
 * sweep does not fit.  Synchronizes the stream; drops captured cycles. */
int fasw_set_exact_preconditioner(fasw_ctx* ctx, int iters);

/* Tile height of the residual kernel (tiles of 31 x rows cells, one thread per face), on every
 * level: rows = 1, 2, 4 or 8, or 0 (the default) for a choice from each level's size.  The
 * result does not depend on it.  Synchronizes the stream; drops captured cycles. */
int fasw_set_residual_tile(fasw_ctx* ctx, int rows);

/* Eddy viscosity of the finest level (Baldwin-Lomax from the current state); n doubles.  A
 * laminar context (turb = 0) keeps a zero eddy viscosity in its own residual. */
int fasw_get_mut(fasw_ctx* ctx, double* mut, int on_device);

/* Holds the finest level's eddy viscosity at mut (n doubles, cell order) in every later cycle,
 * solve and dual-time step (no Baldwin-Lomax evaluation), or returns to the model (mut = NULL).
 * A primal solve so frozen is the one the discrete adjoint linearizes (the adjoint holds mu_t
 * fixed): central differences of such solves check the adjoint gradient.  FASW_ERR_ARG for a
 * laminar context with mut != NULL.  Synchronizes; drops captured cycles. */
int fasw_freeze_mut(fasw_ctx* ctx, const double* mut, int on_device);

/* Dual time stepping, eq. (nonlin-eq): set a_t (3/(2 dt) for BDF2, 1/dt for implicit Euler;
 * 0 = steady) on every level and the history source src (finest level, 4 x nj x ni;
 * NULL = zero), so that F gains a_t u + src and D gains eta dt* a_t I (AW) or a_t I (ARK). */
int fasw_set_time_source(fasw_ctx* ctx, double a_t, const double* src, int on_device);

/* Rigid motion of the whole grid (the pitching motion of section 6): the reference grid rotated
 * by phi (radians, counter-clockwise) about (xc, yc), moving at angular rate phidot.  Recomputes
 * the metrics of every level and the face grid volume fluxes v_grid . S, which enter the
 * convective fluxes (F . S - u v_grid . S), the spectral radii and the FVS eigenvalues
 * (relative normal velocity), the wall ghosts (moving wall) and the far-field in/outflow
 * test.  Volumes are unchanged by a rigid motion, so the discrete geometric conservation law
 * holds.  Synchronizes the stream. */
int fasw_set_motion(fasw_ctx* ctx, double phi, double phidot, double xc, double yc);

/* One physical time step of dual time stepping, eq. (nonlin-eq): the first call takes the
 * current finest-level state as u^n and uses implicit Euler (section 6); later calls use BDF2
 * when bdf_order == 2.  Sets a_t and the history source, runs pseudo-time FAS cycles until the
 * residual drops by `drop` (or max_cycles; history/ncycles as in fasw_solve_steady), then
 * shifts the history.  Place the grid at the new time level first (fasw_set_motion).
 * Returns FASW_OK, FASW_ERR_NOT_CONVERGED, FASW_ERR_DIVERGED or another error. */
int fasw_dual_time_step(fasw_ctx* ctx, double dt, int bdf_order, double drop, int max_cycles, double* history,
                        int* ncycles);

/* ---- Discrete adjoint of the steady residual on the finest level.  The primal method is the
 * paper's; the adjoint is the standard one of F(u, X) = 0 with an objective J(u, X):
 * (dF/du)^T lambda = (dJ/du)^T and dJ/dX = dJ/dX|_u - lambda^T dF/dX.  The eddy viscosity is
 * frozen at its current value (no dependence of mu_t on u or X); fixed grid, steady (a_t = 0).
 * Objectives: lift and drag coefficients (which = 0: C_L, 1: C_D) of the force the scheme's own
 * wall-face fluxes (j = 0 faces off the wake cut: central flux minus dissipation minus viscous
 * flux) exert on the body, for the free stream of the parameters (rho = 1, |v| = 1, chord 1).
 * Vectors are 4 x nj x ni, component-major, like the state. */

/* C_L and C_D at the current state.  Synchronizes. */
int fasw_force_coefficients(fasw_ctx* ctx, double* cl, double* cd);
/* Assembles J = dF/du at the current state, 11 4x4 blocks per cell, and the state gradients of
 * C_L and C_D, colour by colour (a greedy colouring in which no residual stencil holds two cells
 * of one colour).  By default (fasw_adjoint_set_jacobian mode 1) every column comes from the
 * forward-mode linearization of the residual (fasw_tangent_residual's kernels): exact to rounding;
 * mode 0 takes central differences of the residual with relative step h_rel (step
 * h_rel * max(1, |u|) per unit).  The coarse levels' Jacobians of the transposed FAS cycle (a
 * preconditioner only) are always central differences.  The state is restored.  Synchronizes.
 * Errors: FASW_ERR_ARG (moving grid, dual-time term set, h_rel <= 0), FASW_ERR_OOM. */
int fasw_adjoint_jacobian(fasw_ctx* ctx, double h_rel);
/* Jacobian assembly of the finest level: 1 = forward-mode linearization (default), 0 = coloured
 * central differences.  The next fasw_adjoint_jacobian assembles with it. */
int fasw_adjoint_set_jacobian(fasw_ctx* ctx, int mode);
/* The residual's linearization applied to a vector, matrix-free: dF = (dF/du) v at the finest
 * level's current state (fixed grid, eddy viscosity frozen), by the forward-mode evaluation of
 * the residual's own formulas -- every quantity of section 2's discretization carried with its
 * derivative along v, the switches (JST pressure switch, eps4 cutoff, far-field in/outflow) held
 * on the branch the state takes.  Where a max, min or |.| of the switches ties (arguments equal
 * to 1e-8 relative, or |.| of a quantity zero to 1e-8 of its scale, as symmetric flows give
 * exactly) the derivative is the mean of the two one-sided slopes, the central derivative that
 * central differences also take.  v, dF: 4 x nj x ni; F (nullable) receives the residual itself
 * (the value part).  Synchronizes.  FASW_ERR_ARG on a moving grid. */
int fasw_tangent_residual(fasw_ctx* ctx, const double* v, double* dF, double* F, int on_device);
/* out = J v (transpose = 0) or J^T v (transpose != 0) with the assembled J. */
int fasw_adjoint_apply(fasw_ctx* ctx, const double* v, double* out, int transpose, int on_device);
/* State gradient dJ/du of objective `which` (as assembled with J). */
int fasw_adjoint_objective_gradient(fasw_ctx* ctx, int which, double* g, int on_device);
/* Adjoint preconditioner, built at pseudo CFL cfl at the current state: P = S^-1 W, W the primal
 * additive-W preconditioner (D+L) D^-1 (D+U) (section 4), S = eta dt* per cell.  steps = 0:
 * z = P^-T r = S (D+L)^-T D^T (D+U)^-T r; steps > 0: z = that many steps from zero of the
 * transposed primal stage loop x_i = x_0 + (alpha_i / eta) P^-T (r - J^T x_{i-1}) (needs
 * fasw_adjoint_jacobian first).  Rebuilds the finest level's preconditioner blocks and dt*. */
int fasw_adjoint_precond_apply(fasw_ctx* ctx, double cfl, int steps, const double* r, double* z, int on_device);
/* Preconditioner of the adjoint GMRES (the Jacobian must be assembled again after a change):
 *   0: steps of the primal stage loop run on J^T, x_i = x_0 + (alpha_i/eta) P^-T (r - J^T x_(i-1));
 *   1: steps of the exact transpose of the primal's linearised smoothing step (section 4: the
 *      stage loop with the dissipative part F^v blended by beta_i, so J = J^c + J^v is assembled
 *      in two parts);
 *   2 (default): the exact transpose of the primal's linearised FAS cycle (section 3: nu1
 *      smoothing steps per level visit, volume-weighted residual restriction R, gamma coarse
 *      cycles, bilinear prolongation P): C^T v = R^T r + S^T (v - J^T R^T r), r = A^T P^T v, with
 *      the coarse Jacobians taken at the volume-weighted restriction of the state; one level
 *      reduces it to kind 1 with one step;
 *   3: kind 2 with one coarse cycle per level visit (a V-cycle) whatever the primal's gamma.
 * The adjoint iteration with kind 2 has the primal FAS iteration's convergence rate (the two
 * iteration matrices are transposes up to similarity). Host only. */
int fasw_adjoint_set_precond(fasw_ctx* ctx, int kind);
/* z = M r with the linear operator of a preconditioner kind (1: the linearised smoothing step,
 * as many steps as set below; 2: the linearised FAS cycle), as a solver of J (transpose = 0) or
 * its transpose (transpose != 0), built at pseudo CFL cfl at the current state after
 * fasw_adjoint_jacobian (kind 2 needs the cycle selected when the Jacobian was assembled).
 * Rebuilds every level's preconditioner blocks and dt*. */
int fasw_adjoint_cycle_apply(fasw_ctx* ctx, double cfl, int kind, int transpose, const double* r, double* z,
                             int on_device);
/* Smoothing steps per application of the adjoint GMRES preconditioner (1..16; 3 by default):
 * more steps cost more transposed sweeps per Krylov iteration and save iterations.  Host only. */
int fasw_adjoint_set_precond_steps(fasw_ctx* ctx, int steps);
/* Solves J^T lam = g (g null: the gradient of objective `which`) by restarted GMRES(restart),
 * restart <= 251, to relative residual tol or max_iters iterations; *iters and *rel_res report
 * both.  Flexible GMRES, right-preconditioned by the preconditioner set above (by default the
 * transposed linearised FAS cycle; kinds 0 and 1 take three steps unless set otherwise), built
 * at pseudo CFL cfl (<= 0: the parameters' cfl).  Rebuilds the preconditioner blocks and dt* of
 * the levels it uses.
 * Returns FASW_OK or FASW_ERR_NOT_CONVERGED (lam holds the last iterate). */
int fasw_adjoint_solve(fasw_ctx* ctx, int which, const double* g, double* lam, double tol, int max_iters, int restart,
                       double cfl, int* iters, double* rel_res, int on_device);
/* Shape gradient of objective `which` for nparam vertex fields: vy is nparam x (nj+1) x (ni+1)
 * y-displacements per unit parameter (index k*(nj+1)*(ni+1) + j*(ni+1) + i);
 * grad[k] = dJ/dX V_k - lam^T dF/dX V_k, both X-derivatives by central differences of step
 * h_x along V_k at the current state; which = -1 leaves out the objective's explicit part
 * (grad[k] = -lam^T dF/dX V_k, the term through which a state adjoint lam reaches the shape).
 * The grid is restored.  grad is host memory. */
int fasw_adjoint_shape_gradient(fasw_ctx* ctx, int which, const double* lam, int nparam, const double* vy, double h_x,
                                double* grad, int on_device);

/* The objective of the pitching case (section 6's motion, applied as in fasw_set_motion):
 * nsteps dual-time steps (fasw_dual_time_step with bdf_order, drop, max_cycles) from the current
 * state, the grid placed at phi(t_n) = -amp sin(omega t_n) about (xc, yc) with rate
 * -amp omega cos(omega t_n) before step n, t_n = n dt; *objective = the average over the steps of
 * C_L (which 0) or C_D (1) at the end of each step; *cycles (nullable) the pseudo-time cycles run.
 * FASW_ERR_NOT_CONVERGED (soft, objective set) if a step stopped at max_cycles. */
int fasw_pitching_objective(fasw_ctx* ctx, double amp, double omega, double xc, double yc, double dt, int nsteps,
                            int bdf_order, double drop, int max_cycles, int which, double* objective, int* cycles);

/* The transposed product (dF/dX)^T lam with the objective's explicit part: for every vertex
 * coordinate, gx/gy = dJ/dX - lam^T dF/dX ((nj+1) x (ni+1) each, index j*(ni+1) + i), by central
 * differences over colour groups of vertices, each vertex moved by h_x times the shortest grid
 * edge at it (a wall vertex of a stretched grid moves by a small part of its first cell; a fixed
 * step would be a large part of it and the differences nonlinear) (a greedy colouring in which no cell
 * residual and no wall-face force depends on two vertices of one colour: a vertex reaches the
 * 6 x 6 cells around it, the cells that see those across the wake cut, and the wall faces next
 * to it).  Contracting with any vertex displacement field V gives that field's shape gradient
 * (fasw_adjoint_shape_gradient computes the same per field).  Fixed grid.  The grid is restored. */
int fasw_adjoint_vertex_gradient(fasw_ctx* ctx, int which, const double* lam, double h_x, double* gx, double* gy,
                                 int on_device);

/* ---- Discrete adjoint of dual time stepping (section 6: implicit Euler for the first step,
 * BDF2 after) on a rigidly pitching grid.  Level n = 1..N places the grid at rotation
 * phi(t_n) = -amp sin(omega t_n) about (xc, yc) (angle of attack alpha + amp sin(omega t)),
 * t_n = n dt, and solves F^n(u^n) = R(u^n; X^n)/vol + a_n u^n + b_n u^(n-1) + c_n u^(n-2) = 0
 * in pseudo time (fasw_dual_time_step).  Objective: J = (1/N) sum_n C(u^n, X^n), C the lift
 * (which = 0) or drag (1) coefficient.  Adjoint, backwards from n = N:
 *   (dF^n/du^n)^T lam^n = (1/N) dC^n/du^n - b_(n+1) lam^(n+1) - c_(n+2) lam^(n+2),
 * each solved like fasw_adjoint_solve; the shape gradient with the initial state held fixed is
 * sum_n [(1/N) dC^n/dX - lam^n . dF^n/dX] dX^n/dp and the initial-state sensitivity
 * dJ/du^0 = -(b_1 lam^1 + c_2 lam^2).  The eddy viscosity is frozen at each level's value.
 *
 * Checkpointing: the reverse sweep needs u^N, ..., u^1 in that order.  With `snapshots` stored
 * levels (each u^m and u^(m-1)) besides u^0, the states are recomputed from stored levels by
 * the binomial schedule of Griewank and Walther (fewest recomputed physical steps);
 * snapshots >= N - 1 stores every level once.  Recomputation is bit-identical to the first
 * sweep (the library's kernels are deterministic), so the result does not depend on it. */

/* The schedule alone (host code; no GPU needed).  Actions (ops[k], args[k]), k < *nactions, on
 * a working state that holds one time level: 0 advance to level arg, 1 store the current level,
 * 2 restore stored level arg (0 = the initial state), 3 adjoint step of level arg (the current
 * one), 4 free the slot of level arg.  capacity = 0 only reports *nactions.
 * *forward_steps: physical steps run, the initial sweep included.
 * Errors: FASW_ERR_ARG (nsteps < 1 or > 65536, snapshots < 0, too small a capacity). */
int fasw_checkpoint_schedule(int nsteps, int snapshots, int* ops, int* args, int capacity, int* nactions,
                             long long* forward_steps);

/* The unsteady adjoint run from the context's current state u^0 on the grid at rest (no
 * motion set, no dual-time step taken).  vy: nparam x (nj+1) x (ni+1) y-displacement fields of
 * the grid at rest (as fasw_adjoint_shape_gradient), nparam >= 0; h_rel, h_x: difference
 * steps of the Jacobian and of the X-derivatives.  Pseudo-time solves: drop, max_cycles;
 * adjoint solves: tol, max_iters, restart, cfl (as fasw_adjoint_solve).
 * Outputs: *objective = J; grad[nparam] (host); g0 = dJ/du^0 (4 x nj x ni, host or device per
 * on_device; may be NULL); stats (may be NULL) = {physical steps run, recomputed steps, total
 * GMRES iterations, pseudo-time cycles} as doubles, then the largest adjoint relative residual.
 * On return the context holds u^0 again on the grid at rest, with no time term.
 * Returns FASW_OK, FASW_ERR_NOT_CONVERGED (a pseudo-time or adjoint solve hit its limit; all
 * outputs are still filled), FASW_ERR_DIVERGED, FASW_ERR_ARG, FASW_ERR_OOM or FASW_ERR_CUDA. */
int fasw_unsteady_adjoint(fasw_ctx* ctx, double amp, double omega, double xc, double yc, double dt, int nsteps,
                          int bdf_order, double drop, int max_cycles, int snapshots, int which, int nparam,
                          const double* vy, double h_rel, double h_x, double tol, int max_iters, int restart,
                          double cfl, double* objective, double* grad, double* g0, int on_device, double* stats);

/* Number of kernel launches the context has enqueued since creation (instrumentation). */
long long fasw_launch_count(fasw_ctx* ctx);

/* Kernel classes for per-kernel timing. */
enum fasw_kernel_class {
  FASW_K_BC = 0, FASW_K_CELL_AUX = 1, FASW_K_RESIDUAL = 2, FASW_K_FACE_BLOCKS = 3, FASW_K_DIAG_BLOCKS = 4,
  FASW_K_SGS = 5, FASW_K_COPY = 6, FASW_K_RESTRICT = 7, FASW_K_PROLONG = 8, FASW_K_NORM = 9, FASW_K_BL = 10,
  FASW_NKERNELS = 11
};

/* enable != 0: bracket every subsequent launch with CUDA events on the context's stream and
 * accumulate per-class device time (adds an event pair per launch); resets the counters.
 * Synchronizes the stream. */
int fasw_profile(fasw_ctx* ctx, int enable);

/* Launch count and summed device milliseconds of one kernel class since fasw_profile. */
int fasw_kernel_time(fasw_ctx* ctx, int kernel, long long* count, double* total_ms);

/* Residual without any device allocation.  No counterpart in the paper: this is a service
 * for callers that cannot call cudaMalloc where they need a residual -- an application that
 * owns all device memory and gives this library fixed buffers only, or a latency-critical
 * loop that must not pay for cudaMalloc/cudaFree.
 *
 * Computes F = F^c + F^v of the finest level (same definition and layout as fasw_residual,
 * steady, zero forcing, laminar: p->turb must be 0) for an ni x nj C-grid whose vertices
 * x, y ((ni+1)*(nj+1), index j*(ni+1)+i) and state u (4 x nj x ni) are DEVICE pointers; the
 * result goes to the DEVICE buffer F (4 x nj x ni).  Work is enqueued on `stream`; the call
 * does not synchronize.
 *
 * Scratch: a fixed array of FASW_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB) compiled into the
 * library, held by every GPU that loads the library until the process exits; about
 * 7 (ni+4)(nj+4) + 20 ni nj doubles are needed (a 256 x 64 grid fits, 512 x 128 does not);
 * larger grids return FASW_ERR_TOO_LARGE.  The first call on each device looks up the array's
 * device address with that device current; make that first call before any stream capture.
 * All calls share the one array and it keeps the previous call's contents (the parts that
 * must start at zero are cleared each call): calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race and must be serialized by the caller.
 * Errors: FASW_ERR_ARG, FASW_ERR_TOO_LARGE, FASW_ERR_CUDA. */
#define FASW_NOALLOC_SCRATCH_DOUBLES 524288
int fasw_residual_noalloc(int ni, int nj, int n_wake, const double* x, const double* y, const double* u,
                          double* F, const fasw_params* p, void* stream);

/* ---- Batched cases (many independent airfoil cases of uneven size).  Each case is a context
 * on its own stream (created and owned by the batch); fasw_batch_cycle runs one FAS cycle of
 * every case as parallel branches of one captured CUDA graph launched on `stream` (NULL: the
 * batch creates a stream).  Arrays are per case (ncases entries); params[k] is case k's. */
typedef struct fasw_batch fasw_batch;
int fasw_batch_create(int ncases, const int* ni, const int* nj, const int* n_wake, const double* const* x,
                      const double* const* y, int coords_on_device, const fasw_params* params, void* stream,
                      fasw_batch** out);
void fasw_batch_destroy(fasw_batch* batch);
/* The context of case k (owned by the batch; use it for fasw_get_state / fasw_set_state). */
fasw_ctx* fasw_batch_case(fasw_batch* batch, int k);
/* One cycle of every case; norms (nullable, ncases): each case's residual norm at its start. */
int fasw_batch_cycle(fasw_batch* batch, int cycle_index, double* norms);
/* Cycles until every case has dropped its residual by `drop` or diverged; cycles[k] = cycles case
 * k needed (-1 not reached, -2 diverged: NaN or growth by 1e8; the other cases go on),
 * final_drop[k] = its last finite norm ratio, *ncycles = cycles run.  Returns FASW_OK,
 * FASW_ERR_NOT_CONVERGED or FASW_ERR_DIVERGED (some case diverged). */
int fasw_batch_solve(fasw_batch* batch, double drop, int max_cycles, int* cycles, double* final_drop, int* ncycles);
/* Picks, for every grid shape (ni, nj) and precision of the batch, the sweep variant (see
 * fasw_set_sweep) and then the residual tile height (see fasw_set_residual_tile) by timing whole
 * batch cycles: states are saved and restored; each candidate is timed beside the incumbent, the
 * faster of two timings each, and a switch must gain 2 %.  Candidates are the variants whose CTAs
 * never wait on a CTA that might not be resident beside the other cases' kernels: mixed precision
 * 7, 6, 2, 9 and 10 (the warp strips run as one thread-block cluster, which the hardware
 * schedules together); FP64 9, 10 and 2.  Tile heights 0 (size rule), 1, 2, 4, 8.  Results are cached per shape
 * and precision for the process, so a batch whose shapes are all cached is not timed again.
 * choice[k] (nullable) receives kind | (tile height << 8) for case k.  Batch cases start with
 * kind 9 (the warp strips); strip-pipelined kinds are never used inside a batch. */
int fasw_batch_autotune(fasw_batch* batch, int* choice);
long long fasw_batch_launch_count(fasw_batch* batch);

/* Verification hook for two FP64 powers the per-cell auxiliaries form by Newton's method (the
 * sensor quantity p rho^-gamma of section 2's pressure switch, and the cube root in Martinelli's
 * radius scaling), computed beside the CUDA math library on the current device: for t < n,
 * out[4t..4t+3] = (rho^-gamma of a[t] by Newton, pow(a[t], -gamma), (a[t]/b[t])^(1/3) by Newton,
 * cbrt(a[t]/b[t])).  a, b: n doubles (positive, finite); out: 4n doubles; all host pointers, or
 * device pointers with on_device = 1.  Synchronous.  FASW_ERR_ARG for n < 0 or null pointers,
 * FASW_ERR_OOM / FASW_ERR_CUDA on device failures. */
int fasw_check_math(int n, const double* a, const double* b, double* out, int on_device);

/* Coefficients of the stage loop of a scheme, Table "RK smoothers" (section 4.1): *nstages
 * (3 or 5) and alpha[k], beta[k] for k < *nstages (alpha, beta nullable, 5 doubles each).  The
 * W methods use the ARK coefficients of the same name; AW51/AW52 and ARK51/ARK52 take the
 * ARK5J betas (section 4.1), and the ARK5J beta row is read as (1, 0, 0.56, 0, 0.44).  Host
 * only (no device needed).  FASW_ERR_ARG for an unknown scheme or nstages NULL. */
int fasw_scheme_coefficients(int scheme, int* nstages, double* alpha, double* beta);

/* Failure detection without a GPU fault (no counterpart in the paper).  After
 * fasw_fault_inject_alloc(n), the library's (n+1)-th following device allocation fails on the
 * host, before cudaMalloc is called, as if the device were out of memory (FASW_ERR_OOM); n < 0
 * switches the injection off (the default).  It fires once.  fasw_live_allocations() is the
 * number of device buffers the library currently holds (every context, batch and adjoint
 * workspace), so a caller can check that a failed call released what it had allocated.  Both
 * are process-wide and host only. */
void fasw_fault_inject_alloc(long long n);
long long fasw_live_allocations(void);

/* Message for an error code; and the last CUDA error string seen by the library. */
const char* fasw_strerror(int code);
const char* fasw_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FASW_H */
