// Discrete adjoint of the residual (kernels_adjoint.cu): the Jacobian dF/du by coloured central
// differences with the eddy viscosity frozen, its products with vectors and its transpose, the
// transposed smoothing step and FAS cycle, a flexible GMRES solve of the adjoint system, and
// the vertex colouring of the transposed grid product.
#pragma once
#include <vector>

#include "fasw_internal.cuh"
#include "fasw_tangent.cuh"

namespace fasw {

// Residual stencil slots of cell (i, j): 0 the cell, 1-4 i-2, i-1, i+1, i+2, 5-8 j-2, j-1, j+1,
// j+2, 9 and 10 the wake-cut mirror cells (ni-1-i, 0) and (ni-1-i, 1).
constexpr int ADJ_SLOTS = 11;

struct AdjointMG;  // transposed linear FAS cycle: coarse levels, transfer maps, work vectors

// Preconditioners of the adjoint GMRES (fasw_adjoint_set_precond).
enum AdjPrecond {
  ADJ_STAGE_LOOP = 0,     // steps of the stage loop run on J^T (x_i = x_0 + c_i P^-T (r - J^T x_(i-1)))
  ADJ_SMOOTHER_T = 1,     // steps of the exact transpose of the primal's linearised smoothing step
  ADJ_FAS_CYCLE_T = 2,    // the exact transpose of the primal's linearised FAS cycle
  ADJ_FAS_VCYCLE_T = 3    // the same with one coarse cycle per level (V) whatever the primal's gamma
};

struct AdjointDev {
  int ni = 0, nj = 0, n = 0, ncolours = 0;
  int* nbr = nullptr;      // n * ADJ_SLOTS neighbour cell or -1
  int* col = nullptr;      // n colours
  int* rev_ptr = nullptr;  // n + 1: entries (c, s) with nbr[c][s] = d, CSR by d
  int* rev = nullptr;      // c * ADJ_SLOTS + s
  double* J = nullptr;     // n * ADJ_SLOTS * 16, block (c, s) row-major dF_c / du_nbr
  double* Jv = nullptr;    // the same for the dissipative part F^v (JST dissipation + viscous flux)
  double* Fvp = nullptr;   // 4n F^v scratch (+, -)
  double* Fvm = nullptr;
  bool finest = true;      // objective gradients only on the finest level
  double* g = nullptr;     // 2 * 4n state gradients of C_L, C_D
  double* ub = nullptr;    // 4n base state
  double* Fp = nullptr;    // 4n residual scratch (+)
  double* Fm = nullptr;    // 4n residual scratch (-)
  double* fw = nullptr;    // 4 * ni wall forces fx+, fy+, fx-, fy-
  double* parts = nullptr; // reduction partials
  double* h_parts = nullptr;  // pinned host copy of the reduced values
  double* kry = nullptr;   // (2 restart + 7) * 4n: Krylov basis V, preconditioned basis Z, work vectors
  int restart = 0;
  bool built = false;      // Jacobian assembled at the current state
  LevelDev Lp{};           // level whose transfer blocks hold the preconditioner
  double* mgs = nullptr;   // smoother work vectors (4n each): residual, preconditioner scratch
  double* mgy = nullptr;   // and output
  double* mgt = nullptr;
  double* mgz = nullptr;   // start vector of a smoothing step
  double* tbt = nullptr;   // 80n transfer blocks of the transposed couplings (D' = I, G'_W, G'_S, H'_E, H'_N)
  // FP32 transposed sweep (contexts in mixed precision): the transposed blocks in FP32, entry-major
  // (80n) and, where the level fits the hyperplane-staged sweep, hyperplane-major
  bool fp32 = false;
  float* tb32 = nullptr;
  float* yz32 = nullptr;
  float* hpF = nullptr;
  float* hpB = nullptr;
  float* hpC = nullptr;
  float* hpY = nullptr;
  long long* prog = nullptr;  // strip progress flags and device error word of the sweep (the
  int* err = nullptr;         // context's), and the bound of its waits
  long long spin_limit = 0;
  // stage coefficients of the smoother: c_i = alpha_i / eta of the primal AW scheme (the primal
  // step u - alpha_i W^-1 dt* r is u - (alpha_i / eta) P^-1 r), set with the preconditioner
  double stage_c[5] = {1.0, 0.0, 0.0, 0.0, 0.0};
  double stage_b[5] = {1.0, 1.0, 1.0, 1.0, 1.0};  // beta_i: blending of the dissipative part
  int nstages = 1;
  int precond_kind = ADJ_FAS_CYCLE_T;
  AdjointMG* mg = nullptr;  // owned (adj_release)
  // (dF/dX)^T lam by coloured differences over vertices (adj_vertex_setup)
  int nvcolours = 0;
  int* vcol = nullptr;      // (nj+1)(ni+1) vertex colours
  int* vinfl_ptr = nullptr; // CSR: the cells (index < n) and wall faces (n + i) each vertex reaches
  int* vinfl = nullptr;
  double* vx = nullptr;     // 2 x (nj+1)(ni+1) perturbed vertex coordinates
  double* vlen = nullptr;   // (nj+1)(ni+1) shortest edge at each vertex (scale of its step)
  double* mgw = nullptr;    // work vectors of the linearised smoothing step and its transpose (8 x 4n)
  int smooth_steps = 3;    // smoothing steps per application of the GMRES preconditioner
  // How the finest level's Jacobian is assembled (fasw_adjoint_set_jacobian): 1 = forward-mode
  // linearization of the residual (exact), 0 = coloured central differences of the residual.
  int jac_mode = 1;
  TanDev tan{};             // tangent arrays of the finest level (kernels_tangent.cu)
};

// Host-side stencil, colouring and reverse map; allocates the device arrays (cudaMalloc), with
// the FP32 sweep arrays when A.fp32 is set.
int adj_setup(AdjointDev& A, int ni, int nj, int nw, std::vector<void*>& allocs, cudaStream_t st);
// J and the objective gradients at the current state of L (ghosts and auxiliaries are refilled).
int adj_assemble(AdjointDev& A, const LevelDev& L, const PhysParams& ph, double h_rel, cudaStream_t st,
                 long long& launches);
void adj_apply(const AdjointDev& A, const double* v, double* out, int transpose, cudaStream_t st);
// Flexible GMRES(restart) on J^T lam = g, right-preconditioned by A.precond_kind (the transposed
// linearised FAS cycle by default, built on every level at pseudo CFL cfl; overwrites the
// levels' blocks and dt*); the preconditioned basis vectors are kept, so an FP32
// preconditioner does not limit the attainable residual.  Returns FASW_OK or
// FASW_ERR_NOT_CONVERGED; *iters, *relres.
// lev: the context's levels (the coarse ones are used by ADJ_FAS_CYCLE_T).
int adj_solve(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph, const SchemeParams& sc,
              double cfl, const double* g, double* lam, double tol, int max_iters, int restart,
              std::vector<void*>& allocs, cudaStream_t st, int* iters, double* relres, long long& launches);
// Coarse levels of the transposed FAS cycle: per-level adjoint data (stencils, colourings,
// Jacobians) and the prolongation maps; lev is the context's level list (0 = coarsest,
// lev.back() = the finest, whose data is A itself).  Allocates once.
int adj_mg_setup(AdjointDev& A, const std::vector<LevelDev>& lev, int gamma, int nu1, std::vector<void*>& allocs,
                 cudaStream_t st);
// Jacobians of every coarse level at the volume-weighted restriction of the finest state (the
// linearisation point of the FAS coarse operators); overwrites the coarse states.
int adj_mg_assemble(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph, int turb, double h_rel,
                    cudaStream_t st, long long& launches);
// z = C r (transpose = 0: the primal's linearised FAS cycle as a linear solver for J) or
// z = C^T r (transpose != 0); Jacobians and preconditioners of all levels must be current.
void adj_mg_apply(AdjointDev& A, int transpose, const double* r, double* z, cudaStream_t st);
// z = S r or S^T r for the linearised smoothing step (steps of it) of the finest level.
void adj_smoother_apply(AdjointDev& A, int steps, int transpose, const double* r, double* z, cudaStream_t st);
// Vertex colouring for the vertex gradient: every vertex reaches the cells whose residual
// depends on it (a box of 6 x 6 cells around it, and across the wake cut the cells that see the
// box through their ghosts) and the wall faces whose force does; no cell or face is reached by
// two vertices of one colour.  Allocates once.
int adj_vertex_setup(AdjointDev& A, int nw, std::vector<void*>& allocs, cudaStream_t st);
// The shortest grid edge at every vertex (A.vlen): each vertex moves by h_rel times it, so that a
// wall vertex of a stretched grid is moved by a small fraction of its first cell.
void adj_vertex_lengths(const AdjointDev& A, const double* x0, const double* y0, cudaStream_t st);
// Per vertex of colour k, direction dir: g[v] = (dC_which - lam . dF) / (2 h_rel len_v) over the
// cells and wall faces it reaches (dF = F+ - F-, dC from the wall forces fw+ / fw-).
void adj_vertex_accumulate(const AdjointDev& A, int k, int which, double sa, double ca, const double* lam,
                           const double* Fp, const double* Fm, const double* fw, double h_rel, double* g,
                           cudaStream_t st);
// xo, yo = x0, y0 moved by +-h_rel len_v in x (dir 0) or y (dir 1) at the vertices of colour k.
void adj_vertex_perturb(const AdjointDev& A, int k, int dir, double h, const double* x0, const double* y0,
                        double* xo, double* yo, cudaStream_t st);
// Host memory and the coarse levels of A.
void adj_release(AdjointDev& A);
// Lift and drag coefficients of the wall force at the current state (ghosts refilled).
int adj_force_coefficients(AdjointDev& A, const LevelDev& L, const PhysParams& ph, cudaStream_t st, double* cl,
                           double* cd, long long& launches);
// Builds the primal AW blocks of L at pseudo CFL cfl (FP64) as the adjoint preconditioner, and
// applies z = P^-T r with it (scratch: 4n).
void adj_build_precond(AdjointDev& A, const LevelDev& L, const PhysParams& ph, const SchemeParams& sc, double cfl,
                       cudaStream_t st, long long& launches);
// The same for every coarse level of the transposed FAS cycle (lev as in adj_mg_setup).
void adj_mg_build_precond(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph,
                          const SchemeParams& sc, double cfl, cudaStream_t st, long long& launches);
void adj_precond(const AdjointDev& A, const double* r, double* scratch, double* z, cudaStream_t st);
// z = P^-T r (steps <= 0) or z = `steps` transposed stage-loop steps from zero; the
// preconditioner must be built.
void adj_steps_apply(AdjointDev& A, int steps, const double* r, double* z, cudaStream_t st);
// out = x + a v (device vectors of length m).
void adj_lincomb(int m, const double* x, double a, const double* v, double* out, cudaStream_t st);
// y = a x + b y (device vectors of length m; y is read even when b = 0).
void adj_axpby(int m, double a, const double* x, double b, double* y, cudaStream_t st);
// Deterministic dot product of two device vectors of length m.
int adj_dot(AdjointDev& A, const double* a, const double* b, int m, cudaStream_t st, double* out);

}  // namespace fasw
