// Internal declarations shared by the CUDA translation units of the fasw library.
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

namespace fasw {

constexpr double GAM = 1.4;

// Device view of one multigrid level (paper's numbering: level 0 coarsest).
// Ghosted arrays have two ghost layers on every side: cell (i, j), -2 <= i < ni+2,
// -2 <= j < nj+2, at (j+2)*P + (i+2) with pitch P = ni + 4.  Interior arrays hold
// cell (i, j) at j*ni + i.  Vector fields are component-major (4 planes).
// Programmatic dependent launch.  Every kernel of the library starts with pdl_entry(): it waits
// until the kernel before it on the stream has completed and its writes are visible, then lets
// the next kernel be launched, so that launch overlaps this kernel's run instead of following
// its completion.  launch_pdl() launches with the attribute that allows this overlap; without
// it griddepcontrol.wait returns at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KP, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KP>(args)...);
}

// Every device allocation of the library goes through these (fasw_api.cu): they honour the
// host-side failure injection and keep the count of live allocations.
int device_alloc(void** q, size_t bytes);
void device_free(void* q);

struct LevelDev {
  int ni, nj, nw;
  int P;        // ghost pitch ni + 4
  int Gn;       // ghosted plane size P * (nj + 4)
  int n;        // ni * nj
  int nfx;      // i-faces (ni+1)*nj
  int nfe;      // j-faces ni*(nj+1)
  int finest;   // full JST (sensor + fourth differences) on the finest level only
  int res_ty;   // residual tile height (0: chosen from the level size)
  double a_t;   // time-derivative coefficient (0 = steady)
  double* u;    // 4*Gn ghosted conservative state
  double* u0;   // 4*n  state at the start of the smoothing step
  double* fvc;  // 4*n  beta-blended F^v carry
  double* rhs;  // 4*n  stage right-hand side / FAS residual
  double* s;    // 4*n  FAS forcing
  double* ut;   // 4*n  restricted state (coarse levels)
  double* src;  // 4*n  dual-time history source (finest level)
  double* p;    // Gn   pressure (ghosted)
  double* q;    // Gn   sensor quantity (ghosted)
  double* rinv; // Gn   1/rho (ghosted), formed once per state by the cell-auxiliary kernel
  double* rt;   // 2*n  Martinelli-corrected radii (xi plane, eta plane)
  double* dts;  // n    local pseudo time step
  double* sxi;  // 2*nfx  i-face area vectors (x plane, y plane), index j*(ni+1)+i
  double* seta; // 2*nfe  j-face area vectors, index j*ni+i
  double* vol;  // n
  double* mut;  // n    eddy viscosity
  double* wdist;// n    distance to the wall-face midpoint of the column (finest level)
  double* omega;// n    vorticity magnitude scratch (finest level)
  double* coef; // n    block scale c_i
  double* blk64;   // face blocks FP64: Axp[16*nfx] Axm[16*nfx] Aep[16*nfe] Aem[16*nfe], entry-major
  double* dlu64;   // 16*n LU of D (FP64), entry-major
  double* yz64;    // 4*n sweep vector (FP64)
  float* blk32;    // FP32 copies for the mixed-precision preconditioner
  float* dlu32;
  float* yz32;
  double* norm_part;  // per-block partial sums of the residual norm
  double* tb;         // 80*n transfer blocks of the sweeps (FP64, or FP32 reinterpreted, mixed)
  double* vfx;        // nfx grid volume flux v_grid . S of the i-faces (zero on a fixed grid)
  double* vfe;        // nfe grid volume flux of the j-faces
  double* wvx;        // ni  grid velocity at the j = 0 face midpoints (moving wall)
  double* wvy;
  // hyperplane-major FP32 arrays of the staged sweep (mixed precision, levels that fit; else
  // null): entry h = (i + j) * nj + j.  hpF: G_W, G_S; hpB: H_E, H_N (32 floats per entry);
  // hpC: D^-1 r (4); hpY: forward result y (4).
  float* hpF;
  float* hpB;
  float* hpC;
  float* hpY;
  // warp-strip sweep (kernels_sweep_ws.cu; null where the level does not use it): blocks of the
  // forward (G_W, G_S) and backward (H_E, H_N) passes and their right-hand sides in the order a
  // strip consumes them, the lower wake's backward coupling blocks, the sweep results z0 and dz
  // (skewed in the backward order) and the FP64 defect vector
  float* wsF;
  float* wsB;
  float* wsC;
  float* wsY;
  float* wsCut;
  float* wsZ;
  double* wsT;
  double* wsX;  // accumulated solution of the exact-preconditioner iterations (4 per cell)
};

struct PhysParams {
  double mach, alpha_deg, re, pr, prt;
  double inv_re, inv_pr, inv_prt;  // reciprocals of re, pr, prt (set with them by the host)
  double uinf[4];
  double finf[4];  // free-stream u, v, p, a (set by the host with uinf: set_free_stream_prims)
  double s_coarse;
  int viscous, turb, sensor;
  int moving;  // grid in rigid motion: moving-wall ghosts
  int flux;    // residual face flux: 0 = JST, 1 = first-order flux-vector splitting
  double d_cut;  // eigenvalue cutoff of the flux-vector splitting (also the preconditioner's)
};

// Primitive variables of the free stream for the far-field boundary, formed once on the host.
inline void set_free_stream_prims(PhysParams& ph) {
  const double rr = 1.0 / ph.uinf[0], u = ph.uinf[1] * rr, v = ph.uinf[2] * rr;
  const double p = (GAM - 1.0) * (ph.uinf[3] - 0.5 * (ph.uinf[1] * u + ph.uinf[2] * v));
  ph.finf[0] = u;
  ph.finf[1] = v;
  ph.finf[2] = p;
  ph.finf[3] = std::sqrt(GAM * p * rr);
}

struct SchemeParams {
  int aw;        // 1 = additive W, 0 = preconditioned ARK
  int nstages;
  double alpha[5], beta[5];
  double eta, d_cut;
};

// Residual kernel modes
enum ResMode {
  RES_FULL = 0,     // F (and optionally Fc, Fv) to caller arrays
  RES_STAGE = 1,    // stage rhs with carry update
  RES_FORCING = 2,  // s = F(u) (with s excluded) + rhs (restricted residual)
  RES_FASRES = 3    // rhs = -(F)  (r_l = s_l - F_l(u_l))
};

struct ResArgs {
  int mode;
  int stage;          // 1-based stage (RES_STAGE)
  double beta;        // beta_stage
  int aw;             // scale rhs by dt* (AW)
  int want_norm;      // accumulate norm partials (stage 1 / FULL)
  int norm_all;
  double* F;          // RES_FULL outputs (may be null), interior layout
  double* Fc;
  double* Fv;
};

// ---- launchers (kernels_residual.cu)
cudaError_t launch_bc(const LevelDev& L, const PhysParams& ph, cudaStream_t st);
cudaError_t launch_cell_aux(const LevelDev& L, const PhysParams& ph, double cfl, int want_dts, cudaStream_t st);
// ghost fill and cell auxiliaries in one launch
void launch_bc_aux(const LevelDev& L, const PhysParams& ph, double cfl, int want_dts, cudaStream_t st);
cudaError_t launch_residual(const LevelDev& L, const PhysParams& ph, const ResArgs& a, cudaStream_t st);
int residual_blocks(const LevelDev& L);
int residual_blocks_max(const LevelDev& L);  // the most tiles any tile height gives (height 1)
void launch_norm_final(const LevelDev& L, int nparts, int ncomp_cells, double* out, cudaStream_t st);
void launch_bl(const LevelDev& L, const PhysParams& ph, cudaStream_t st);
// the auxiliaries' FP64 powers beside pow()/cbrt(), n values (device pointers)
void launch_check_math(int n, const double* a, const double* b, double* out, cudaStream_t st);
// per-wall-face force on the body from the j = 0 face fluxes (ghosts and auxiliaries current)
void launch_wall_force(const LevelDev& L, const PhysParams& ph, double* fx, double* fy, cudaStream_t st);

// ---- launchers (kernels_sgs.cu)
void launch_face_blocks(const LevelDev& L, const PhysParams& ph, const SchemeParams& sc, int mixed, cudaStream_t st);
void launch_diag_blocks(const LevelDev& L, const SchemeParams& sc, int mixed, cudaStream_t st);
// forward/backward sweeps; backward fuses the stage update u = u0 - alpha * z (scaled by dt* for ARK)
void launch_sgs(const LevelDev& L, const SchemeParams& sc, int mixed, int do_update, double alpha,
                const double* r_in, double* z_out, cudaStream_t st);

// ---- launchers (kernels_transfer.cu)
void launch_copy_u0(const LevelDev& L, cudaStream_t st);
void launch_restrict(const LevelDev& F, const LevelDev& C, int restrict_mut, cudaStream_t st);
void launch_prolong(const LevelDev& F, const LevelDev& C, cudaStream_t st);
cudaError_t launch_pack(const LevelDev& L, const double* interior_in, int to_ghosted, double* out, cudaStream_t st);

}  // namespace fasw
