// Launchers of the transfer-block preparation and the SGS sweep kernels (kernels_sweep.cu).
#pragma once
#include "fasw_internal.cuh"

namespace fasw {

// SWEEP_HP: hyperplane-staged FP32 sweep with the default ring depth; SWEEP_HP4 / SWEEP_HP8: with a
// ring of 4 / 8 steps (where 8 does not fit in shared memory, 4).  SWEEP_STRIPS / STRIPS16 /
// STRIPS4: pipelined strips of 8 / 16 / 4 rows.
// SWEEP_WS: warp strips of 32 rows, operands staged by bulk copies, FP32 recurrence; in FP64
// contexts followed by one FP64 defect correction (a second FP32 sweep on the FP64 residual of
// the first), which brings the result to FP64 accuracy.
enum SweepKind {
  SWEEP_AUTO = 0, SWEEP_LEGACY = 1, SWEEP_CTA = 2, SWEEP_STRIPS = 3, SWEEP_STRIPS16 = 4,
  SWEEP_HP = 5, SWEEP_HP4 = 6, SWEEP_HP8 = 7, SWEEP_STRIPS4 = 8, SWEEP_WS = 9, SWEEP_WS8 = 10
};
inline bool is_hp(int kind) { return kind == SWEEP_HP || kind == SWEEP_HP4 || kind == SWEEP_HP8; }
// SWEEP_WS8: the warp strips staging chunks of 8 steps instead of 16 (half the shared memory, so
// that two strips, of different cases of a batch, can share an SM)
inline bool is_ws(int kind) { return kind == SWEEP_WS || kind == SWEEP_WS8; }

// kind: the resolved sweep kind of this level (SWEEP_HP writes the hyperplane-major blocks,
// SWEEP_WS also the skewed FP32 blocks of the warp strips).
void launch_sgs_prep(const LevelDev& L, int mixed, int kind, cudaStream_t st);
// Forward and backward sweep of one stage: y = (D+L)^-1 rhs, z = (D+U)^-1 D y into L.yz64 /
// L.yz32, with the stage update u = u0 - alpha z (AW) or u0 - alpha dt* z (ARK) when
// do_update.  prog: 2 * sweep_strips(L) flags, err: device error word.  Returns the number of
// kernels launched.
int launch_sweep(const LevelDev& L, int mixed, int kind, int do_update, int aw, double alpha, const double* rhs,
                 long long* prog, int* err, long long limit, cudaStream_t st, int exact_iters = 0);
int sweep_strips(const LevelDev& L);
// Warp-strip sweep (kernels_sweep_ws.cu): whether a level can use it, the sizes of its arrays
// (floats of wsF / wsB; of wsC / wsY), its strips, and one application (refine: FP64 defect
// correction in FP64 contexts; the skewed blocks come from launch_sgs_prep).  Returns the
// kernels launched.
// Warp-strip layout: strips of WS_ROWS rows, a strip's operands stored step by step (lane jl at
// step s holds cell i = s - jl), the steps padded to whole chunks of WS_K (the default staging
// chunk; kind 10 stages half-chunks of 8), WS_F4_STEP float4 of blocks per step.
constexpr int WS_ROWS = 32;
constexpr int WS_K = 16;
constexpr int WS_F4_STEP = 8 * WS_ROWS;
// steps stored per strip: the ni + R - 1 steps that hold a cell (R = min(nj, 32) rows in a
// strip: a level of fewer than 32 rows skews by its own rows only), padded to whole chunks
__host__ __device__ __forceinline__ int ws_steps(int ni, int nj) {
  const int R = nj < WS_ROWS ? nj : WS_ROWS;
  return (ni + R - 1 + WS_K - 1) / WS_K * WS_K;
}
bool ws_fits(int ni, int nj, int nw);
size_t ws_floats(int ni, int nj);
size_t ws_vec_floats(int ni, int nj);
int ws_strips(int nj);
// exact_iters > 0: that many block Gauss-Seidel corrections toward the exact (D + L + U)^-1;
// chunk: steps per staged chunk (16, or 8 for SWEEP_WS8)
int launch_ws_sweep(const LevelDev& L, int mixed, int refine, int do_update, int aw, double alpha, const double* rhs,
                    long long* prog, int* err, long long limit, cudaStream_t st, int exact_iters = 0,
                    int chunk = WS_K);
// Hyperplane-staged FP32 sweep: whether a level fits (rows, shared memory), and the entries
// (ni + nj - 1) * nj of its hyperplane-major arrays (hpF, hpB: 32 floats each; hpC, hpY: 4).
bool hp_fits(int ni, int nj, int nw);
size_t hp_floats(int ni, int nj);

}  // namespace fasw
