// Launchers for set-up and data-movement kernels (kernels_transfer.cu).
#pragma once
#include "fasw_internal.cuh"

namespace fasw {
// Finest-level metrics of the reference vertices rotated by phi about (xc, yc), with the face grid
// volume fluxes of the rotation rate phidot (phi = phidot = 0: the fixed grid).
cudaError_t launch_metrics_fine(const LevelDev& L, const double* x, const double* y, cudaStream_t st, int rotate = 0,
                                double phi = 0.0, double phidot = 0.0, double xc = 0.25, double yc = 0.0);
void launch_time_source(double* src, const double* un, const double* unm1, double c1, double c2, int m, cudaStream_t st);
void launch_agglomerate(const LevelDev& F, const LevelDev& C, cudaStream_t st);
cudaError_t launch_fill_state(const LevelDev& L, const double w[4], cudaStream_t st);
void launch_f2d(const float* a, double* b, int m, cudaStream_t st);
void launch_blocks_transpose(const double* a, double* b, int nf, cudaStream_t st);
}  // namespace fasw
