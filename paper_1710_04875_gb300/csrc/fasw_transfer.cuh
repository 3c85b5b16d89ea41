// Launchers for set-up and data-movement kernels (kernels_transfer.cu).
#pragma once
#include "fasw_internal.cuh"

namespace fasw {
void launch_metrics_fine(const LevelDev& L, const double* x, const double* y, cudaStream_t st);
void launch_agglomerate(const LevelDev& F, const LevelDev& C, cudaStream_t st);
void launch_fill_state(const LevelDev& L, const double w[4], cudaStream_t st);
void launch_f2d(const float* a, double* b, int m, cudaStream_t st);
void launch_blocks_transpose(const double* a, double* b, int nf, cudaStream_t st);
}  // namespace fasw
