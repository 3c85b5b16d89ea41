// Forward-mode linearization of the residual (kernels_tangent.cu).
#pragma once
#include "fasw_internal.cuh"

namespace fasw {

// Tangent arrays of one level, laid out like the level's own: the ghosted state (4 Gn), pressure,
// sensor quantity and 1/rho (Gn each), the Martinelli radii (2n), and the face fluxes of the
// i- and j-faces (16 per face: values and tangents of the central part and the dissipation).
struct TanDev {
  double* u;
  double* p;
  double* q;
  double* rinv;
  double* rt;
  double* fx;
  double* fe;
};

// One evaluation at the level's current state (ghosts and auxiliaries current): the interior
// tangent is v (4n, component-major; dir < 0) or the seed scale * max(1, |u|) at component dir of
// the cells of colour k; then dF = (dF/du) du (dF^v, its dissipative part, and Fval, the residual
// itself, each nullable), and with wfx / wfy (nullable) the tangent of the wall force.
void launch_tangent(const LevelDev& L, const TanDev& T, const PhysParams& ph, const double* v, const int* col, int k,
                    int dir, double scale, double* dF, double* dFv, double* Fval, double* wfx, double* wfy,
                    cudaStream_t st);
size_t tangent_doubles(const LevelDev& L);
void tangent_carve(const LevelDev& L, double* base, TanDev& T);

}  // namespace fasw
