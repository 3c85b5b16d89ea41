// A residual entry point that never allocates device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a residual: a host
// application that owns every byte of device memory and hands plugins fixed buffers only,
// or a latency-critical loop that must not pay for cudaMalloc/cudaFree (which may
// synchronize the device).  fasw_residual_noalloc serves them: the caller passes the grid
// vertices, the state and the output buffer (all device pointers); everything else the
// kernels need (metrics, ghosted state, pressure, sensor and radii, norm partials) lives in
// the fixed array below, which every GPU that loads this library holds until the process
// exits.
#include <cstring>
#include <string>

#include "../../include/fasw.h"
#include "fasw_internal.cuh"
#include "fasw_transfer.cuh"

using namespace fasw;

namespace {

constexpr size_t kScratchDoubles = FASW_NOALLOC_SCRATCH_DOUBLES;

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

size_t round_up(size_t v) { return (v + 31) & ~size_t(31); }  // keep every sub-array 256-byte aligned

// Carve the scratch into the arrays of one level; returns the doubles needed.
size_t carve(LevelDev& L, double* base) {
  size_t off = 0;
  auto take = [&](double*& p, size_t count) {
    p = base ? base + off : nullptr;
    off += round_up(count);
  };
  take(L.u, 4 * (size_t)L.Gn);
  take(L.p, (size_t)L.Gn);
  take(L.q, (size_t)L.Gn);
  take(L.rinv, (size_t)L.Gn);
  take(L.rt, 2 * (size_t)L.n);
  take(L.dts, (size_t)L.n);
  take(L.sxi, 2 * (size_t)L.nfx);
  take(L.seta, 2 * (size_t)L.nfe);
  take(L.vol, (size_t)L.n);
  take(L.wdist, (size_t)L.n);
  take(L.mut, (size_t)L.n);
  take(L.s, 4 * (size_t)L.n);
  take(L.src, 4 * (size_t)L.n);
  take(L.norm_part, (size_t)residual_blocks(L));
  take(L.vfx, (size_t)L.nfx);
  take(L.vfe, (size_t)L.nfe);
  take(L.wvx, (size_t)L.ni);
  take(L.wvy, (size_t)L.ni);
  return off;
}

}  // namespace

extern "C" int fasw_residual_noalloc(int ni, int nj, int n_wake, const double* x, const double* y,
                                     const double* u, double* F, const fasw_params* p, void* stream) {
  if (!x || !y || !u || !F || !p) return FASW_ERR_ARG;
  if (ni < 4 || nj < 2 || n_wake < 0 || n_wake >= ni / 2 + (ni % 2) || p->turb != 0 || !(p->mach > 0.0) ||
      (p->viscous && !(p->re > 0.0)))
    return FASW_ERR_ARG;
  // The scratch need in 64-bit arithmetic from the raw sizes, before any int product of them
  // is formed: a grid that cannot fit is rejected here, whatever its size.
  {
    const unsigned long long I = (unsigned long long)ni, J = (unsigned long long)nj;
    const unsigned long long G = (I + 4) * (J + 4), n = I * J;
    const unsigned long long need = 7 * G + 20 * n + 64 * 32;  // every sub-array padded to 32 doubles
    if (need > (unsigned long long)kScratchDoubles) return FASW_ERR_TOO_LARGE;
  }
  LevelDev L;
  std::memset(&L, 0, sizeof(L));
  L.ni = ni;
  L.nj = nj;
  L.nw = n_wake;
  L.P = ni + 4;
  L.Gn = L.P * (nj + 4);
  L.n = ni * nj;
  L.nfx = (ni + 1) * nj;
  L.nfe = ni * (nj + 1);
  L.finest = 1;
  L.a_t = 0.0;
  if (carve(L, nullptr) > kScratchDoubles) return FASW_ERR_TOO_LARGE;

  // Once per device, with that device current: the host-side name of the array is not a
  // device address, so ask the runtime for it.  The first call on a device does this, so it
  // should be made before any stream capture.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FASW_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return FASW_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(addr);
  }
  carve(L, g_scratch_addr[dev]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  PhysParams ph;
  std::memset(&ph, 0, sizeof(ph));
  ph.mach = p->mach;
  ph.alpha_deg = p->alpha_deg;
  ph.re = p->re;
  ph.pr = p->pr;
  ph.prt = p->prt;
  ph.inv_re = p->re > 0.0 ? 1.0 / p->re : 0.0;
  ph.inv_pr = p->pr > 0.0 ? 1.0 / p->pr : 0.0;
  ph.inv_prt = p->prt > 0.0 ? 1.0 / p->prt : 0.0;
  ph.s_coarse = p->s_coarse;
  ph.viscous = p->viscous;
  ph.turb = 0;
  ph.sensor = p->sensor;
  ph.flux = p->flux == 1 ? 1 : 0;
  ph.d_cut = p->d_cut;
  {
    const double al = p->alpha_deg * M_PI / 180.0;
    const double pinf = 1.0 / (GAM * p->mach * p->mach);
    const double uu = cos(al), vv = sin(al);
    ph.uinf[0] = 1.0;
    ph.uinf[1] = uu;
    ph.uinf[2] = vv;
    ph.uinf[3] = pinf / (GAM - 1.0) + 0.5 * (uu * uu + vv * vv);
  }
  set_free_stream_prims(ph);

  // The scratch keeps the previous call's contents: clear what the residual reads as zero
  // (eddy viscosity, forcing, dual-time source) before use.
  if (cudaMemsetAsync(L.mut, 0, (size_t)L.n * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(L.s, 0, 4 * (size_t)L.n * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(L.src, 0, 4 * (size_t)L.n * sizeof(double), st) != cudaSuccess)
    return FASW_ERR_CUDA;
  ResArgs a;
  std::memset(&a, 0, sizeof(a));
  a.mode = RES_FULL;
  a.F = F;
  // each launch's own status: an error left by unrelated earlier work is neither reported
  // nor cleared here
  if (launch_metrics_fine(L, x, y, st) != cudaSuccess || launch_fill_state(L, ph.uinf, st) != cudaSuccess ||
      launch_pack(L, u, 1, nullptr, st) != cudaSuccess || launch_bc(L, ph, st) != cudaSuccess ||
      launch_cell_aux(L, ph, 1.0, 0, st) != cudaSuccess || launch_residual(L, ph, a, st) != cudaSuccess)
    return FASW_ERR_CUDA;
  return FASW_OK;
}
