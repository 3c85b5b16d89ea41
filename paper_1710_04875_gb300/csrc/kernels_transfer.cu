// Grid metrics, agglomeration, FAS restriction / prolongation (section 3 of arXiv
// 1710.04875) and small data-movement kernels.
#include "fasw_internal.cuh"
#include "fasw_transfer.cuh"

namespace fasw {

namespace {

__device__ __forceinline__ int gidx(const LevelDev& L, int i, int j) { return (j + 2) * L.P + (i + 2); }
__device__ __forceinline__ bool on_cut(const LevelDev& L, int i) { return L.nw > 0 && (i < L.nw || i >= L.ni - L.nw); }

// Finest-level metrics from vertices: i-face S = (dy, -dx) along (i,j)->(i,j+1), j-face
// S = (-dy, dx) along (i,j)->(i+1,j), volume = half the cross product of the diagonals.
// The vertices are the reference vertices rotated by (cs, sn) = (cos, sin) of the pitch angle
// about (xc, yc); the grid velocity of the rigid rotation, v = phidot (-(y - yc), x - xc), is
// linear, so each face's grid volume flux is its midpoint value dotted with S.
struct Motion { double cs, sn, phidot, xc, yc; int rotate; };

__device__ __forceinline__ void vert(const double* x, const double* y, int k, const Motion& m, double& px, double& py) {
  if (!m.rotate) {  // fixed grid: the vertices as given
    px = x[k];
    py = y[k];
    return;
  }
  const double dx = x[k] - m.xc, dy = y[k] - m.yc;
  px = m.xc + m.cs * dx - m.sn * dy;
  py = m.yc + m.sn * dx + m.cs * dy;
}

__global__ void k_metrics_fine(LevelDev L, const double* x, const double* y, Motion mo) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ni = L.ni, V = ni + 1;
  auto vgx = [&](double, double py) { return -mo.phidot * (py - mo.yc); };
  auto vgy = [&](double px, double) { return mo.phidot * (px - mo.xc); };
  if (t < L.nfx) {
    const int i = t % (ni + 1), j = t / (ni + 1);
    double xa, ya, xb, yb;
    vert(x, y, j * V + i, mo, xa, ya);
    vert(x, y, (j + 1) * V + i, mo, xb, yb);
    const double dx = xb - xa, dy = yb - ya;
    L.sxi[t] = dy;
    L.sxi[L.nfx + t] = -dx;
    const double mx = 0.5 * (xa + xb), my = 0.5 * (ya + yb);
    L.vfx[t] = vgx(mx, my) * dy + vgy(mx, my) * (-dx);
  }
  if (t < L.nfe) {
    const int i = t % ni, j = t / ni;
    double xa, ya, xb, yb;
    vert(x, y, j * V + i, mo, xa, ya);
    vert(x, y, j * V + i + 1, mo, xb, yb);
    const double dx = xb - xa, dy = yb - ya;
    L.seta[t] = -dy;
    L.seta[L.nfe + t] = dx;
    const double mx = 0.5 * (xa + xb), my = 0.5 * (ya + yb);
    L.vfe[t] = vgx(mx, my) * (-dy) + vgy(mx, my) * dx;
    if (j == 0) {
      L.wvx[i] = vgx(mx, my);
      L.wvy[i] = vgy(mx, my);
    }
  }
  if (t < L.n) {
    const int i = t % ni, j = t / ni;
    double x00, y00, x10, y10, x11, y11, x01, y01, xw0, yw0, xw1, yw1;
    vert(x, y, j * V + i, mo, x00, y00);
    vert(x, y, j * V + i + 1, mo, x10, y10);
    vert(x, y, (j + 1) * V + i + 1, mo, x11, y11);
    vert(x, y, (j + 1) * V + i, mo, x01, y01);
    vert(x, y, i, mo, xw0, yw0);
    vert(x, y, i + 1, mo, xw1, yw1);
    const double d1x = x11 - x00, d1y = y11 - y00, d2x = x01 - x10, d2y = y01 - y10;
    L.vol[t] = 0.5 * (d1x * d2y - d1y * d2x);
    const double cx = 0.25 * (x00 + x10 + x11 + x01), cy = 0.25 * (y00 + y10 + y11 + y01);
    const double mx = 0.5 * (xw0 + xw1), my = 0.5 * (yw0 + yw1);
    L.wdist[t] = sqrt((cx - mx) * (cx - mx) + (cy - my) * (cy - my));
  }
}

// Coarse metrics by agglomerating 2x2 fine cells: face vectors add, volumes add.
__global__ void k_agglomerate(LevelDev F, LevelDev C) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ni = C.ni;
  if (t < C.nfx) {
    const int i = t % (ni + 1), j = t / (ni + 1);
    const int fa = (2 * j) * (F.ni + 1) + 2 * i, fb = (2 * j + 1) * (F.ni + 1) + 2 * i;
    C.sxi[t] = F.sxi[fa] + F.sxi[fb];
    C.sxi[C.nfx + t] = F.sxi[F.nfx + fa] + F.sxi[F.nfx + fb];
    C.vfx[t] = F.vfx[fa] + F.vfx[fb];
  }
  if (t < C.nfe) {
    const int i = t % ni, j = t / ni;
    const int fa = (2 * j) * F.ni + 2 * i, fb = fa + 1;
    C.seta[t] = F.seta[fa] + F.seta[fb];
    C.seta[C.nfe + t] = F.seta[F.nfe + fa] + F.seta[F.nfe + fb];
    C.vfe[t] = F.vfe[fa] + F.vfe[fb];
    if (j == 0) {
      C.wvx[i] = 0.5 * (F.wvx[2 * i] + F.wvx[2 * i + 1]);
      C.wvy[i] = 0.5 * (F.wvy[2 * i] + F.wvy[2 * i + 1]);
    }
  }
  if (t < C.n) {
    const int i = t % ni, j = t / ni;
    const int a = (2 * j) * F.ni + 2 * i, b = (2 * j + 1) * F.ni + 2 * i;
    C.vol[t] = (F.vol[a] + F.vol[a + 1]) + (F.vol[b] + F.vol[b + 1]);
  }
}

__global__ void k_fill_state(LevelDev L, double w0, double w1, double w2, double w3) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.Gn) return;
  L.u[t] = w0;
  L.u[L.Gn + t] = w1;
  L.u[2 * L.Gn + t] = w2;
  L.u[3 * L.Gn + t] = w3;
}

__global__ void k_copy_u0(LevelDev L) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int i = c % L.ni, j = c / L.ni;
  const int g = gidx(L, i, j);
#pragma unroll
  for (int k = 0; k < 4; ++k) L.u0[k * L.n + c] = L.u[k * L.Gn + g];
}

// Volume-weighted agglomeration restriction of the state and of the FAS residual (rhs),
// and of the eddy viscosity when requested; the coarse state starts at u~.
__global__ void k_restrict(LevelDev F, LevelDev C, int restrict_mut) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C.n) return;
  const int I = t % C.ni, J = t / C.ni;
  const int fi[4] = {2 * I, 2 * I + 1, 2 * I, 2 * I + 1};
  const int fj[4] = {2 * J, 2 * J, 2 * J + 1, 2 * J + 1};
  const double vc = C.vol[t];
  double au[4] = {0, 0, 0, 0}, ar[4] = {0, 0, 0, 0}, am = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int fc = fj[q] * F.ni + fi[q];
    const int fg = gidx(F, fi[q], fj[q]);
    const double w = F.vol[fc];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      au[k] += w * F.u[k * F.Gn + fg];
      ar[k] += w * F.rhs[k * F.n + fc];
    }
    am += w * F.mut[fc];
  }
  const int cg = gidx(C, I, J);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = au[k] / vc;
    C.u[k * C.Gn + cg] = v;
    C.ut[k * C.n + t] = v;
    C.rhs[k * C.n + t] = ar[k] / vc;
  }
  if (restrict_mut) C.mut[t] = am / vc;
}

// Correction u_{l-1} - u~_{l-1} at a possibly-ghost coarse cell: zero-gradient copy at the
// far field and wall, mirror across the wake cut.
__device__ __forceinline__ double coarse_delta(const LevelDev& C, int I, int J, int k) {
  int Ic = min(max(I, 0), C.ni - 1);
  int Jc;
  if (J < 0) {
    if (on_cut(C, Ic)) Ic = C.ni - 1 - Ic;
    Jc = 0;
  } else {
    Jc = min(J, C.nj - 1);
  }
  const int c = Jc * C.ni + Ic;
  return C.u[k * C.Gn + gidx(C, Ic, Jc)] - C.ut[k * C.n + c];
}

// Bilinear prolongation of the correction: 9/16, 3/16, 3/16, 1/16 of the coarse cell
// containing the fine cell and its three nearest coarse neighbours.
__global__ void k_prolong(LevelDev F, LevelDev C) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= F.n) return;
  const int i = t % F.ni, j = t / F.ni;
  const int I = i / 2, J = j / 2;
  const int I2 = (i % 2 == 0) ? I - 1 : I + 1;
  const int J2 = (j % 2 == 0) ? J - 1 : J + 1;
  const int g = gidx(F, i, j);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double a = coarse_delta(C, I, J, k), b = coarse_delta(C, I2, J, k);
    const double c = coarse_delta(C, I, J2, k), d = coarse_delta(C, I2, J2, k);
    F.u[k * F.Gn + g] += (9.0 * a + 3.0 * b + 3.0 * c + d) / 16.0;
  }
}

__global__ void k_pack(LevelDev L, const double* in, int to_ghosted, double* out) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int g = gidx(L, c % L.ni, c / L.ni);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (to_ghosted)
      L.u[k * L.Gn + g] = in[k * L.n + c];
    else
      out[k * L.n + c] = L.u[k * L.Gn + g];
  }
}

__global__ void k_f2d(const float* a, double* b, int m) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) b[t] = double(a[t]);
}

// entry-major (e * nf + f) -> face-major (f * 16 + e)
__global__ void k_blocks_transpose(const double* a, double* b, int nf) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf * 16) return;
  const int f = t / 16, e = t % 16;
  b[t] = a[e * nf + f];
}

}  // namespace

cudaError_t launch_metrics_fine(const LevelDev& L, const double* x, const double* y, cudaStream_t st, int rotate,
                                double phi, double phidot, double xc, double yc) {
  const int m = L.nfx > L.nfe ? L.nfx : L.nfe;
  Motion mo{cos(phi), sin(phi), phidot, xc, yc, rotate};
  return launch_pdl(k_metrics_fine, (m + 127) / 128, 128, 0, st, L, x, y, mo);
}

// Dual-time source of the finest level: src = c1 u^n + c2 u^(n-1)
__global__ void k_time_source(double* src, const double* un, const double* unm1, double c1, double c2, int m) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) src[t] = c1 * un[t] + (unm1 ? c2 * unm1[t] : 0.0);
}

void launch_time_source(double* src, const double* un, const double* unm1, double c1, double c2, int m, cudaStream_t st) {
  launch_pdl(k_time_source, (m + 255) / 256, 256, 0, st, src, un, unm1, c1, c2, m);
}

void launch_agglomerate(const LevelDev& F, const LevelDev& C, cudaStream_t st) {
  const int m = C.nfx > C.nfe ? C.nfx : C.nfe;
  launch_pdl(k_agglomerate, (m + 127) / 128, 128, 0, st, F, C);
}

cudaError_t launch_fill_state(const LevelDev& L, const double w[4], cudaStream_t st) {
  return launch_pdl(k_fill_state, (L.Gn + 255) / 256, 256, 0, st, L, w[0], w[1], w[2], w[3]);
}

void launch_copy_u0(const LevelDev& L, cudaStream_t st) { launch_pdl(k_copy_u0, (L.n + 255) / 256, 256, 0, st, L); }

void launch_restrict(const LevelDev& F, const LevelDev& C, int restrict_mut, cudaStream_t st) {
  launch_pdl(k_restrict, (C.n + 63) / 64, 64, 0, st, F, C, restrict_mut);
}

void launch_prolong(const LevelDev& F, const LevelDev& C, cudaStream_t st) {
  launch_pdl(k_prolong, (F.n + 63) / 64, 64, 0, st, F, C);
}

cudaError_t launch_pack(const LevelDev& L, const double* in, int to_ghosted, double* out, cudaStream_t st) {
  return launch_pdl(k_pack, (L.n + 255) / 256, 256, 0, st, L, in, to_ghosted, out);
}

void launch_f2d(const float* a, double* b, int m, cudaStream_t st) { launch_pdl(k_f2d, (m + 255) / 256, 256, 0, st, a, b, m); }

void launch_blocks_transpose(const double* a, double* b, int nf, cudaStream_t st) {
  launch_pdl(k_blocks_transpose, (nf * 16 + 255) / 256, 256, 0, st, a, b, nf);
}

}  // namespace fasw
