// Boundary ghosts, per-cell auxiliaries, the JST / thin-layer residual (section 2 of
// arXiv 1710.04875) and the Baldwin-Lomax closure, FP64.
#include "fasw_internal.cuh"
#include "fasw_roots.cuh"

namespace fasw {

namespace {

// Residual tile: TX x TY cells.  Warps 0..TY-1 compute the TX+1 = 32 i-faces of one tile row
// each, warps TY..2TY compute the TX j-faces of one row of j-faces each (lane 31 idle), so no
// warp mixes the two kinds of face and a j-face (with the viscous terms) is a thread of its
// own: on GB300 an SM sub-partition issues one FP64 warp-instruction every few dozen cycles,
// so the FP64 work of a launch is spread over as many warps and SMs as the grid allows.
// Tile height 4 where that still gives at least half as many blocks as SMs, else 1: a coarse
// level then spreads over four times as many SMs for 1.6 times the j-face work (its j-faces are
// computed by both neighbouring tiles).
constexpr int TX = 31;
constexpr int res_threads(int ty) { return 32 * (2 * ty + 1); }
// Tile height: the level's setting (1, 2, 4 or 8, chosen by the batch autotuner or the caller),
// else 4 rows where that still gives a grid of at least 76 tiles (half the SMs), else 1.
inline int res_ty(const LevelDev& L) {
  if (L.res_ty > 0) return L.res_ty;
  return ((L.ni + TX - 1) / TX) * ((L.nj + 3) / 4) >= 76 ? 4 : 1;
}

__device__ __forceinline__ int gidx(const LevelDev& L, int i, int j) { return (j + 2) * L.P + (i + 2); }
__device__ __forceinline__ bool on_cut(const LevelDev& L, int i) { return L.nw > 0 && (i < L.nw || i >= L.ni - L.nw); }

__device__ __forceinline__ void load4(const LevelDev& L, int g, double w[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = L.u[k * L.Gn + g];
}
__device__ __forceinline__ void store4(const LevelDev& L, int g, const double w[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) L.u[k * L.Gn + g] = w[k];
}

__device__ __forceinline__ double pressure(const double w[4]) {
  return (GAM - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}

// Far-field boundary state by 1-D Riemann invariants along the outward unit normal (nx, ny).
// vb: normal velocity of the (moving) boundary; in/outflow is decided on the relative velocity.
// The density follows from the entropy of the upwind side: with s = p/rho^gamma fixed,
// rho_b = (a_b^2 / (gamma s))^(1/(gamma-1)) = rho_up (a_b / a_up)^(2/(gamma-1)), and for
// gamma = 1.4 the exponent is the integer 5 (FP64 pow costs about a hundred FP64 instructions
// on a part whose FP64 issue rate is the bound of this kernel).
static_assert(GAM == 1.4, "far-field density uses 2/(gamma-1) = 5");
// The free stream's primitives (u, v, p, a) come from the host (PhysParams::finf).
__device__ void farfield(const double wi[4], const PhysParams& ph, double nx, double ny, double vb, double out[4]) {
  const double* wf = ph.uinf;
  const double ri = wi[0], rri = 1.0 / ri, ui = wi[1] * rri, vi = wi[2] * rri;
  const double pi = (GAM - 1.0) * (wi[3] - 0.5 * (wi[1] * ui + wi[2] * vi));
  const double rf = wf[0], uf = ph.finf[0], vf = ph.finf[1], af = ph.finf[3];
  const double ai = sqrt(GAM * pi * rri);
  const double vni = ui * nx + vi * ny, vnf = uf * nx + vf * ny;
  if (fabs(vni - vb) >= ai) {
    const double* src = vni - vb > 0.0 ? wi : wf;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = src[k];
    return;
  }
  constexpr double k2 = 2.0 / (GAM - 1.0);
  const double Rp = vni + k2 * ai;
  const double Rm = vnf - k2 * af;
  const double vnb = 0.5 * (Rp + Rm);
  const double ab = 0.25 * (GAM - 1.0) * (Rp - Rm);
  double rup, aup, ut, vt;
  if (vnb - vb > 0.0) {
    rup = ri;
    aup = ai;
    ut = ui - vni * nx;
    vt = vi - vni * ny;
  } else {
    rup = rf;
    aup = af;
    ut = uf - vnf * nx;
    vt = vf - vnf * ny;
  }
  const double ra = ab / aup, ra2 = ra * ra;
  const double rho = rup * (ra2 * ra2 * ra);
  const double p = rho * ab * ab * (1.0 / GAM);
  const double u = ut + vnb * nx, v = vt + vnb * ny;
  out[0] = rho;
  out[1] = rho * u;
  out[2] = rho * v;
  out[3] = p * (1.0 / (GAM - 1.0)) + 0.5 * rho * (u * u + v * v);
}

// Boundary value of ghost cell (gi, gj) (two layers on every side; corners excluded):
// j < 0: wake-cut copy of the mirror cell or wall reflection (slip / no-slip, moving wall);
// j >= nj, i < 0, i >= ni: Riemann far-field state (section 2, G9).
__device__ void ghost_state(const LevelDev& L, const PhysParams& ph, int gi, int gj, double g[4]) {
  const int ni = L.ni, nj = L.nj;
  if (gj < 0) {
    const int i = gi, k = -1 - gj;  // source row 0 or 1
    if (on_cut(L, i)) {
      load4(L, gidx(L, ni - 1 - i, k), g);
      return;
    }
    const double sx = L.seta[i], sy = L.seta[L.nfe + i];
    const double len = sqrt(sx * sx + sy * sy);
    const double nx = sx / len, ny = sy / len;
    double w[4];
    load4(L, gidx(L, i, k), w);
    if (!ph.moving) {
      g[0] = w[0];
      g[3] = w[3];
      if (ph.viscous) {
        g[1] = -w[1];
        g[2] = -w[2];
      } else {
        const double mn = w[1] * nx + w[2] * ny;
        g[1] = w[1] - 2.0 * mn * nx;
        g[2] = w[2] - 2.0 * mn * ny;
      }
    } else {  // moving wall: velocity mirrored about the wall velocity, same rho and p
      const double rho = w[0], u = w[1] / rho, v = w[2] / rho, p = pressure(w);
      const double wx = L.wvx[i], wy = L.wvy[i];
      double ug, vg;
      if (ph.viscous) {
        ug = 2.0 * wx - u;
        vg = 2.0 * wy - v;
      } else {
        const double rn = (u - wx) * nx + (v - wy) * ny;
        ug = u - 2.0 * rn * nx;
        vg = v - 2.0 * rn * ny;
      }
      g[0] = rho;
      g[1] = rho * ug;
      g[2] = rho * vg;
      g[3] = p / (GAM - 1.0) + 0.5 * rho * (ug * ug + vg * vg);
    }
    return;
  }
  double w[4];
  if (gj >= nj) {  // outward +S_eta
    const int i = gi, f = nj * ni + i;
    const double sx = L.seta[f], sy = L.seta[L.nfe + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    load4(L, gidx(L, i, nj - 1), w);
    farfield(w, ph, sx * il, sy * il, L.vfe[f] * il, g);
  } else if (gi < 0) {  // outward -S_xi
    const int j = gj, f = j * (ni + 1);
    const double sx = L.sxi[f], sy = L.sxi[L.nfx + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    load4(L, gidx(L, 0, j), w);
    farfield(w, ph, -sx * il, -sy * il, -L.vfx[f] * il, g);
  } else {  // gi >= ni, outward +S_xi
    const int j = gj, f = j * (ni + 1) + ni;
    const double sx = L.sxi[f], sy = L.sxi[L.nfx + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    load4(L, gidx(L, ni - 1, j), w);
    farfield(w, ph, sx * il, sy * il, L.vfx[f] * il, g);
  }
}

// Ghost cell t of the two layers around the domain (corners excluded): rows j = -1, -2, rows
// j = nj, nj+1, columns i = -1, -2, columns i = ni, ni+1; false past the last one.
__device__ __forceinline__ bool ghost_of(const LevelDev& L, int t, int& gi, int& gj) {
  const int ni = L.ni, nj = L.nj;
  if (t < 2 * ni) {
    gi = t % ni;
    gj = -1 - t / ni;
  } else if (t < 4 * ni) {
    gi = (t - 2 * ni) % ni;
    gj = nj + (t - 2 * ni) / ni;
  } else if (t < 4 * ni + 2 * nj) {
    gj = (t - 4 * ni) % nj;
    gi = -1 - (t - 4 * ni) / nj;
  } else if (t < 4 * ni + 4 * nj) {
    gj = (t - 4 * ni - 2 * nj) % nj;
    gi = ni + (t - 4 * ni - 2 * nj) / nj;
  } else {
    return false;
  }
  return true;
}

// Ghost fill alone: one thread per ghost cell of the two layers.
__global__ void k_bc(LevelDev L, PhysParams ph) {
  pdl_entry();
  int gi, gj;
  if (!ghost_of(L, blockIdx.x * blockDim.x + threadIdx.x, gi, gj)) return;
  double g[4];
  ghost_state(L, ph, gi, gj, g);
  store4(L, gidx(L, gi, gj), g);
}

// FP64 on this part issues one warp instruction per ~64 clocks per scheduler, and the library
// pow() costs about 3.3 us of dependent chain per call (cbrt 0.54 us, a division 0.29 us, an
// FMA 32 ns): the per-cell auxiliaries are bound by that chain, not by memory.  The two powers
// they need are computed as roots of polynomial equations by Newton's method in FP64 from an
// FP32 estimate; both are checked against pow() and cbrt() by fasw_check_math.

// Pressure, 1/rho and (finest level only: the coarse levels' dissipation has no sensor) the
// sensor quantity of one (ghosted) cell.
__device__ __forceinline__ void cell_thermo(const LevelDev& L, const PhysParams& ph, int g, const double w[4],
                                            double& rr, double& u, double& v, double& p) {
  rr = 1.0 / w[0];
  u = w[1] * rr;
  v = w[2] * rr;
  p = (GAM - 1.0) * (w[3] - 0.5 * (w[1] * u + w[2] * v));
  L.p[g] = p;
  L.rinv[g] = rr;
  if (L.finest) L.q[g] = ph.sensor ? p * pow_neg_gamma(w[0]) : p;
}

// Auxiliaries: blocks [0, nbi) take the interior cells (pressure, 1/rho, sensor quantity,
// Martinelli radii, dt*), the blocks after them the ghost cells (with fill_ghosts their
// boundary value first, which depends on interior cells only; then pressure, 1/rho, sensor).
// Interior and ghost work never share a warp, so neither path waits on the other's FP64 chain.
__global__ void k_cell_aux(LevelDev L, PhysParams ph, double cfl, int want_dts, int fill_ghosts, int nbi) {
  pdl_entry();
  if ((int)blockIdx.x >= nbi) {
    int gi, gj;
    if (!ghost_of(L, (blockIdx.x - nbi) * blockDim.x + threadIdx.x, gi, gj)) return;
    const int g = gidx(L, gi, gj);
    double w[4];
    if (fill_ghosts) {
      ghost_state(L, ph, gi, gj, w);
      store4(L, g, w);
    } else {
      load4(L, g, w);
    }
    double rr, u, v, p;
    cell_thermo(L, ph, g, w, rr, u, v, p);
    return;
  }
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  const int g = gidx(L, i, j);
  double w[4];
  load4(L, g, w);
  double rr, u, v, p;
  cell_thermo(L, ph, g, w, rr, u, v, p);
  const double a = sqrt(GAM * p * rr);
  const int fw = j * (ni + 1) + i, fs = j * ni + i;
  const double sx = 0.5 * (L.sxi[fw] + L.sxi[fw + 1]);
  const double sy = 0.5 * (L.sxi[L.nfx + fw] + L.sxi[L.nfx + fw + 1]);
  const double ex = 0.5 * (L.seta[fs] + L.seta[fs + ni]);
  const double ey = 0.5 * (L.seta[L.nfe + fs] + L.seta[L.nfe + fs + ni]);
  const double vx = 0.5 * (L.vfx[fw] + L.vfx[fw + 1]);
  const double ve = 0.5 * (L.vfe[fs] + L.vfe[fs + ni]);
  const double rxi = fabs(u * sx + v * sy - vx) + a * sqrt(sx * sx + sy * sy);
  const double reta = fabs(u * ex + v * ey - ve) + a * sqrt(ex * ex + ey * ey);
  // Martinelli scaling: with cr = (r_eta/r_xi)^(1/3), r_xi (r_eta/r_xi)^(2/3) = r_xi cr^2 and
  // r_eta (r_xi/r_eta)^(2/3) = r_xi cr (one cube root, no division).
  const double cr = cbrt_ratio(reta, rxi);
  L.rt[c] = rxi + rxi * (cr * cr);
  L.rt[L.n + c] = reta + rxi * cr;
  if (want_dts) L.dts[c] = cfl * L.vol[c] / (rxi + reta);
}

// Martinelli radius of a possibly-ghost cell: ghosts take the adjacent interior cell's value,
// across the wake cut the mirror cell's.
__device__ __forceinline__ double rt_cell(const LevelDev& L, int i, int j, int dir) {
  if (j < 0) {
    int ic = min(max(i, 0), L.ni - 1);
    i = on_cut(L, ic) ? L.ni - 1 - ic : ic;
    j = 0;
  }
  i = min(max(i, 0), L.ni - 1);
  j = min(j, L.nj - 1);
  return L.rt[dir * L.n + j * L.ni + i];
}

__device__ __forceinline__ double sensor_val(double qm, double q0, double qp) {
  return fabs(qp - 2.0 * q0 + qm) / (qp + 2.0 * q0 + qm + 0.001);
}

// JST flux through a face with area vector (sx, sy) from L to R; stencil LL, L, R, RR
// given as ghosted indices.  hc: central part; hd: dissipation d (section 2).
// On a moving face (grid volume flux vf) the convective flux is F . S - u vf.
// First-order flux-vector-split face flux (the discretization section 4.4 linearizes for the
// preconditioner): h = A+(u_bar) u_L + A-(u_bar) u_R at the mean state u_bar, with the cutoff
// eigenvalues of eq. (cutoff), split as the JST flux is (h = hc - hd): hc = A(u_bar)(u_L + u_R)/2,
// hd = (A+ - A-)(u_R - u_L)/2.  Each product uses the closed rank-2 form of R diag(l) R^-1 for
// the wave pattern (l1, l1, l3, l4): M(l) x = l1 x + r0 (g0 . x) + r1 (g1 . x) with
// r0 = (1, u, v, H), r1 = (0, nx, ny, vn), g0 = c1/a^2 dp + c2/a dvn, g1 = c2/a dp + c1 dvn,
// dp = (gamma-1)(q^2/2, -u, -v, 1), dvn = (-vn, nx, ny, 0), c1 = (l3+l4)/2 - l1, c2 = (l3-l4)/2.
__device__ __forceinline__ double fvs_cutabs(double lam, double a, double d) {
  const double al = fabs(lam), ad = a * d;
  return (d > 0.0 && al <= ad) ? 0.5 * (ad + lam * lam / ad) : al;
}

__device__ void fvs_face(const LevelDev& L, int gL, int gR, double sx, double sy, double vf, double dcut,
                         double hc[4], double hd[4]) {
  double uL[4], uR[4], ub[4], xs[4], xd[4];
  load4(L, gL, uL);
  load4(L, gR, uR);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ub[k] = 0.5 * (uL[k] + uR[k]);
    xs[k] = uL[k] + uR[k];
    xd[k] = uR[k] - uL[k];
  }
  const double g1 = GAM - 1.0;
  const double len = sqrt(sx * sx + sy * sy), rl = 1.0 / len;
  const double nx = sx * rl, ny = sy * rl;
  const double rr = 1.0 / ub[0], u = ub[1] * rr, v = ub[2] * rr;
  const double q2 = u * u + v * v;
  const double p = g1 * (ub[3] - 0.5 * ub[0] * q2);
  const double a = sqrt(GAM * p * rr), ia = 1.0 / a;
  const double H = (ub[3] + p) * rr;
  const double vn = u * nx + v * ny, vr = vn - vf * rl;
  const double r0[4] = {1.0, u, v, H}, r1[4] = {0.0, nx, ny, vn};
  const double dp[4] = {0.5 * g1 * q2, -g1 * u, -g1 * v, g1}, dv[4] = {-vn, nx, ny, 0.0};
  // M(l) x for the eigenvalue triple (l1, l3, l4), times the face length
  auto apply = [&](double l1, double l3, double l4, const double x[4], double out[4]) {
    double dpx = 0.0, dvx = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dpx += dp[k] * x[k];
      dvx += dv[k] * x[k];
    }
    const double c1 = 0.5 * (l3 + l4) - l1, c2 = 0.5 * (l3 - l4);
    const double s0 = c1 * ia * ia * dpx + c2 * ia * dvx, s1 = c2 * ia * dpx + c1 * dvx;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = len * (l1 * x[k] + r0[k] * s0 + r1[k] * s1);
  };
  apply(vr, vr + a, vr - a, xs, hc);
  apply(fvs_cutabs(vr, a, dcut), fvs_cutabs(vr + a, a, dcut), fvs_cutabs(vr - a, a, dcut), xd, hd);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hc[k] *= 0.5;
    hd[k] *= 0.5;
  }
}

__device__ void jst_face(const LevelDev& L, int gLL, int gL, int gR, int gRR, double sx, double sy, double vf,
                         double rtL, double rtR, double s_coarse, double hc[4], double hd[4]) {
  double uL[4], uR[4];
  load4(L, gL, uL);
  load4(L, gR, uR);
  const double pL = L.p[gL], pR = L.p[gR];
  {
    const double qnL = (uL[1] * sx + uL[2] * sy) * L.rinv[gL];
    const double qnR = (uR[1] * sx + uR[2] * sy) * L.rinv[gR];
    hc[0] = 0.5 * ((uL[0] * qnL - uL[0] * vf) + (uR[0] * qnR - uR[0] * vf));
    hc[1] = 0.5 * (((uL[1] * qnL + pL * sx) - uL[1] * vf) + ((uR[1] * qnR + pR * sx) - uR[1] * vf));
    hc[2] = 0.5 * (((uL[2] * qnL + pL * sy) - uL[2] * vf) + ((uR[2] * qnR + pR * sy) - uR[2] * vf));
    hc[3] = 0.5 * (((uL[3] + pL) * qnL - uL[3] * vf) + ((uR[3] + pR) * qnR - uR[3] * vf));
  }
  const double r = fmax(rtL, rtR);
  double eps2, eps4;
  if (L.finest) {
    const double qLL = L.q[gLL], qL = L.q[gL], qR = L.q[gR], qRR = L.q[gRR];
    const double sL = sensor_val(qLL, qL, qR), sR = sensor_val(qL, qR, qRR);
    const double s = fmin(0.25, fmax(sL, sR));
    eps2 = s * r;
    eps4 = fmax(0.0, r / 32.0 - 2.0 * eps2);
  } else {
    eps2 = s_coarse * r;
    eps4 = 0.0;
  }
  double uLL[4], uRR[4];
  if (eps4 != 0.0) {
    load4(L, gLL, uLL);
    load4(L, gRR, uRR);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double wL = k == 3 ? uL[3] + pL : uL[k];
    const double wR = k == 3 ? uR[3] + pR : uR[k];
    const double dw0 = wR - wL;
    double d = eps2 * dw0;
    if (eps4 != 0.0) {
      const double wLL = k == 3 ? uLL[3] + L.p[gLL] : uLL[k];
      const double wRR = k == 3 ? uRR[3] + L.p[gRR] : uRR[k];
      const double dwm = wL - wLL, dwp = wRR - wR;
      d -= eps4 * ((dwp + dwm) - 2.0 * dw0);
    }
    hd[k] = d;
  }
}

// Thin-layer viscous flux through j-face (i, j): gradients = jump across the face times S over
// the mean volume of the two cells (ghost volumes: interior neighbour; across the cut: mirror).
__device__ void visc_face(const LevelDev& L, const PhysParams& ph, int i, int j, double sx, double sy, double hv[4]) {
  const int ni = L.ni, nj = L.nj;
  double volL, volR, mutf;
  if (j == 0) {
    volR = L.vol[i];
    if (on_cut(L, i)) {
      const int m = ni - 1 - i;
      volL = L.vol[m];
      mutf = 0.5 * (L.mut[i] + L.mut[m]);
    } else {
      volL = volR;
      mutf = 0.0;
    }
  } else if (j == nj) {
    volL = L.vol[(nj - 1) * ni + i];
    volR = volL;
    mutf = L.mut[(nj - 1) * ni + i];
  } else {
    volL = L.vol[(j - 1) * ni + i];
    volR = L.vol[j * ni + i];
    mutf = 0.5 * (L.mut[(j - 1) * ni + i] + L.mut[j * ni + i]);
  }
  const double rvf = 2.0 / (volL + volR);  // 1 / mean volume
  double wL[4], wR[4];
  const int gL = gidx(L, i, j - 1), gR = gidx(L, i, j);
  load4(L, gL, wL);
  load4(L, gR, wR);
  const double rL = L.rinv[gL], rR = L.rinv[gR];
  const double uL = wL[1] * rL, vL = wL[2] * rL, uR = wR[1] * rR, vR = wR[2] * rR;
  constexpr double cp = GAM / (GAM - 1.0);
  const double hL = cp * L.p[gL] * rL, hR = cp * L.p[gR] * rR;
  const double mu = ph.inv_re;
  const double mueff = mu + mutf;
  const double keff = mu * ph.inv_pr + mutf * ph.inv_prt;
  const double sxv = sx * rvf, syv = sy * rvf;
  const double gux = (uR - uL) * sxv, guy = (uR - uL) * syv;
  const double gvx = (vR - vL) * sxv, gvy = (vR - vL) * syv;
  const double ghx = (hR - hL) * sxv, ghy = (hR - hL) * syv;
  const double div = gux + gvy;
  const double txx = mueff * (2.0 * gux - 2.0 / 3.0 * div);
  const double tyy = mueff * (2.0 * gvy - 2.0 / 3.0 * div);
  const double txy = mueff * (guy + gvx);
  const double uf = 0.5 * (uL + uR), vf = 0.5 * (vL + vR);
  const double fx = txx * sx + txy * sy, fy = txy * sx + tyy * sy;
  hv[0] = 0.0;
  hv[1] = fx;
  hv[2] = fy;
  hv[3] = uf * fx + vf * fy + keff * (ghx * sx + ghy * sy);
}

// Deterministic block sum of one double per thread (fixed shuffle tree, then warps in order).
__device__ double block_sum(double v, double* wsum) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) wsum[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) s += wsum[k];
  return s;
}

// One tile of TX x TY cells: every face of the tile is computed once into shared memory,
// then each cell assembles F^c and F^v and writes what the mode asks for.
template <int TY>
__global__ void __launch_bounds__(res_threads(TY)) k_residual(LevelDev L, PhysParams ph, ResArgs a) {
  pdl_entry();
  __shared__ double xc[4][TY][TX + 1], xd[4][TY][TX + 1];
  __shared__ double ec[4][TY + 1][TX], ed[4][TY + 1][TX];
  __shared__ double wsum[2 * TY + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int ni = L.ni, nj = L.nj;
  if (warp < TY) {  // i-face (i0 + lane, j0 + warp)
    const int tx = lane, ty = warp;
    const int i = i0 + tx, j = j0 + ty;
    if (i <= ni && j < nj) {
      const int f = j * (ni + 1) + i;
      double hc[4], hd[4];
      if (ph.flux)
        fvs_face(L, gidx(L, i - 1, j), gidx(L, i, j), L.sxi[f], L.sxi[L.nfx + f], L.vfx[f], ph.d_cut, hc, hd);
      else
        jst_face(L, gidx(L, i - 2, j), gidx(L, i - 1, j), gidx(L, i, j), gidx(L, i + 1, j), L.sxi[f],
                 L.sxi[L.nfx + f], L.vfx[f], rt_cell(L, i - 1, j, 0), rt_cell(L, i, j, 0), ph.s_coarse, hc, hd);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        xc[k][ty][tx] = hc[k];
        xd[k][ty][tx] = hd[k];
      }
    }
  } else if (lane < TX) {  // j-face (i0 + lane, j0 + warp - TY)
    const int tx = lane, ty = warp - TY;
    const int i = i0 + tx, j = j0 + ty;
    if (i < ni && j <= nj) {
      const int f = j * ni + i;
      const double sx = L.seta[f], sy = L.seta[L.nfe + f];
      double hc[4], hd[4];
      if (ph.flux)
        fvs_face(L, gidx(L, i, j - 1), gidx(L, i, j), sx, sy, L.vfe[f], ph.d_cut, hc, hd);
      else
        jst_face(L, gidx(L, i, j - 2), gidx(L, i, j - 1), gidx(L, i, j), gidx(L, i, j + 1), sx, sy, L.vfe[f],
                 rt_cell(L, i, j - 1, 1), rt_cell(L, i, j, 1), ph.s_coarse, hc, hd);
      if (ph.viscous) {
        double hv[4];
        visc_face(L, ph, i, j, sx, sy, hv);
#pragma unroll
        for (int k = 0; k < 4; ++k) hd[k] += hv[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ec[k][ty][tx] = hc[k];
        ed[k][ty][tx] = hd[k];
      }
    }
  }
  __syncthreads();
  double nacc = 0.0;
  if (warp < TY && lane < TX) {  // cell (i0 + lane, j0 + warp)
    const int tx = lane, ty = warp;
    const int i = i0 + tx, j = j0 + ty;
    if (i < ni && j < nj) {
      const int c = j * ni + i;
      const int n = L.n;
      const double rvol = 1.0 / L.vol[c];
      const int g = gidx(L, i, j);
      double Fc[4], Fv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double fc = (xc[k][ty][tx + 1] - xc[k][ty][tx]) + (ec[k][ty + 1][tx] - ec[k][ty][tx]);
        const double fd = -((xd[k][ty][tx + 1] - xd[k][ty][tx]) + (ed[k][ty + 1][tx] - ed[k][ty][tx]));
        double fcv = fc * rvol + L.a_t * L.u[k * L.Gn + g] + L.src[k * n + c];
        if (a.mode != RES_FORCING) fcv -= L.s[k * n + c];
        Fc[k] = fcv;
        Fv[k] = fd * rvol;
      }
      if (a.want_norm) {
        if (a.norm_all) {
#pragma unroll
          for (int k = 0; k < 4; ++k) nacc += (Fc[k] + Fv[k]) * (Fc[k] + Fv[k]);
        } else {
          nacc = (Fc[0] + Fv[0]) * (Fc[0] + Fv[0]);
        }
      }
      if (a.mode == RES_STAGE) {
        const double sc = a.aw ? L.dts[c] : 1.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          double carry;
          if (a.stage == 1) {
            carry = Fv[k];
          } else {
            carry = a.beta * Fv[k] + (1.0 - a.beta) * L.fvc[k * n + c];
          }
          L.fvc[k * n + c] = carry;
          L.rhs[k * n + c] = sc * (Fc[k] + carry);
        }
      } else if (a.mode == RES_FULL) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (a.F) a.F[k * n + c] = Fc[k] + Fv[k];
          if (a.Fc) a.Fc[k * n + c] = Fc[k];
          if (a.Fv) a.Fv[k * n + c] = Fv[k];
        }
      } else if (a.mode == RES_FORCING) {
#pragma unroll
        for (int k = 0; k < 4; ++k) L.s[k * n + c] = (Fc[k] + Fv[k]) + L.rhs[k * n + c];
      } else {  // RES_FASRES
#pragma unroll
        for (int k = 0; k < 4; ++k) L.rhs[k * n + c] = -(Fc[k] + Fv[k]);
      }
    }
  }
  if (a.want_norm) {
    const double s = block_sum(nacc, wsum);
    if (threadIdx.x == 0) L.norm_part[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Force on the body through each wall face (j = 0 off the wake cut): the residual's own
// j-face flux (central part minus dissipation minus viscous part) with the opposite sign,
// since the face vector points into the fluid.  fx, fy: ni entries, zero on the cut.
__global__ void k_wall_force(LevelDev L, PhysParams ph, double* fx, double* fy) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.ni) return;
  if (on_cut(L, i)) {
    fx[i] = fy[i] = 0.0;
    return;
  }
  const double sx = L.seta[i], sy = L.seta[L.nfe + i];
  double hc[4], hd[4];
  if (ph.flux)
    fvs_face(L, gidx(L, i, -1), gidx(L, i, 0), sx, sy, L.vfe[i], ph.d_cut, hc, hd);
  else
    jst_face(L, gidx(L, i, -2), gidx(L, i, -1), gidx(L, i, 0), gidx(L, i, 1), sx, sy, L.vfe[i],
             rt_cell(L, i, -1, 1), rt_cell(L, i, 0, 1), ph.s_coarse, hc, hd);
  if (ph.viscous) {
    double hv[4];
    visc_face(L, ph, i, 0, sx, sy, hv);
    for (int k = 0; k < 4; ++k) hd[k] += hv[k];
  }
  fx[i] = -(hc[1] - hd[1]);
  fy[i] = -(hc[2] - hd[2]);
}

__global__ void k_norm_final(const double* part, int nparts, double count, double* out) {
  pdl_entry();
  __shared__ double wsum[8];
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[k];
  const double t = block_sum(s, wsum);
  if (threadIdx.x == 0) out[0] = sqrt(t / count);
}

// ---- Baldwin-Lomax (finest level): vorticity by Green-Gauss, then one thread per i-line.
__global__ void k_vorticity(LevelDev L) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  const int g0 = gidx(L, i, j);
  const double u0 = L.u[L.Gn + g0] * L.rinv[g0], v0 = L.u[2 * L.Gn + g0] * L.rinv[g0];
  double fu[4], fv[4];
  const int nb[4][2] = {{i + 1, j}, {i - 1, j}, {i, j + 1}, {i, j - 1}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int g = gidx(L, nb[k][0], nb[k][1]);
    fu[k] = 0.5 * (u0 + L.u[L.Gn + g] * L.rinv[g]);
    fv[k] = 0.5 * (v0 + L.u[2 * L.Gn + g] * L.rinv[g]);
  }
  const int fe = j * (ni + 1) + i + 1, fw = j * (ni + 1) + i, fn = (j + 1) * ni + i, fs = j * ni + i;
  const double circ = (fv[0] * L.sxi[fe] - fu[0] * L.sxi[L.nfx + fe]) - (fv[1] * L.sxi[fw] - fu[1] * L.sxi[L.nfx + fw]) +
                      (fv[2] * L.seta[fn] - fu[2] * L.seta[L.nfe + fn]) - (fv[3] * L.seta[fs] - fu[3] * L.seta[L.nfe + fs]);
  L.omega[c] = fabs(circ / L.vol[c]);
}

// Baldwin-Lomax along each grid line i = const: one warp per line, lanes over j.  The search
// for F_max takes the first j of the largest F (as a sequential scan with a strict > would),
// and the inner/outer crossover is the first j where the inner value reaches the outer one.
__global__ void k_bl_lines(LevelDev L, PhysParams ph) {
  pdl_entry();
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= L.ni) return;  // whole warps leave together
  const double Aplus = 26.0, Ccp = 1.6, Ckleb = 0.3, Cwk = 0.25, kap = 0.4, Kc = 0.0168;
  const int ni = L.ni, nj = L.nj;
  const double mu = ph.inv_re;
  const bool wake = on_cut(L, i);
  const double rhow = L.u[gidx(L, i, 0)];
  const double tauw = mu * L.omega[i];
  const double utr = sqrt(rhow * tauw);
  const double yplus_scale = utr * ph.re / Aplus;  // y+ / A+ = y * utr / (mu A+)
  const int jsearch = max(1, nj / 2);
  double Fmax = 0.0, smax = 0.0, smin = 1e300;
  int jmax = 1 << 30;
  for (int j = lane; j < jsearch; j += 32) {
    const int c = j * ni + i;
    const double y = L.wdist[c];
    const double damp = wake ? 1.0 : 1.0 - exp(-y * yplus_scale);
    const double F = y * L.omega[c] * damp;
    if (F > Fmax) {  // lanes scan increasing j: keeps the first j of the lane's largest F
      Fmax = F;
      jmax = j;
    }
    const int g = gidx(L, i, j);
    const double rr = L.rinv[g], uu = L.u[L.Gn + g] * rr, vv = L.u[2 * L.Gn + g] * rr;
    const double sp = sqrt(uu * uu + vv * vv);
    smax = fmax(smax, sp);
    smin = fmin(smin, sp);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double F2 = __shfl_xor_sync(0xffffffffu, Fmax, o);
    const int j2 = __shfl_xor_sync(0xffffffffu, jmax, o);
    if (F2 > Fmax || (F2 == Fmax && j2 < jmax)) {
      Fmax = F2;
      jmax = j2;
    }
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    smin = fmin(smin, __shfl_xor_sync(0xffffffffu, smin, o));
  }
  const double ymax = Fmax > 0.0 ? L.wdist[jmax * ni + i] : 0.0;
  const double udif = wake ? smax - smin : smax;
  const double Fwake = Fmax > 0.0 ? fmin(ymax * Fmax, Cwk * ymax * udif * udif / Fmax) : 0.0;
  const double rym = ymax > 0.0 ? Ckleb / ymax : 0.0;
  int jcross = wake ? 0 : nj;
  for (int j0 = 0; j0 < nj; j0 += 32) {
    const int j = j0 + lane;
    double mo = 0.0, mi = 0.0;
    if (j < nj) {
      const int c = j * ni + i;
      const double y = L.wdist[c];
      const double rho = L.u[gidx(L, i, j)];
      const double x = y * rym, x2 = x * x;
      const double fk = ymax > 0.0 ? 1.0 / (1.0 + 5.5 * (x2 * x2 * x2)) : 0.0;
      mo = Kc * Ccp * rho * Fwake * fk;
      const double damp = wake ? 1.0 : 1.0 - exp(-y * yplus_scale);
      const double l = kap * y * damp;
      mi = rho * l * l * L.omega[c];
    }
    if (jcross == nj) {
      const unsigned hit = __ballot_sync(0xffffffffu, j < nj && mi >= mo);
      if (hit) jcross = j0 + __ffs(hit) - 1;
    }
    if (j < nj) L.mut[j * ni + i] = j >= jcross ? mo : mi;
  }
}

// The two powers of the auxiliaries beside the CUDA math library's: out[4 t ..] =
// (pow_neg_gamma(a), pow(a, -gamma), cbrt_ratio(a, b), cbrt(a / b)).
__global__ void k_check_math(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  out[4 * t + 0] = pow_neg_gamma(a[t]);
  out[4 * t + 1] = pow(a[t], -GAM);
  out[4 * t + 2] = cbrt_ratio(a[t], b[t]);
  out[4 * t + 3] = cbrt(a[t] / b[t]);
}

}  // namespace

void launch_check_math(int n, const double* a, const double* b, double* out, cudaStream_t st) {
  if (n > 0) k_check_math<<<(n + 127) / 128, 128, 0, st>>>(n, a, b, out);
}

cudaError_t launch_bc(const LevelDev& L, const PhysParams& ph, cudaStream_t st) {
  const int nt = 4 * L.ni + 4 * L.nj;
  return launch_pdl(k_bc, (nt + 63) / 64, 64, 0, st, L, ph);
}

cudaError_t launch_cell_aux(const LevelDev& L, const PhysParams& ph, double cfl, int want_dts, cudaStream_t st) {
  const int nbi = (L.n + 63) / 64, nbg = (4 * (L.ni + L.nj) + 63) / 64;
  return launch_pdl(k_cell_aux, nbi + nbg, 64, 0, st, L, ph, cfl, want_dts, 0, nbi);
}

void launch_bc_aux(const LevelDev& L, const PhysParams& ph, double cfl, int want_dts, cudaStream_t st) {
  const int nbi = (L.n + 63) / 64, nbg = (4 * (L.ni + L.nj) + 63) / 64;
  launch_pdl(k_cell_aux, nbi + nbg, 64, 0, st, L, ph, cfl, want_dts, 1, nbi);
}

void launch_wall_force(const LevelDev& L, const PhysParams& ph, double* fx, double* fy, cudaStream_t st) {
  launch_pdl(k_wall_force, (L.ni + 63) / 64, 64, 0, st, L, ph, fx, fy);
}

int residual_blocks(const LevelDev& L) {
  const int ty = res_ty(L);
  return ((L.ni + TX - 1) / TX) * ((L.nj + ty - 1) / ty);
}

cudaError_t launch_residual(const LevelDev& L, const PhysParams& ph, const ResArgs& a, cudaStream_t st) {
  const int ty = res_ty(L);
  const dim3 grid((L.ni + TX - 1) / TX, (L.nj + ty - 1) / ty);
  switch (ty) {
    case 8: return launch_pdl(k_residual<8>, grid, res_threads(8), 0, st, L, ph, a);
    case 4: return launch_pdl(k_residual<4>, grid, res_threads(4), 0, st, L, ph, a);
    case 2: return launch_pdl(k_residual<2>, grid, res_threads(2), 0, st, L, ph, a);
    default: return launch_pdl(k_residual<1>, grid, res_threads(1), 0, st, L, ph, a);
  }
}

int residual_blocks_max(const LevelDev& L) { return ((L.ni + TX - 1) / TX) * L.nj; }

void launch_norm_final(const LevelDev& L, int nparts, int ncomp_cells, double* out, cudaStream_t st) {
  launch_pdl(k_norm_final, 1, 256, 0, st, L.norm_part, nparts, (double)ncomp_cells, out);
}

void launch_bl(const LevelDev& L, const PhysParams& ph, cudaStream_t st) {
  launch_pdl(k_vorticity, (L.n + 63) / 64, 64, 0, st, L);
  launch_pdl(k_bl_lines, (L.ni + 1) / 2, 64, 0, st, L, ph);
}

}  // namespace fasw
