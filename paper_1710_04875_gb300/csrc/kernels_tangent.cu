// Forward-mode linearization of the residual of section 2 (JST or first-order flux-vector-split
// convective flux, thin-layer viscous flux, the boundary ghosts): dF = (dF/du) du at the level's
// current state, exactly (to rounding), with the eddy viscosity held at its current value.
//
// Every quantity of the residual is carried as a pair (value, derivative along du): the sums,
// products, quotients and square roots by their differentiation rules, |x|, max and min on the
// branch the value takes (the JST pressure switch, the eps4 cutoff, Martinelli's radii and the
// far-field in/outflow tests are held where the state is), and the two Newton-root powers of the
// auxiliaries by their derivatives, d(rho^-gamma) = -gamma rho^-gamma drho / rho and
// d(n/d)^(1/3) = c (dn/n - dd/d) / 3.  The value parts repeat the residual kernels' formulas in
// the same order, so they reproduce the residual itself (the tests check both parts).
//
// The pipeline per evaluation: the tangent of the interior state (a seed, or a given vector), the
// tangents of the ghost cells and the per-cell auxiliaries (pressure, 1/rho, sensor quantity,
// Martinelli radii), the face fluxes of the i- and j-faces, and the cell sums.
#include "fasw_internal.cuh"
#include "fasw_roots.cuh"
#include "fasw_tangent.cuh"

namespace fasw {

namespace {

struct Dual {
  double v, d;
};

__device__ __forceinline__ Dual cst(double v) { return Dual{v, 0.0}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual{-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual{q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual{a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual{a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual{a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual{a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual{a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual{a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual{a.v / b, a.d / b}; }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual{q, -q * b.d / b.v};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
  const double s = sqrt(a.v);
  return Dual{s, a.d / (2.0 * s)};
}
// The switches' max, min and |.| are not differentiable where their arguments tie.  A tie (the
// two arguments of max / min equal to TIE relative, or the argument of |.| zero to TIE times the
// scale of the quantities it is formed from) takes the mean of the two one-sided slopes: the
// central derivative, which central differences of the residual also give there.  Symmetric
// flows tie exactly (the sensors of mirror cells across the wake cut, the normal velocity on the
// symmetry line), so one branch taken there would give a gradient without the flow's symmetry.
constexpr double TIE = 1e-8;
__device__ __forceinline__ Dual dabs(Dual a, double scale) {
  if (fabs(a.v) <= TIE * scale) return Dual{fabs(a.v), 0.0};
  return a.v > 0.0 ? a : -a;
}
__device__ __forceinline__ Dual dmax(Dual a, Dual b) {
  if (fabs(a.v - b.v) <= TIE * fmax(fabs(a.v), fabs(b.v))) return Dual{fmax(a.v, b.v), 0.5 * (a.d + b.d)};
  return a.v > b.v ? a : b;
}
__device__ __forceinline__ Dual dmin(Dual a, Dual b) {
  if (fabs(a.v - b.v) <= TIE * fmax(fabs(a.v), fabs(b.v))) return Dual{fmin(a.v, b.v), 0.5 * (a.d + b.d)};
  return a.v < b.v ? a : b;
}
// rho^(-gamma) and (num/den)^(1/3): the residual kernels' Newton roots for the values
__device__ __forceinline__ Dual dpow_neg_gamma(Dual r) {
  const double z = pow_neg_gamma(r.v);
  return Dual{z, -GAM * z / r.v * r.d};
}
__device__ __forceinline__ Dual dcbrt_ratio(Dual num, Dual den) {
  const double c = cbrt_ratio(num.v, den.v);
  return Dual{c, c * (num.d / num.v - den.d / den.v) * (1.0 / 3.0)};
}

__device__ __forceinline__ int gix(const LevelDev& L, int i, int j) { return (j + 2) * L.P + (i + 2); }
__device__ __forceinline__ bool cut(const LevelDev& L, int i) { return L.nw > 0 && (i < L.nw || i >= L.ni - L.nw); }

// state and auxiliaries of a (ghosted) cell as pairs: values from the level, tangents from T
__device__ __forceinline__ void ld4(const LevelDev& L, const TanDev& T, int g, Dual w[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = Dual{L.u[k * L.Gn + g], T.u[k * L.Gn + g]};
}
__device__ __forceinline__ Dual P_(const LevelDev& L, const TanDev& T, int g) { return Dual{L.p[g], T.p[g]}; }
__device__ __forceinline__ Dual R_(const LevelDev& L, const TanDev& T, int g) { return Dual{L.rinv[g], T.rinv[g]}; }
__device__ __forceinline__ Dual Q_(const LevelDev& L, const TanDev& T, int g) { return Dual{L.q[g], T.q[g]}; }

__device__ __forceinline__ Dual pressure_d(const Dual w[4]) {
  return (GAM - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}

// Riemann far-field state (the residual kernels' construction; branches on the values)
__device__ void farfield_d(const Dual wi[4], const PhysParams& ph, double nx, double ny, double vb, Dual out[4]) {
  const double* wf = ph.uinf;
  const Dual ri = wi[0], rri = 1.0 / ri, ui = wi[1] * rri, vi = wi[2] * rri;
  const Dual pi = (GAM - 1.0) * (wi[3] - 0.5 * (wi[1] * ui + wi[2] * vi));
  const double rf = wf[0], uf = ph.finf[0], vf = ph.finf[1], af = ph.finf[3];
  const Dual ai = dsqrt(GAM * pi * rri);
  const Dual vni = ui * nx + vi * ny;
  const double vnf = uf * nx + vf * ny;
  if (fabs(vni.v - vb) >= ai.v) {
    if ((vni - vb).v > 0.0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) out[k] = wi[k];
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) out[k] = cst(wf[k]);
    }
    return;
  }
  constexpr double k2 = 2.0 / (GAM - 1.0);
  const Dual Rp = vni + k2 * ai;
  const double Rm = vnf - k2 * af;
  const Dual vnb = 0.5 * (Rp + Rm);
  const Dual ab = 0.25 * (GAM - 1.0) * (Rp - Rm);
  Dual rup, aup, ut, vt;
  if ((vnb - vb).v > 0.0) {
    rup = ri;
    aup = ai;
    ut = ui - vni * nx;
    vt = vi - vni * ny;
  } else {
    rup = cst(rf);
    aup = cst(af);
    ut = cst(uf - vnf * nx);
    vt = cst(vf - vnf * ny);
  }
  const Dual ra = ab / aup, ra2 = ra * ra;
  const Dual rho = rup * (ra2 * ra2 * ra);
  const Dual p = rho * ab * ab * (1.0 / GAM);
  const Dual u = ut + vnb * nx, v = vt + vnb * ny;
  out[0] = rho;
  out[1] = rho * u;
  out[2] = rho * v;
  out[3] = p * (1.0 / (GAM - 1.0)) + 0.5 * rho * (u * u + v * v);
}

// Ghost cell (gi, gj): wake-cut copy, wall reflection (slip / no-slip, moving wall) or far field.
__device__ void ghost_d(const LevelDev& L, const TanDev& T, const PhysParams& ph, int gi, int gj, Dual g[4]) {
  const int ni = L.ni, nj = L.nj;
  if (gj < 0) {
    const int i = gi, k = -1 - gj;
    if (cut(L, i)) {
      ld4(L, T, gix(L, ni - 1 - i, k), g);
      return;
    }
    const double sx = L.seta[i], sy = L.seta[L.nfe + i];
    const double len = sqrt(sx * sx + sy * sy);
    const double nx = sx / len, ny = sy / len;
    Dual w[4];
    ld4(L, T, gix(L, i, k), w);
    if (!ph.moving) {
      g[0] = w[0];
      g[3] = w[3];
      if (ph.viscous) {
        g[1] = -w[1];
        g[2] = -w[2];
      } else {
        const Dual mn = w[1] * nx + w[2] * ny;
        g[1] = w[1] - 2.0 * mn * nx;
        g[2] = w[2] - 2.0 * mn * ny;
      }
    } else {
      const Dual rho = w[0], u = w[1] / rho, v = w[2] / rho, p = pressure_d(w);
      const double wx = L.wvx[i], wy = L.wvy[i];
      Dual ug, vg;
      if (ph.viscous) {
        ug = 2.0 * wx - u;
        vg = 2.0 * wy - v;
      } else {
        const Dual rn = (u - wx) * nx + (v - wy) * ny;
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
  Dual w[4];
  if (gj >= nj) {
    const int i = gi, f = nj * ni + i;
    const double sx = L.seta[f], sy = L.seta[L.nfe + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    ld4(L, T, gix(L, i, nj - 1), w);
    farfield_d(w, ph, sx * il, sy * il, L.vfe[f] * il, g);
  } else if (gi < 0) {
    const int j = gj, f = j * (ni + 1);
    const double sx = L.sxi[f], sy = L.sxi[L.nfx + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    ld4(L, T, gix(L, 0, j), w);
    farfield_d(w, ph, -sx * il, -sy * il, -L.vfx[f] * il, g);
  } else {
    const int j = gj, f = j * (ni + 1) + ni;
    const double sx = L.sxi[f], sy = L.sxi[L.nfx + f];
    const double il = 1.0 / sqrt(sx * sx + sy * sy);
    ld4(L, T, gix(L, ni - 1, j), w);
    farfield_d(w, ph, sx * il, sy * il, L.vfx[f] * il, g);
  }
}

__device__ __forceinline__ bool ghost_at(const LevelDev& L, int t, int& gi, int& gj) {
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

// tangents of pressure, 1/rho and (finest level) the sensor quantity of one cell
__device__ __forceinline__ void thermo_d(const LevelDev& L, const TanDev& T, const PhysParams& ph, int g,
                                         const Dual w[4], Dual& rr, Dual& u, Dual& v, Dual& p) {
  rr = 1.0 / w[0];
  u = w[1] * rr;
  v = w[2] * rr;
  p = (GAM - 1.0) * (w[3] - 0.5 * (w[1] * u + w[2] * v));
  T.p[g] = p.d;
  T.rinv[g] = rr.d;
  if (L.finest) T.q[g] = ph.sensor ? (p * dpow_neg_gamma(w[0])).d : p.d;
}

// interior tangent = seed or vector: dir < 0 copies v (4n, component-major), else
// scale * max(1, |u|) at component dir of the cells of colour k
__global__ void k_tan_set(LevelDev L, TanDev T, const double* v, const int* col, int k, int dir, double scale) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, g = gix(L, c % L.ni, c / L.ni);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double t;
    if (dir < 0)
      t = v[(size_t)q * n + c];
    else
      t = (q == dir && col[c] == k) ? scale * fmax(1.0, fabs(L.u[q * L.Gn + g])) : 0.0;
    T.u[q * L.Gn + g] = t;
  }
}

// ghosts (their tangents from the interior's) and the per-cell auxiliaries' tangents
__global__ void k_tan_aux(LevelDev L, TanDev T, PhysParams ph, int nbi) {
  pdl_entry();
  if ((int)blockIdx.x >= nbi) {
    int gi, gj;
    if (!ghost_at(L, (blockIdx.x - nbi) * blockDim.x + threadIdx.x, gi, gj)) return;
    const int g = gix(L, gi, gj);
    Dual w[4];
    ghost_d(L, T, ph, gi, gj, w);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.u[k * L.Gn + g] = w[k].d;
    Dual rr, u, v, p;
    thermo_d(L, T, ph, g, w, rr, u, v, p);
    return;
  }
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  const int g = gix(L, i, j);
  Dual w[4];
  ld4(L, T, g, w);
  Dual rr, u, v, p;
  thermo_d(L, T, ph, g, w, rr, u, v, p);
  const Dual a = dsqrt(GAM * p * rr);
  const int fw = j * (ni + 1) + i, fs = j * ni + i;
  const double sx = 0.5 * (L.sxi[fw] + L.sxi[fw + 1]);
  const double sy = 0.5 * (L.sxi[L.nfx + fw] + L.sxi[L.nfx + fw + 1]);
  const double ex = 0.5 * (L.seta[fs] + L.seta[fs + ni]);
  const double ey = 0.5 * (L.seta[L.nfe + fs] + L.seta[L.nfe + fs + ni]);
  const double vx = 0.5 * (L.vfx[fw] + L.vfx[fw + 1]);
  const double ve = 0.5 * (L.vfe[fs] + L.vfe[fs + ni]);
  const double sl = sqrt(sx * sx + sy * sy), el = sqrt(ex * ex + ey * ey);
  const Dual rxi = dabs(u * sx + v * sy - vx, a.v * sl) + a * sl;
  const Dual reta = dabs(u * ex + v * ey - ve, a.v * el) + a * el;
  const Dual cr = dcbrt_ratio(reta, rxi);
  T.rt[c] = (rxi + rxi * (cr * cr)).d;
  T.rt[L.n + c] = (reta + rxi * cr).d;
}

__device__ __forceinline__ Dual rt_d(const LevelDev& L, const TanDev& T, int i, int j, int dir) {
  if (j < 0) {
    int ic = min(max(i, 0), L.ni - 1);
    i = cut(L, ic) ? L.ni - 1 - ic : ic;
    j = 0;
  }
  i = min(max(i, 0), L.ni - 1);
  j = min(j, L.nj - 1);
  const int x = dir * L.n + j * L.ni + i;
  return Dual{L.rt[x], T.rt[x]};
}

__device__ __forceinline__ Dual sensor_d(Dual qm, Dual q0, Dual qp) {
  const Dual den = qp + 2.0 * q0 + qm + 0.001;
  return dabs(qp - 2.0 * q0 + qm, den.v) / den;
}

__device__ void jst_d(const LevelDev& L, const TanDev& T, int gLL, int gL, int gR, int gRR, double sx, double sy,
                      double vf, Dual rtL, Dual rtR, double s_coarse, Dual hc[4], Dual hd[4]) {
  Dual uL[4], uR[4];
  ld4(L, T, gL, uL);
  ld4(L, T, gR, uR);
  const Dual pL = P_(L, T, gL), pR = P_(L, T, gR);
  {
    const Dual qnL = (uL[1] * sx + uL[2] * sy) * R_(L, T, gL);
    const Dual qnR = (uR[1] * sx + uR[2] * sy) * R_(L, T, gR);
    hc[0] = 0.5 * ((uL[0] * qnL - uL[0] * vf) + (uR[0] * qnR - uR[0] * vf));
    hc[1] = 0.5 * (((uL[1] * qnL + pL * sx) - uL[1] * vf) + ((uR[1] * qnR + pR * sx) - uR[1] * vf));
    hc[2] = 0.5 * (((uL[2] * qnL + pL * sy) - uL[2] * vf) + ((uR[2] * qnR + pR * sy) - uR[2] * vf));
    hc[3] = 0.5 * (((uL[3] + pL) * qnL - uL[3] * vf) + ((uR[3] + pR) * qnR - uR[3] * vf));
  }
  const Dual r = dmax(rtL, rtR);
  Dual eps2, eps4;
  if (L.finest) {
    const Dual qLL = Q_(L, T, gLL), qL = Q_(L, T, gL), qR = Q_(L, T, gR), qRR = Q_(L, T, gRR);
    const Dual sL = sensor_d(qLL, qL, qR), sR = sensor_d(qL, qR, qRR);
    const Dual s = dmin(cst(0.25), dmax(sL, sR));
    eps2 = s * r;
    eps4 = dmax(cst(0.0), r / 32.0 - 2.0 * eps2);
  } else {
    eps2 = s_coarse * r;
    eps4 = cst(0.0);
  }
  Dual uLL[4], uRR[4];
  const bool e4 = eps4.v != 0.0 || eps4.d != 0.0;
  if (e4) {
    ld4(L, T, gLL, uLL);
    ld4(L, T, gRR, uRR);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const Dual wL = k == 3 ? uL[3] + pL : uL[k];
    const Dual wR = k == 3 ? uR[3] + pR : uR[k];
    const Dual dw0 = wR - wL;
    Dual d = eps2 * dw0;
    if (e4) {
      const Dual wLL = k == 3 ? uLL[3] + P_(L, T, gLL) : uLL[k];
      const Dual wRR = k == 3 ? uRR[3] + P_(L, T, gRR) : uRR[k];
      const Dual dwm = wL - wLL, dwp = wRR - wR;
      d = d - eps4 * ((dwp + dwm) - 2.0 * dw0);
    }
    hd[k] = d;
  }
}

__device__ __forceinline__ Dual cutabs_d(Dual lam, Dual a, double d) {
  const Dual al = dabs(lam, a.v), ad = a * d;
  return (d > 0.0 && al.v <= ad.v) ? 0.5 * (ad + lam * lam / ad) : al;
}

__device__ void fvs_d(const LevelDev& L, const TanDev& T, int gL, int gR, double sx, double sy, double vf, double dcut,
                      Dual hc[4], Dual hd[4]) {
  Dual uL[4], uR[4], ub[4], xs[4], xd[4];
  ld4(L, T, gL, uL);
  ld4(L, T, gR, uR);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ub[k] = 0.5 * (uL[k] + uR[k]);
    xs[k] = uL[k] + uR[k];
    xd[k] = uR[k] - uL[k];
  }
  const double g1 = GAM - 1.0;
  const double len = sqrt(sx * sx + sy * sy), rl = 1.0 / len;
  const double nx = sx * rl, ny = sy * rl;
  const Dual rr = 1.0 / ub[0], u = ub[1] * rr, v = ub[2] * rr;
  const Dual q2 = u * u + v * v;
  const Dual p = g1 * (ub[3] - 0.5 * ub[0] * q2);
  const Dual a = dsqrt(GAM * p * rr), ia = 1.0 / a;
  const Dual H = (ub[3] + p) * rr;
  const Dual vn = u * nx + v * ny, vr = vn - vf * rl;
  const Dual r0[4] = {cst(1.0), u, v, H}, r1[4] = {cst(0.0), cst(nx), cst(ny), vn};
  const Dual dp[4] = {0.5 * g1 * q2, -g1 * u, -g1 * v, cst(g1)}, dv[4] = {-vn, cst(nx), cst(ny), cst(0.0)};
  auto apply = [&](Dual l1, Dual l3, Dual l4, const Dual x[4], Dual out[4]) {
    Dual dpx = cst(0.0), dvx = cst(0.0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dpx = dpx + dp[k] * x[k];
      dvx = dvx + dv[k] * x[k];
    }
    const Dual c1 = 0.5 * (l3 + l4) - l1, c2 = 0.5 * (l3 - l4);
    const Dual s0 = c1 * ia * ia * dpx + c2 * ia * dvx, s1 = c2 * ia * dpx + c1 * dvx;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = len * (l1 * x[k] + r0[k] * s0 + r1[k] * s1);
  };
  apply(vr, vr + a, vr - a, xs, hc);
  apply(cutabs_d(vr, a, dcut), cutabs_d(vr + a, a, dcut), cutabs_d(vr - a, a, dcut), xd, hd);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hc[k] = hc[k] * 0.5;
    hd[k] = hd[k] * 0.5;
  }
}

// thin-layer viscous flux of j-face (i, j); the eddy viscosity is a constant of the linearization
__device__ void visc_d(const LevelDev& L, const TanDev& T, const PhysParams& ph, int i, int j, double sx, double sy,
                       Dual hv[4]) {
  const int ni = L.ni, nj = L.nj;
  double volL, volR, mutf;
  if (j == 0) {
    volR = L.vol[i];
    if (cut(L, i)) {
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
  const double rvf = 2.0 / (volL + volR);
  Dual wL[4], wR[4];
  const int gL = gix(L, i, j - 1), gR = gix(L, i, j);
  ld4(L, T, gL, wL);
  ld4(L, T, gR, wR);
  const Dual rL = R_(L, T, gL), rR = R_(L, T, gR);
  const Dual uL = wL[1] * rL, vL = wL[2] * rL, uR = wR[1] * rR, vR = wR[2] * rR;
  constexpr double cp = GAM / (GAM - 1.0);
  const Dual hL = cp * P_(L, T, gL) * rL, hR = cp * P_(L, T, gR) * rR;
  const double mu = ph.inv_re;
  const double mueff = mu + mutf;
  const double keff = mu * ph.inv_pr + mutf * ph.inv_prt;
  const double sxv = sx * rvf, syv = sy * rvf;
  const Dual gux = (uR - uL) * sxv, guy = (uR - uL) * syv;
  const Dual gvx = (vR - vL) * sxv, gvy = (vR - vL) * syv;
  const Dual ghx = (hR - hL) * sxv, ghy = (hR - hL) * syv;
  const Dual div = gux + gvy;
  const Dual txx = mueff * (2.0 * gux - 2.0 / 3.0 * div);
  const Dual tyy = mueff * (2.0 * gvy - 2.0 / 3.0 * div);
  const Dual txy = mueff * (guy + gvx);
  const Dual uf = 0.5 * (uL + uR), vf = 0.5 * (vL + vR);
  const Dual fx = txx * sx + txy * sy, fy = txy * sx + tyy * sy;
  hv[0] = cst(0.0);
  hv[1] = fx;
  hv[2] = fy;
  hv[3] = uf * fx + vf * fy + keff * (ghx * sx + ghy * sy);
}

// face fluxes: 16 doubles per face, [hc value 4][hd value 4][hc tangent 4][hd tangent 4]
__device__ __forceinline__ void put_face(double* F, int nf, int f, const Dual hc[4], const Dual hd[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    F[(size_t)k * nf + f] = hc[k].v;
    F[(size_t)(4 + k) * nf + f] = hd[k].v;
    F[(size_t)(8 + k) * nf + f] = hc[k].d;
    F[(size_t)(12 + k) * nf + f] = hd[k].d;
  }
}

__global__ void k_tan_iface(LevelDev L, TanDev T, PhysParams ph) {
  pdl_entry();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= L.nfx) return;
  const int i = f % (L.ni + 1), j = f / (L.ni + 1);
  Dual hc[4], hd[4];
  if (ph.flux)
    fvs_d(L, T, gix(L, i - 1, j), gix(L, i, j), L.sxi[f], L.sxi[L.nfx + f], L.vfx[f], ph.d_cut, hc, hd);
  else
    jst_d(L, T, gix(L, i - 2, j), gix(L, i - 1, j), gix(L, i, j), gix(L, i + 1, j), L.sxi[f], L.sxi[L.nfx + f],
          L.vfx[f], rt_d(L, T, i - 1, j, 0), rt_d(L, T, i, j, 0), ph.s_coarse, hc, hd);
  put_face(T.fx, L.nfx, f, hc, hd);
}

__global__ void k_tan_jface(LevelDev L, TanDev T, PhysParams ph) {
  pdl_entry();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= L.nfe) return;
  const int i = f % L.ni, j = f / L.ni;
  const double sx = L.seta[f], sy = L.seta[L.nfe + f];
  Dual hc[4], hd[4];
  if (ph.flux)
    fvs_d(L, T, gix(L, i, j - 1), gix(L, i, j), sx, sy, L.vfe[f], ph.d_cut, hc, hd);
  else
    jst_d(L, T, gix(L, i, j - 2), gix(L, i, j - 1), gix(L, i, j), gix(L, i, j + 1), sx, sy, L.vfe[f],
          rt_d(L, T, i, j - 1, 1), rt_d(L, T, i, j, 1), ph.s_coarse, hc, hd);
  if (ph.viscous) {
    Dual hv[4];
    visc_d(L, T, ph, i, j, sx, sy, hv);
#pragma unroll
    for (int k = 0; k < 4; ++k) hd[k] = hd[k] + hv[k];
  }
  put_face(T.fe, L.nfe, f, hc, hd);
}

// cell sums: F = F^c + F^v and its tangent (values of F^c and F^v as the residual kernel forms
// them, with the time term a_t u, the history source and the forcing; tangents of the same)
__global__ void k_tan_cells(LevelDev L, TanDev T, double* dF, double* dFv, double* Fval) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, n = L.n, i = c % ni, j = c / ni;
  const int fw = j * (ni + 1) + i, fe = fw + 1, fs = j * ni + i, fn = fs + ni;
  const int g = gix(L, i, j);
  const double rvol = 1.0 / L.vol[c];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double* X = T.fx;
    const double* E = T.fe;
    const size_t cx = (size_t)k * L.nfx, dx = (size_t)(4 + k) * L.nfx, tcx = (size_t)(8 + k) * L.nfx,
                 tdx = (size_t)(12 + k) * L.nfx;
    const size_t ce = (size_t)k * L.nfe, de = (size_t)(4 + k) * L.nfe, tce = (size_t)(8 + k) * L.nfe,
                 tde = (size_t)(12 + k) * L.nfe;
    const double fc = (X[cx + fe] - X[cx + fw]) + (E[ce + fn] - E[ce + fs]);
    const double fd = -((X[dx + fe] - X[dx + fw]) + (E[de + fn] - E[de + fs]));
    const double tfc = (X[tcx + fe] - X[tcx + fw]) + (E[tce + fn] - E[tce + fs]);
    const double tfd = -((X[tdx + fe] - X[tdx + fw]) + (E[tde + fn] - E[tde + fs]));
    const double tc = tfc * rvol + L.a_t * T.u[k * L.Gn + g];
    const double tv = tfd * rvol;
    if (dF) dF[(size_t)k * n + c] = tc + tv;
    if (dFv) dFv[(size_t)k * n + c] = tv;
    if (Fval)
      Fval[(size_t)k * n + c] = (fc * rvol + L.a_t * L.u[k * L.Gn + g] + L.src[(size_t)k * n + c] -
                                 L.s[(size_t)k * n + c]) + fd * rvol;
  }
}

// tangent of the wall force of each wall face (j = 0 off the cut): -(hc - hd) of j-face (i, 0)
__global__ void k_tan_wall(LevelDev L, TanDev T, double* fx, double* fy) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.ni) return;
  if (cut(L, i)) {
    fx[i] = fy[i] = 0.0;
    return;
  }
  const size_t nf = L.nfe;
  fx[i] = -(T.fe[(8 + 1) * nf + i] - T.fe[(12 + 1) * nf + i]);
  fy[i] = -(T.fe[(8 + 2) * nf + i] - T.fe[(12 + 2) * nf + i]);
}

}  // namespace

void launch_tangent(const LevelDev& L, const TanDev& T, const PhysParams& ph, const double* v, const int* col, int k,
                    int dir, double scale, double* dF, double* dFv, double* Fval, double* wfx, double* wfy,
                    cudaStream_t st) {
  const int nb = (L.n + 127) / 128;
  launch_pdl(k_tan_set, nb, 128, 0, st, L, T, v, col, k, dir, scale);
  const int nbi = (L.n + 63) / 64, nbg = (4 * (L.ni + L.nj) + 63) / 64;
  launch_pdl(k_tan_aux, nbi + nbg, 64, 0, st, L, T, ph, nbi);
  launch_pdl(k_tan_iface, (L.nfx + 127) / 128, 128, 0, st, L, T, ph);
  launch_pdl(k_tan_jface, (L.nfe + 127) / 128, 128, 0, st, L, T, ph);
  launch_pdl(k_tan_cells, nb, 128, 0, st, L, T, dF, dFv, Fval);
  if (wfx) launch_pdl(k_tan_wall, (L.ni + 127) / 128, 128, 0, st, L, T, wfx, wfy);
}

size_t tangent_doubles(const LevelDev& L) {
  auto r = [](size_t v) { return (v + 31) & ~size_t(31); };  // every array 256-byte aligned
  return r(4 * (size_t)L.Gn) + 3 * r((size_t)L.Gn) + r(2 * (size_t)L.n) + r(16 * (size_t)L.nfx) +
         r(16 * (size_t)L.nfe);
}

void tangent_carve(const LevelDev& L, double* base, TanDev& T) {
  size_t off = 0;
  auto take = [&](double*& p, size_t count) {
    p = base + off;
    off += (count + 31) & ~size_t(31);
  };
  take(T.u, 4 * (size_t)L.Gn);
  take(T.p, (size_t)L.Gn);
  take(T.q, (size_t)L.Gn);
  take(T.rinv, (size_t)L.Gn);
  take(T.rt, 2 * (size_t)L.n);
  take(T.fx, 16 * (size_t)L.nfx);
  take(T.fe, 16 * (size_t)L.nfe);
}

}  // namespace fasw
