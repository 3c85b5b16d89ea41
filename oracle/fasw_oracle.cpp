// Oracle: plain, slow, single-threaded FP64 reference solver for the method of
// Birken, Bull & Jameson, "Preconditioned smoothers for the full approximation
// scheme for the RANS equations" (arXiv 1710.04875).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark may load this library.  It shares no code,
// header or constant with the CUDA library; the two meet only in the seeded
// synthetic grids.
//
// It follows the paper's steps in its own order and notation:
//   section 2     governing equations, JST flux (eqs. e2, e4, spectralcorrection),
//                 far-field/wall boundary conditions, BDF2 (eq. nonlin-eq),
//                 steady system (eq. nonlin-eq-steady)
//   section 3     FAS cycle, volume-weighted agglomeration restriction,
//                 bilinear prolongation, coarse equation (eq. coarse-nonlin-eq)
//   section 4.1-2 low-storage additive RK / additive W stage loop (eqs. stage
//                 derivatives 1-3 and the low-storage form of eq. additive W)
//   section 4.4   flux-vector-split Jacobians at face-averaged states with the
//                 parabolic eigenvalue cutoff (eq. cutoff), blocks of eqs.
//                 d-l-u-matrices-J / d-l-u-matrices-W, block SGS (eq. sgs-precon)
// Readings of points the paper leaves open are listed in the design notes
// (G-readings); the ones that change arithmetic are restated at their use.
//
// Deliberately naive choices (the point is that a reader can check them):
//   * flux-vector-split blocks are formed as R diag(lambda+-) R^{-1} from the
//     textbook eigenvectors, not from a closed form;
//   * 4x4 diagonal solves redo Gaussian elimination every time;
//   * the SGS sweep is a lexicographic loop (j outer, i inner);
//   * an independent dense path assembles (D+L) D^{-1} (D+U) and solves it
//     with partially pivoted LU (used by tests on tiny grids).
//
// The Baldwin-Lomax closure is pinned by closed forms (linear shear over a
// plate and across the wake cut, where every discrete step is exact) and by
// the model's exact similarity laws (velocity, density and length scalings).

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

namespace orc {

constexpr double GAM = 1.4;
template <class T> using V4T = std::array<T, 4>;
template <class T> using M4T = std::array<std::array<T, 4>, 4>;
using V4 = V4T<double>;
using M4 = M4T<double>;
using CX = std::complex<double>;

// The residual's functions are written once for a scalar type T: double (the oracle itself) or
// std::complex<double> (the complex-step derivative, Squire & Trapp 1998: F(u + i h v) =
// F(u) + i h (dF/du) v + O(h^2) with no subtractive cancellation).  Comparisons and branches take
// the real part; |x| takes the sign of the real part.  For double these are the plain operations.
inline double re(double x) { return x; }
inline double re(const CX& x) { return x.real(); }
inline double absr(double x) { return std::fabs(x); }
inline CX absr(const CX& x) { return x.real() < 0.0 ? -x : x; }
inline double maxr(double a, double b) { return std::max(a, b); }
inline CX maxr(const CX& a, const CX& b) { return a.real() < b.real() ? b : a; }
inline double minr(double a, double b) { return std::min(a, b); }
inline CX minr(const CX& a, const CX& b) { return b.real() < a.real() ? b : a; }

// ---------------------------------------------------------------- parameters
struct OrParams {
  int scheme;          // 0 = additive W (AW), 1 = preconditioned additive RK (ARK)
  int nstages;         // s
  double alpha[5];     // alpha_1..alpha_s
  double beta[5];      // beta_1..beta_s (beta_1 == 1)
  int nlevels;         // multigrid levels (1 = single grid)
  int gamma_cycle;     // 1 = V-cycle, 2 = W-cycle
  int nu1;             // presmoothing steps per level visit
  int viscous;         // 0 = Euler, 1 = thin-layer Navier-Stokes
  int turb;            // 0 = laminar, 1 = Baldwin-Lomax
  int sensor;          // 0 = pressure sensor, 1 = entropy sensor
  double mach, alpha_deg, re, pr, prt;
  double eta;          // W-method parameter
  double d_cut;        // eigenvalue cutoff fraction d
  double cfl;          // c*
  double cfl_ramp;     // c* cap for the first ramp_cycles cycles
  int ramp_cycles;
  double s_coarse;     // constant sensor value on coarse levels (first-order JST)
  double dt_phys;      // physical time step (0 = steady)
  int bdf_order;       // 1 = implicit Euler, 2 = BDF2
  int norm_all;        // 0 = density RMS, 1 = RMS over 4 components
  int flux;            // residual face flux: 0 = JST (section 2), 1 = first-order flux-vector splitting
  int precond;         // smoother preconditioner: 0 = SGS (D+L) D^-1 (D+U), 1 = exact D+L+U (dense)
};

// ---------------------------------------------------------------- gas model
template <class T> struct PrimT { T rho, u, v, p; };
using Prim = PrimT<double>;

template <class T> static PrimT<T> prim(const V4T<T>& w) {
  PrimT<T> q;
  q.rho = w[0];
  q.u = w[1] / w[0];
  q.v = w[2] / w[0];
  q.p = (GAM - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
  return q;
}

// Free stream: rho = 1, |v| = 1, a = 1/M, p = 1/(gamma M^2).
static V4 free_stream(double mach, double alpha_deg) {
  const double al = alpha_deg * M_PI / 180.0;
  const double p = 1.0 / (GAM * mach * mach);
  const double u = std::cos(al), v = std::sin(al);
  return V4{1.0, u, v, p / (GAM - 1.0) + 0.5 * (u * u + v * v)};
}

// Convective flux F^c_1 Sx + F^c_2 Sy (section 2; G1: third row rho v_i v_2 + p delta_i2).
template <class T> static V4T<T> conv_flux(const V4T<T>& w, double sx, double sy) {
  const PrimT<T> q = prim(w);
  const T qn = q.u * sx + q.v * sy;
  V4T<T> f;
  f[0] = q.rho * qn;
  f[1] = w[1] * qn + q.p * sx;
  f[2] = w[2] * qn + q.p * sy;
  f[3] = (w[3] + q.p) * qn;
  return f;
}

// ---------------------------------------------------------------- small dense algebra
static V4 matvec(const M4& A, const V4& x) {
  V4 y{};
  for (int r = 0; r < 4; ++r) {
    double s = 0.0;
    for (int c = 0; c < 4; ++c) s += A[r][c] * x[c];
    y[r] = s;
  }
  return y;
}

template <class T> static M4T<T> matmul(const M4T<T>& A, const M4T<T>& B) {
  M4T<T> C{};
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      T s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[r][k] * B[k][c];
      C[r][c] = s;
    }
  return C;
}

// Solve A x = b by Gaussian elimination without pivoting (G28).
static V4 solve4(const M4& Ain, const V4& bin) {
  M4 A = Ain;
  V4 b = bin;
  for (int k = 0; k < 4; ++k) {
    for (int r = k + 1; r < 4; ++r) {
      const double m = A[r][k] / A[k][k];
      for (int c = k; c < 4; ++c) A[r][c] -= m * A[k][c];
      b[r] -= m * b[k];
    }
  }
  V4 x{};
  for (int r = 3; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < 4; ++c) s -= A[r][c] * x[c];
    x[r] = s / A[r][r];
  }
  return x;
}

// ---------------------------------------------------------------- flux-vector splitting
// Parabolic cutoff of eq. (cutoff): |lambda| -> (ad + lambda^2/(ad))/2 for |lambda| <= ad.
// d = 0 leaves |lambda| unchanged (G26).
template <class T> static T cutoff_abs(const T& lam, const T& a, double d) {
  const T al = absr(lam);
  const T ad = a * d;
  if (d > 0.0 && re(al) <= re(ad)) return 0.5 * (ad + lam * lam / ad);
  return al;
}

// Right eigenvectors R (columns) and R^{-1} of A_n = dF.n/du at state w, unit normal n.
template <class T>
static void eigvecs(const V4T<T>& w, double nx, double ny, M4T<T>& R, M4T<T>& Ri, T& vn, T& a) {
  const PrimT<T> q = prim(w);
  const T H = (w[3] + q.p) / q.rho;
  a = std::sqrt(GAM * q.p / q.rho);
  vn = q.u * nx + q.v * ny;
  const double tx = -ny, ty = nx;
  const T vt = q.u * tx + q.v * ty;
  const T q2 = q.u * q.u + q.v * q.v;
  const double g1 = GAM - 1.0;
  // columns: entropy, shear, acoustic +, acoustic -
  const T cols[4][4] = {
      {1.0, q.u, q.v, 0.5 * q2},
      {0.0, tx, ty, vt},
      {1.0, q.u + a * nx, q.v + a * ny, H + a * vn},
      {1.0, q.u - a * nx, q.v - a * ny, H - a * vn}};
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) R[r][c] = cols[c][r];
  const T a2 = a * a;
  const T rows[4][4] = {
      {1.0 - g1 * q2 / (2.0 * a2), g1 * q.u / a2, g1 * q.v / a2, -g1 / a2},
      {-vt, tx, ty, 0.0},
      {(g1 * q2 / 2.0 - a * vn) / (2.0 * a2), (-g1 * q.u + a * nx) / (2.0 * a2),
       (-g1 * q.v + a * ny) / (2.0 * a2), g1 / (2.0 * a2)},
      {(g1 * q2 / 2.0 + a * vn) / (2.0 * a2), (-g1 * q.u - a * nx) / (2.0 * a2),
       (-g1 * q.v - a * ny) / (2.0 * a2), g1 / (2.0 * a2)}};
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Ri[r][c] = rows[r][c];
}

// A^+ = R diag((lambda + |lambda|_cut)/2) R^{-1}, A^- = R diag((lambda - |lambda|_cut)/2) R^{-1}
// (section 4.4), each multiplied by the face length |S|.
// On a moving face with grid volume flux vf (= v_grid . S) the eigenvalues are shifted by
// -vf/|S| (relative normal velocity); the eigenvectors are those of the fixed face.
template <class T>
static void split_jacobians(const V4T<T>& w, double sx, double sy, double vf, double d, M4T<T>& Ap, M4T<T>& Am) {
  const double len = std::sqrt(sx * sx + sy * sy);
  const double nx = sx / len, ny = sy / len;
  M4T<T> R, Ri;
  T vn, a;
  eigvecs(w, nx, ny, R, Ri, vn, a);
  const T vr = vn - vf / len;
  const T lam[4] = {vr, vr, vr + a, vr - a};
  M4T<T> Lp{}, Lm{};
  for (int k = 0; k < 4; ++k) {
    const T ab = cutoff_abs(lam[k], a, d);
    Lp[k][k] = 0.5 * (lam[k] + ab) * len;
    Lm[k][k] = 0.5 * (lam[k] - ab) * len;
  }
  Ap = matmul(matmul(R, Lp), Ri);
  Am = matmul(matmul(R, Lm), Ri);
}

// ---------------------------------------------------------------- grid levels
struct Level {
  int ni = 0, nj = 0, nw = 0;
  std::vector<double> sxi_x, sxi_y;    // i-faces, (ni+1)*nj, index j*(ni+1)+i; area vector towards +i
  std::vector<double> seta_x, seta_y;  // j-faces, ni*(nj+1), index j*ni+i; area vector towards +j
  std::vector<double> vol;             // ni*nj
  std::vector<double> wdist;           // distance of cell centroid to its j=0 face midpoint (finest)
  std::vector<double> vfx, vfe;        // grid volume flux v_grid . S of each face (zero on a fixed grid)
  std::vector<double> wvx, wvy;        // grid velocity at the j=0 face midpoints (moving wall)
  std::vector<V4> u;                   // ghosted state, (ni+4)*(nj+4)
  std::vector<V4> ut;                  // restricted state u~ (coarse levels), interior
  std::vector<V4> s;                   // FAS forcing s_l, interior (zero on the finest level)
  std::vector<V4> src;                 // dual-time history source (finest level), interior
  std::vector<double> mut;             // eddy viscosity, interior
  double a_t = 0.0;                    // coefficient of u in the time derivative (0 = steady)
  // frozen per smoothing step
  std::vector<double> dts;             // local pseudo time step
  std::vector<M4> Axp, Axm, Aep, Aem;  // split face Jacobians (times |S|)
  std::vector<M4> D;                   // diagonal blocks
  std::vector<double> coef;            // c_i multiplying the face blocks

  int G(int i, int j) const { return (j + 2) * (ni + 4) + (i + 2); }
  int C(int i, int j) const { return j * ni + i; }
  int FX(int i, int j) const { return j * (ni + 1) + i; }
  int FE(int i, int j) const { return j * ni + i; }
  bool cut(int i) const { return nw > 0 && (i < nw || i >= ni - nw); }
  int mirror(int i) const { return ni - 1 - i; }
};

struct Solver {
  OrParams P{};
  std::vector<Level> lev;   // lev[0] = coarsest, lev[L] = finest (paper's numbering)
  V4 uinf{};
  double norm_first = 0.0;  // residual norm recorded at the first stage of the finest smoothing step
  bool record_norm = false;
  // rigid motion of the whole grid (pitching): rotation by phi about (xc, yc) at rate phidot
  std::vector<double> x0, y0;
  double xc = 0.25, yc = 0.0, phi = 0.0, phidot = 0.0;
  bool moving = false;
  std::vector<V4> un, unm1;  // dual-time history of the finest level (interior)
  int steps_done = 0;
  int L() const { return (int)lev.size() - 1; }
};

static void fine_metrics(Level& g, const double* x, const double* y, double phidot = 0.0, double xc = 0.0,
                         double yc = 0.0) {
  const int ni = g.ni, nj = g.nj;
  auto X = [&](int i, int j) { return x[j * (ni + 1) + i]; };
  auto Y = [&](int i, int j) { return y[j * (ni + 1) + i]; };
  g.sxi_x.assign((ni + 1) * nj, 0.0);
  g.sxi_y.assign((ni + 1) * nj, 0.0);
  g.seta_x.assign(ni * (nj + 1), 0.0);
  g.seta_y.assign(ni * (nj + 1), 0.0);
  g.vol.assign(ni * nj, 0.0);
  g.wdist.assign(ni * nj, 0.0);
  g.vfx.assign((ni + 1) * nj, 0.0);
  g.vfe.assign(ni * (nj + 1), 0.0);
  g.wvx.assign(ni, 0.0);
  g.wvy.assign(ni, 0.0);
  // rigid rotation: v_grid(x, y) = phidot (-(y - yc), x - xc); linear, so its flux through a
  // straight face is its value at the face midpoint dotted with S
  auto vgx = [&](double, double py) { return -phidot * (py - yc); };
  auto vgy = [&](double px, double) { return phidot * (px - xc); };
  // i-face from vertex (i,j) to (i,j+1): S = (dy, -dx)
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i <= ni; ++i) {
      const double dx = X(i, j + 1) - X(i, j), dy = Y(i, j + 1) - Y(i, j);
      g.sxi_x[g.FX(i, j)] = dy;
      g.sxi_y[g.FX(i, j)] = -dx;
      const double mx = 0.5 * (X(i, j) + X(i, j + 1)), my = 0.5 * (Y(i, j) + Y(i, j + 1));
      g.vfx[g.FX(i, j)] = vgx(mx, my) * dy + vgy(mx, my) * (-dx);
    }
  // j-face from vertex (i,j) to (i+1,j): S = (-dy, dx)
  for (int j = 0; j <= nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const double dx = X(i + 1, j) - X(i, j), dy = Y(i + 1, j) - Y(i, j);
      g.seta_x[g.FE(i, j)] = -dy;
      g.seta_y[g.FE(i, j)] = dx;
      const double mx = 0.5 * (X(i, j) + X(i + 1, j)), my = 0.5 * (Y(i, j) + Y(i + 1, j));
      g.vfe[g.FE(i, j)] = vgx(mx, my) * (-dy) + vgy(mx, my) * dx;
      if (j == 0) {
        g.wvx[i] = vgx(mx, my);
        g.wvy[i] = vgy(mx, my);
      }
    }
  // volume: half the cross product of the diagonals
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const double d1x = X(i + 1, j + 1) - X(i, j), d1y = Y(i + 1, j + 1) - Y(i, j);
      const double d2x = X(i, j + 1) - X(i + 1, j), d2y = Y(i, j + 1) - Y(i + 1, j);
      g.vol[g.C(i, j)] = 0.5 * (d1x * d2y - d1y * d2x);
      const double cx = 0.25 * (X(i, j) + X(i + 1, j) + X(i + 1, j + 1) + X(i, j + 1));
      const double cy = 0.25 * (Y(i, j) + Y(i + 1, j) + Y(i + 1, j + 1) + Y(i, j + 1));
      const double mx = 0.5 * (X(i, 0) + X(i + 1, 0)), my = 0.5 * (Y(i, 0) + Y(i + 1, 0));
      g.wdist[g.C(i, j)] = std::sqrt((cx - mx) * (cx - mx) + (cy - my) * (cy - my));
    }
}

// Coarse level by agglomerating 2x2 fine cells (section 3): a coarse face is the
// union of two fine faces (area vectors add), a coarse volume the sum of four.
static void agglomerate(const Level& f, Level& c) {
  c.ni = f.ni / 2;
  c.nj = f.nj / 2;
  c.nw = f.nw / 2;
  const int ni = c.ni, nj = c.nj;
  c.sxi_x.assign((ni + 1) * nj, 0.0);
  c.sxi_y.assign((ni + 1) * nj, 0.0);
  c.seta_x.assign(ni * (nj + 1), 0.0);
  c.seta_y.assign(ni * (nj + 1), 0.0);
  c.vol.assign(ni * nj, 0.0);
  c.vfx.assign((ni + 1) * nj, 0.0);
  c.vfe.assign(ni * (nj + 1), 0.0);
  c.wvx.assign(ni, 0.0);
  c.wvy.assign(ni, 0.0);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i <= ni; ++i) {
      c.vfx[c.FX(i, j)] = f.vfx[f.FX(2 * i, 2 * j)] + f.vfx[f.FX(2 * i, 2 * j + 1)];
      c.sxi_x[c.FX(i, j)] = f.sxi_x[f.FX(2 * i, 2 * j)] + f.sxi_x[f.FX(2 * i, 2 * j + 1)];
      c.sxi_y[c.FX(i, j)] = f.sxi_y[f.FX(2 * i, 2 * j)] + f.sxi_y[f.FX(2 * i, 2 * j + 1)];
    }
  for (int j = 0; j <= nj; ++j)
    for (int i = 0; i < ni; ++i) {
      c.vfe[c.FE(i, j)] = f.vfe[f.FE(2 * i, 2 * j)] + f.vfe[f.FE(2 * i + 1, 2 * j)];
      if (j == 0) {
        c.wvx[i] = 0.5 * (f.wvx[2 * i] + f.wvx[2 * i + 1]);
        c.wvy[i] = 0.5 * (f.wvy[2 * i] + f.wvy[2 * i + 1]);
      }
      c.seta_x[c.FE(i, j)] = f.seta_x[f.FE(2 * i, 2 * j)] + f.seta_x[f.FE(2 * i + 1, 2 * j)];
      c.seta_y[c.FE(i, j)] = f.seta_y[f.FE(2 * i, 2 * j)] + f.seta_y[f.FE(2 * i + 1, 2 * j)];
    }
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i)
      c.vol[c.C(i, j)] = (f.vol[f.C(2 * i, 2 * j)] + f.vol[f.C(2 * i + 1, 2 * j)]) +
                         (f.vol[f.C(2 * i, 2 * j + 1)] + f.vol[f.C(2 * i + 1, 2 * j + 1)]);
}

static void alloc_level_state(Level& g) {
  const int n = g.ni * g.nj;
  g.u.assign((g.ni + 4) * (g.nj + 4), V4{});
  g.ut.assign(n, V4{});
  g.s.assign(n, V4{});
  g.src.assign(n, V4{});
  g.mut.assign(n, 0.0);
  g.dts.assign(n, 0.0);
  g.D.assign(n, M4{});
  g.coef.assign(n, 0.0);
  g.Axp.assign((g.ni + 1) * g.nj, M4{});
  g.Axm.assign((g.ni + 1) * g.nj, M4{});
  g.Aep.assign(g.ni * (g.nj + 1), M4{});
  g.Aem.assign(g.ni * (g.nj + 1), M4{});
}

// ---------------------------------------------------------------- boundary conditions
// Far field by 1-D Riemann invariants normal to the boundary (section 2, G9);
// n = outward unit normal.  Returns the boundary state given to both ghost layers.
template <class T>
static V4T<T> farfield_state(const V4T<T>& wi, const V4& winf, double nx, double ny, double vb = 0.0) {
  const PrimT<T> qi = prim(wi);
  const Prim qf = prim(winf);
  const T ai = std::sqrt(GAM * qi.p / qi.rho);
  const double af = std::sqrt(GAM * qf.p / qf.rho);
  const T vni = qi.u * nx + qi.v * ny;
  const double vnf = qf.u * nx + qf.v * ny;
  if (re(absr(vni - vb)) >= re(ai)) {
    if (re(vni - vb) > 0.0) return wi;
    return V4T<T>{winf[0], winf[1], winf[2], winf[3]};
  }
  const T Rp = vni + 2.0 * ai / (GAM - 1.0);
  const double Rm = vnf - 2.0 * af / (GAM - 1.0);
  const T vnb = 0.5 * (Rp + Rm);
  const T ab = 0.25 * (GAM - 1.0) * (Rp - Rm);
  T s, ut, vt;
  if (re(vnb - vb) > 0.0) {
    s = qi.p / std::pow(qi.rho, GAM);
    ut = qi.u - vni * nx;
    vt = qi.v - vni * ny;
  } else {
    s = qf.p / std::pow(qf.rho, GAM);
    ut = qf.u - vnf * nx;
    vt = qf.v - vnf * ny;
  }
  const T rho = std::pow(ab * ab / (GAM * s), 1.0 / (GAM - 1.0));
  const T p = rho * ab * ab / GAM;
  const T u = ut + vnb * nx, v = vt + vnb * ny;
  return V4T<T>{rho, rho * u, rho * v, p / (GAM - 1.0) + 0.5 * rho * (u * u + v * v)};
}

// Ghost states of the state array u (ghosted layout of level g).
template <class T> static void bc_fill_t(const Solver& S, const Level& g, std::vector<V4T<T>>& u) {
  const int ni = g.ni, nj = g.nj;
  const bool noslip = S.P.viscous != 0;
  // corners (never read by the stencils) get the free stream
  for (int j = -2; j < nj + 2; ++j)
    for (int i = -2; i < ni + 2; ++i)
      if ((i < 0 || i >= ni) && (j < 0 || j >= nj)) u[g.G(i, j)] = V4T<T>{S.uinf[0], S.uinf[1], S.uinf[2], S.uinf[3]};
  // j = 0: wall or wake cut
  for (int i = 0; i < ni; ++i) {
    if (g.cut(i)) {
      const int m = g.mirror(i);
      u[g.G(i, -1)] = u[g.G(m, 0)];
      u[g.G(i, -2)] = u[g.G(m, 1)];
    } else {
      const double sx = g.seta_x[g.FE(i, 0)], sy = g.seta_y[g.FE(i, 0)];
      const double len = std::sqrt(sx * sx + sy * sy);
      const double nx = sx / len, ny = sy / len;
      for (int k = 0; k < 2; ++k) {
        const V4T<T> w = u[g.G(i, k)];
        V4T<T> gw;
        if (!S.moving) {
          gw[0] = w[0];
          gw[3] = w[3];
          if (noslip) {
            gw[1] = -w[1];
            gw[2] = -w[2];
          } else {
            const T mn = w[1] * nx + w[2] * ny;
            gw[1] = w[1] - 2.0 * mn * nx;
            gw[2] = w[2] - 2.0 * mn * ny;
          }
        } else {
          // moving wall with velocity (wx, wy): same density and pressure, velocity mirrored
          // about the wall velocity (no-slip) or its normal component reflected relative to it
          const PrimT<T> q = prim(w);
          const double wx = g.wvx[i], wy = g.wvy[i];
          T ug, vg;
          if (noslip) {
            ug = 2.0 * wx - q.u;
            vg = 2.0 * wy - q.v;
          } else {
            const T rn = (q.u - wx) * nx + (q.v - wy) * ny;
            ug = q.u - 2.0 * rn * nx;
            vg = q.v - 2.0 * rn * ny;
          }
          gw[0] = q.rho;
          gw[1] = q.rho * ug;
          gw[2] = q.rho * vg;
          gw[3] = q.p / (GAM - 1.0) + 0.5 * q.rho * (ug * ug + vg * vg);
        }
        u[g.G(i, -1 - k)] = gw;
      }
    }
  }
  // j = nj: far field, outward normal = +S_eta
  for (int i = 0; i < ni; ++i) {
    const double sx = g.seta_x[g.FE(i, nj)], sy = g.seta_y[g.FE(i, nj)];
    const double len = std::sqrt(sx * sx + sy * sy);
    const V4T<T> b = farfield_state(u[g.G(i, nj - 1)], S.uinf, sx / len, sy / len, g.vfe[g.FE(i, nj)] / len);
    u[g.G(i, nj)] = b;
    u[g.G(i, nj + 1)] = b;
  }
  // i = 0 (outward = -S_xi) and i = ni (outward = +S_xi): far field
  for (int j = 0; j < nj; ++j) {
    {
      const double sx = g.sxi_x[g.FX(0, j)], sy = g.sxi_y[g.FX(0, j)];
      const double len = std::sqrt(sx * sx + sy * sy);
      const V4T<T> b = farfield_state(u[g.G(0, j)], S.uinf, -sx / len, -sy / len, -g.vfx[g.FX(0, j)] / len);
      u[g.G(-1, j)] = b;
      u[g.G(-2, j)] = b;
    }
    {
      const double sx = g.sxi_x[g.FX(ni, j)], sy = g.sxi_y[g.FX(ni, j)];
      const double len = std::sqrt(sx * sx + sy * sy);
      const V4T<T> b = farfield_state(u[g.G(ni - 1, j)], S.uinf, sx / len, sy / len, g.vfx[g.FX(ni, j)] / len);
      u[g.G(ni, j)] = b;
      u[g.G(ni + 1, j)] = b;
    }
  }
}

static void bc_fill(const Solver& S, Level& g) { bc_fill_t(S, g, g.u); }

// ---------------------------------------------------------------- JST residual
// Directional spectral radii of a cell: r = |v . S_bar| + a |S_bar|, with S_bar
// the mean of the cell's two opposite face area vectors (G6).
// On a moving grid the convective speed is relative: |v . S_bar - V_bar| with V_bar the mean
// grid volume flux of the same two faces.
template <class T> static void cell_radii(const Level& g, const V4T<T>& w, int i, int j, T& rxi, T& reta) {
  const PrimT<T> q = prim(w);
  const T a = std::sqrt(GAM * q.p / q.rho);
  const double sx = 0.5 * (g.sxi_x[g.FX(i, j)] + g.sxi_x[g.FX(i + 1, j)]);
  const double sy = 0.5 * (g.sxi_y[g.FX(i, j)] + g.sxi_y[g.FX(i + 1, j)]);
  const double ex = 0.5 * (g.seta_x[g.FE(i, j)] + g.seta_x[g.FE(i, j + 1)]);
  const double ey = 0.5 * (g.seta_y[g.FE(i, j)] + g.seta_y[g.FE(i, j + 1)]);
  const double vx = 0.5 * (g.vfx[g.FX(i, j)] + g.vfx[g.FX(i + 1, j)]);
  const double ve = 0.5 * (g.vfe[g.FE(i, j)] + g.vfe[g.FE(i, j + 1)]);
  rxi = absr(q.u * sx + q.v * sy - vx) + a * std::sqrt(sx * sx + sy * sy);
  reta = absr(q.u * ex + q.v * ey - ve) + a * std::sqrt(ex * ex + ey * ey);
}

// Martinelli correction (eq. spectralcorrection): r~_i = r_i (1 + (r_j/r_i)^(2/3)).
template <class T> static void martinelli(const T& rxi, const T& reta, T& txi, T& teta) {
  txi = rxi * (1.0 + std::pow(reta / rxi, 2.0 / 3.0));
  teta = reta * (1.0 + std::pow(rxi / reta, 2.0 / 3.0));
}

// Sensor quantity: pressure for Euler, p / rho^gamma (entropy) otherwise.
template <class T> static T sensor_q(const Solver& S, const V4T<T>& w) {
  const PrimT<T> q = prim(w);
  return S.P.sensor ? q.p / std::pow(q.rho, GAM) : q.p;
}

// s_k = |S_{k+1} - 2 S_k + S_{k-1}| / (S_{k+1} + 2 S_k + S_{k-1} + 0.001)  (G4)
template <class T> static T sensor_val(const T& qm, const T& q0, const T& qp) {
  return absr(qp - 2.0 * q0 + qm) / (qp + 2.0 * q0 + qm + 0.001);
}

template <class T> struct FaceFluxT { V4T<T> hc, hd; };
using FaceFlux = FaceFluxT<double>;

// JST flux through one face with area vector S (pointing from L to R), given
// the stencil LL, L, R, RR along the face-normal grid line (section 2):
//   h = (F(u_L) + F(u_R)) . S / 2 - d,
//   d = eps2 dw - eps4 (dw_+ - 2 dw + dw_-),  w = (rho, rho u, rho v, rho H),
//   eps2 = s r, eps4 = max(0, r/32 - 2 eps2),  s = min(0.25, max(s_L, s_R)),
//   r = max(r~_L, r~_R).   On coarse levels: s = s_coarse and no eps4 term.
// On a moving face (grid volume flux vf) the convective flux is F . S - u vf.
template <class T>
static FaceFluxT<T> jst_face(const Solver& S, const V4T<T>& uLL, const V4T<T>& uL, const V4T<T>& uR,
                             const V4T<T>& uRR, double sx, double sy, double vf, const T& rtL, const T& rtR,
                             bool finest) {
  FaceFluxT<T> out;
  const V4T<T> fL = conv_flux(uL, sx, sy), fR = conv_flux(uR, sx, sy);
  for (int k = 0; k < 4; ++k) out.hc[k] = 0.5 * ((fL[k] - uL[k] * vf) + (fR[k] - uR[k] * vf));
  auto wvec = [](const V4T<T>& w) {
    const PrimT<T> q = prim(w);
    return V4T<T>{w[0], w[1], w[2], w[3] + q.p};
  };
  const V4T<T> wLL = wvec(uLL), wL = wvec(uL), wR = wvec(uR), wRR = wvec(uRR);
  const T r = maxr(rtL, rtR);
  T eps2, eps4;
  if (finest) {
    const T qLL = sensor_q(S, uLL), qL = sensor_q(S, uL), qR = sensor_q(S, uR), qRR = sensor_q(S, uRR);
    const T sL = sensor_val(qLL, qL, qR), sR = sensor_val(qL, qR, qRR);
    const T s = minr(T(0.25), maxr(sL, sR));
    eps2 = s * r;
    eps4 = maxr(T(0.0), r / 32.0 - 2.0 * eps2);
  } else {
    eps2 = S.P.s_coarse * r;
    eps4 = T(0.0);
  }
  for (int k = 0; k < 4; ++k) {
    const T dw0 = wR[k] - wL[k];
    const T dwm = wL[k] - wLL[k];
    const T dwp = wRR[k] - wR[k];
    out.hd[k] = eps2 * dw0 - eps4 * ((dwp + dwm) - 2.0 * dw0);
  }
  return out;
}

// First-order flux-vector-split face flux (the discretization the preconditioner linearizes,
// section 4.4): h = A+(u_bar) u_L + A-(u_bar) u_R with u_bar the mean of the two states (G22)
// and the cutoff eigenvalues of eq. (cutoff).  Split as the JST flux is (h = hc - hd): the
// central part hc = A(u_bar) (u_L + u_R) / 2 and the upwind dissipation
// hd = (A+ - A-)(u_R - u_L) / 2, since A+ + A- = A.  A(u) u = F(u) . S for the Euler flux
// (homogeneous of degree one), so the flux is consistent: uniform flow gives F . S.
template <class T>
static FaceFluxT<T> fvs_face(const Solver& S, const V4T<T>& uL, const V4T<T>& uR, double sx, double sy, double vf) {
  V4T<T> ub;
  for (int k = 0; k < 4; ++k) ub[k] = 0.5 * (uL[k] + uR[k]);
  M4T<T> Ap, Am;
  split_jacobians(ub, sx, sy, vf, S.P.d_cut, Ap, Am);
  FaceFluxT<T> out;
  for (int r = 0; r < 4; ++r) {
    T c = 0.0, d = 0.0;
    for (int k = 0; k < 4; ++k) {
      c += (Ap[r][k] + Am[r][k]) * (uL[k] + uR[k]);
      d += (Ap[r][k] - Am[r][k]) * (uR[k] - uL[k]);
    }
    out.hc[r] = 0.5 * c;
    out.hd[r] = 0.5 * d;
  }
  return out;
}

// Martinelli-corrected radius of a (possibly ghost) cell in direction dir (0 = xi, 1 = eta).
// Ghost cells take the adjacent interior cell's value; across the wake cut the mirror cell's.
template <class T> static T rtilde_t(const Level& g, const std::vector<V4T<T>>& u, int i, int j, int dir) {
  int ii = i, jj = j;
  if (jj < 0) {
    const int ic = std::min(std::max(ii, 0), g.ni - 1);
    if (g.cut(ic)) {
      ii = g.mirror(ic);
      jj = 0;
    } else {
      ii = ic;
      jj = 0;
    }
  }
  ii = std::min(std::max(ii, 0), g.ni - 1);
  jj = std::min(jj, g.nj - 1);
  T rxi, reta, txi, teta;
  cell_radii(g, u[g.G(ii, jj)], ii, jj, rxi, reta);
  martinelli(rxi, reta, txi, teta);
  return dir == 0 ? txi : teta;
}

static double rtilde(const Level& g, int i, int j, int dir) { return rtilde_t(g, g.u, i, j, dir); }

// Thin-layer viscous flux through j-face (i, j) between (i, j-1) and (i, j) (G8):
// gradients from the difference across the face over the mean of the two volumes.
template <class T>
static V4T<T> visc_face_t(const Solver& S, const Level& g, const std::vector<V4T<T>>& u, int i, int j) {
  const int nj = g.nj;
  const V4T<T> wL = u[g.G(i, j - 1)], wR = u[g.G(i, j)];
  const double sx = g.seta_x[g.FE(i, j)], sy = g.seta_y[g.FE(i, j)];
  double volL, volR, mutf;
  if (j == 0) {
    if (g.cut(i)) {
      volL = g.vol[g.C(g.mirror(i), 0)];
      mutf = 0.5 * (g.mut[g.C(i, 0)] + g.mut[g.C(g.mirror(i), 0)]);
    } else {
      volL = g.vol[g.C(i, 0)];
      mutf = 0.0;
    }
    volR = g.vol[g.C(i, 0)];
  } else if (j == nj) {
    volL = g.vol[g.C(i, nj - 1)];
    volR = volL;
    mutf = g.mut[g.C(i, nj - 1)];
  } else {
    volL = g.vol[g.C(i, j - 1)];
    volR = g.vol[g.C(i, j)];
    mutf = 0.5 * (g.mut[g.C(i, j - 1)] + g.mut[g.C(i, j)]);
  }
  const double volf = 0.5 * (volL + volR);
  const PrimT<T> qL = prim(wL), qR = prim(wR);
  const double mu = 1.0 / S.P.re;
  const double mueff = mu + mutf;
  const double keff = mu / S.P.pr + mutf / S.P.prt;
  const T hL = GAM / (GAM - 1.0) * qL.p / qL.rho, hR = GAM / (GAM - 1.0) * qR.p / qR.rho;
  const T gux = (qR.u - qL.u) * sx / volf, guy = (qR.u - qL.u) * sy / volf;
  const T gvx = (qR.v - qL.v) * sx / volf, gvy = (qR.v - qL.v) * sy / volf;
  const T ghx = (hR - hL) * sx / volf, ghy = (hR - hL) * sy / volf;
  const T div = gux + gvy;
  const T txx = mueff * (2.0 * gux - 2.0 / 3.0 * div);
  const T tyy = mueff * (2.0 * gvy - 2.0 / 3.0 * div);
  const T txy = mueff * (guy + gvx);
  const T uf = 0.5 * (qL.u + qR.u), vf = 0.5 * (qL.v + qR.v);
  const T fx = txx * sx + txy * sy, fy = txy * sx + tyy * sy;
  return V4T<T>{T(0.0), fx, fy, uf * fx + vf * fy + keff * (ghx * sx + ghy * sy)};
}

static V4 visc_face(const Solver& S, const Level& g, int i, int j) { return visc_face_t(S, g, g.u, i, j); }

// F^c and F^v of the split (eq. split-rhs), per unit volume, at the level's current
// (ghost-filled) state:  F^c = Omega^{-1} (central fluxes) + a_t u + src - s,
//                        F^v = Omega^{-1} (-(dissipation) - (viscous fluxes)).
template <class T>
static void residual_t(const Solver& S, const Level& g, const std::vector<V4T<T>>& u, bool finest,
                       std::vector<V4T<T>>& Fc, std::vector<V4T<T>>& Fv) {
  const int ni = g.ni, nj = g.nj;
  std::vector<FaceFluxT<T>> fx((ni + 1) * nj), fe(ni * (nj + 1));
  std::vector<V4T<T>> fvis(ni * (nj + 1), V4T<T>{});
  const bool fvs = S.P.flux == 1;
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i <= ni; ++i)
      fx[g.FX(i, j)] = fvs ? fvs_face(S, u[g.G(i - 1, j)], u[g.G(i, j)], g.sxi_x[g.FX(i, j)],
                                      g.sxi_y[g.FX(i, j)], g.vfx[g.FX(i, j)])
                           : jst_face(S, u[g.G(i - 2, j)], u[g.G(i - 1, j)], u[g.G(i, j)],
                                      u[g.G(i + 1, j)], g.sxi_x[g.FX(i, j)], g.sxi_y[g.FX(i, j)],
                                      g.vfx[g.FX(i, j)], rtilde_t(g, u, i - 1, j, 0), rtilde_t(g, u, i, j, 0), finest);
  for (int j = 0; j <= nj; ++j)
    for (int i = 0; i < ni; ++i) {
      fe[g.FE(i, j)] = fvs ? fvs_face(S, u[g.G(i, j - 1)], u[g.G(i, j)], g.seta_x[g.FE(i, j)],
                                      g.seta_y[g.FE(i, j)], g.vfe[g.FE(i, j)])
                           : jst_face(S, u[g.G(i, j - 2)], u[g.G(i, j - 1)], u[g.G(i, j)],
                                      u[g.G(i, j + 1)], g.seta_x[g.FE(i, j)], g.seta_y[g.FE(i, j)],
                                      g.vfe[g.FE(i, j)], rtilde_t(g, u, i, j - 1, 1), rtilde_t(g, u, i, j, 1), finest);
      if (S.P.viscous) fvis[g.FE(i, j)] = visc_face_t(S, g, u, i, j);
    }
  Fc.assign(ni * nj, V4T<T>{});
  Fv.assign(ni * nj, V4T<T>{});
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const int c = g.C(i, j);
      const FaceFluxT<T> &w = fx[g.FX(i, j)], &e = fx[g.FX(i + 1, j)];
      const FaceFluxT<T> &s = fe[g.FE(i, j)], &n = fe[g.FE(i, j + 1)];
      const V4T<T> &vs = fvis[g.FE(i, j)], &vn = fvis[g.FE(i, j + 1)];
      for (int k = 0; k < 4; ++k) {
        const T fc = (e.hc[k] - w.hc[k]) + (n.hc[k] - s.hc[k]);
        const T fd = -((e.hd[k] - w.hd[k]) + (n.hd[k] - s.hd[k]));
        const T fv = -(vn[k] - vs[k]);
        Fc[c][k] = fc / g.vol[c] + g.a_t * u[g.G(i, j)][k] + g.src[c][k] - g.s[c][k];
        Fv[c][k] = (fd + fv) / g.vol[c];
      }
    }
}

static void residual(const Solver& S, Level& g, bool finest, std::vector<V4>& Fc, std::vector<V4>& Fv) {
  residual_t(S, g, g.u, finest, Fc, Fv);
}

// ---------------------------------------------------------------- Baldwin-Lomax
// Algebraic eddy viscosity (section 2 cites the 1978 model; constants from that model, G33).
static void baldwin_lomax(const Solver& S, Level& g) {
  const double Aplus = 26.0, Ccp = 1.6, Ckleb = 0.3, Cwk = 0.25, kap = 0.4, Kc = 0.0168;
  const int ni = g.ni, nj = g.nj;
  const double mu = 1.0 / S.P.re;
  std::vector<double> om(ni * nj), spd(ni * nj);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const Prim q = prim(g.u[g.G(i, j)]);
      auto vel = [&](int ii, int jj, double& uu, double& vv) {
        const Prim p = prim(g.u[g.G(ii, jj)]);
        uu = 0.5 * (q.u + p.u);
        vv = 0.5 * (q.v + p.v);
      };
      double ue, ve, uw, vw, un, vn, us, vs;
      vel(i + 1, j, ue, ve);
      vel(i - 1, j, uw, vw);
      vel(i, j + 1, un, vn);
      vel(i, j - 1, us, vs);
      // omega = dv/dx - du/dy by Green-Gauss with outward face vectors
      const double circ = (ve * g.sxi_x[g.FX(i + 1, j)] - ue * g.sxi_y[g.FX(i + 1, j)]) -
                          (vw * g.sxi_x[g.FX(i, j)] - uw * g.sxi_y[g.FX(i, j)]) +
                          (vn * g.seta_x[g.FE(i, j + 1)] - un * g.seta_y[g.FE(i, j + 1)]) -
                          (vs * g.seta_x[g.FE(i, j)] - us * g.seta_y[g.FE(i, j)]);
      om[g.C(i, j)] = std::fabs(circ / g.vol[g.C(i, j)]);
      spd[g.C(i, j)] = std::sqrt(q.u * q.u + q.v * q.v);
    }
  const int jsearch = std::max(1, nj / 2);
  for (int i = 0; i < ni; ++i) {
    const bool wake = g.cut(i);
    const double rhow = g.u[g.G(i, 0)][0];
    const double tauw = mu * om[g.C(i, 0)];
    const double utau_rho = std::sqrt(rhow * tauw);  // sqrt(rho_w tau_w)
    double Fmax = 0.0, ymax = 0.0, smax = 0.0, smin = 1e300;
    std::vector<double> damp(nj);
    for (int j = 0; j < nj; ++j) {
      const double y = g.wdist[g.C(i, j)];
      const double yplus = utau_rho * y / mu;
      damp[j] = wake ? 1.0 : 1.0 - std::exp(-yplus / Aplus);
      if (j < jsearch) {
        const double F = y * om[g.C(i, j)] * damp[j];
        if (F > Fmax) {
          Fmax = F;
          ymax = y;
        }
        smax = std::max(smax, spd[g.C(i, j)]);
        smin = std::min(smin, spd[g.C(i, j)]);
      }
    }
    const double udif = wake ? smax - smin : smax;
    const double Fwake = Fmax > 0.0 ? std::min(ymax * Fmax, Cwk * ymax * udif * udif / Fmax) : 0.0;
    bool outer = wake;
    for (int j = 0; j < nj; ++j) {
      const int c = g.C(i, j);
      const double y = g.wdist[c];
      const double rho = g.u[g.G(i, j)][0];
      const double fk = ymax > 0.0 ? 1.0 / (1.0 + 5.5 * std::pow(Ckleb * y / ymax, 6.0)) : 0.0;
      const double mo = Kc * Ccp * rho * Fwake * fk;
      const double l = kap * y * damp[j];
      const double mi = rho * l * l * om[c];
      if (!outer && mi >= mo) outer = true;
      g.mut[c] = outer ? mo : mi;
    }
  }
}

// ---------------------------------------------------------------- preconditioner
// Thin-layer viscous Jacobian of j-face (i, j) in scalar form (reading G37): the face flux
// behaves like nu |S|^2 / Omega_f (u_R - u_L) with nu = max(mu + mu_t, gamma (mu/Pr + mu_t/Pr_t)) / rho,
// so it adds +V I to A+ and -V I to A- of that face (A+ + A- keeps the convective Jacobian).
static double visc_radius(const Solver& S, const Level& g, int i, int j, double rho) {
  const int nj = g.nj;
  double volL, volR, mutf;
  if (j == 0) {
    volR = g.vol[g.C(i, 0)];
    if (g.cut(i)) {
      volL = g.vol[g.C(g.mirror(i), 0)];
      mutf = 0.5 * (g.mut[g.C(i, 0)] + g.mut[g.C(g.mirror(i), 0)]);
    } else {
      volL = volR;
      mutf = 0.0;
    }
  } else if (j == nj) {
    volL = g.vol[g.C(i, nj - 1)];
    volR = volL;
    mutf = g.mut[g.C(i, nj - 1)];
  } else {
    volL = g.vol[g.C(i, j - 1)];
    volR = g.vol[g.C(i, j)];
    mutf = 0.5 * (g.mut[g.C(i, j - 1)] + g.mut[g.C(i, j)]);
  }
  const double volf = 0.5 * (volL + volR);
  const double mu = 1.0 / S.P.re;
  const double nu = std::max(mu + mutf, GAM * (mu / S.P.pr + mutf / S.P.prt)) / rho;
  const double sx = g.seta_x[g.FE(i, j)], sy = g.seta_y[g.FE(i, j)];
  return nu * (sx * sx + sy * sy) / volf;
}

// Pseudo time step (G17): dt*_i = c* Omega_i / (r_xi + r_eta).
static void pseudo_dt(const Solver& S, Level& g, double cfl) {
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i) {
      double rxi, reta;
      cell_radii(g, g.u[g.G(i, j)], i, j, rxi, reta);
      g.dts[g.C(i, j)] = cfl * g.vol[g.C(i, j)] / (rxi + reta);
    }
}

// Split face Jacobians at the face-averaged state of the current (ghost-filled)
// state (section 4.4, G22), and the block diagonal (G23):
//   AW : D_i = (1 + eta dt*_i a_t) I + (eta dt*_i / Omega_i) (A+_e - A-_w + B+_n - B-_s)
//   ARK: D_i = a_t I + (1 / Omega_i) (A+_e - A-_w + B+_n - B-_s)
static void build_blocks(const Solver& S, Level& g) {
  const int ni = g.ni, nj = g.nj;
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i <= ni; ++i) {
      V4 ub;
      const V4 &a = g.u[g.G(i - 1, j)], &b = g.u[g.G(i, j)];
      for (int k = 0; k < 4; ++k) ub[k] = 0.5 * (a[k] + b[k]);
      split_jacobians(ub, g.sxi_x[g.FX(i, j)], g.sxi_y[g.FX(i, j)], g.vfx[g.FX(i, j)], S.P.d_cut, g.Axp[g.FX(i, j)],
                      g.Axm[g.FX(i, j)]);
    }
  for (int j = 0; j <= nj; ++j)
    for (int i = 0; i < ni; ++i) {
      V4 ub;
      const V4 &a = g.u[g.G(i, j - 1)], &b = g.u[g.G(i, j)];
      for (int k = 0; k < 4; ++k) ub[k] = 0.5 * (a[k] + b[k]);
      split_jacobians(ub, g.seta_x[g.FE(i, j)], g.seta_y[g.FE(i, j)], g.vfe[g.FE(i, j)], S.P.d_cut, g.Aep[g.FE(i, j)],
                      g.Aem[g.FE(i, j)]);
      if (S.P.viscous) {
        const double V = visc_radius(S, g, i, j, ub[0]);
        for (int k = 0; k < 4; ++k) {
          g.Aep[g.FE(i, j)][k][k] += V;
          g.Aem[g.FE(i, j)][k][k] -= V;
        }
      }
    }
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const int c = g.C(i, j);
      double coef, sigma;
      if (S.P.scheme == 0) {
        coef = S.P.eta * g.dts[c] / g.vol[c];
        sigma = 1.0 + S.P.eta * g.dts[c] * g.a_t;
      } else {
        coef = 1.0 / g.vol[c];
        sigma = g.a_t;
      }
      g.coef[c] = coef;
      const M4 &Ae = g.Axp[g.FX(i + 1, j)], &Aw = g.Axm[g.FX(i, j)];
      const M4 &Bn = g.Aep[g.FE(i, j + 1)], &Bs = g.Aem[g.FE(i, j)];
      M4 D{};
      for (int r = 0; r < 4; ++r)
        for (int k = 0; k < 4; ++k)
          D[r][k] = (r == k ? sigma : 0.0) + coef * ((Ae[r][k] - Aw[r][k]) + (Bn[r][k] - Bs[r][k]));
      g.D[c] = D;
    }
}

// Neighbour coupling of cell (i,j): block times coefficient, and neighbour index.
struct Nb { int c; M4 B; };

static void neighbours(const Level& g, int i, int j, std::vector<Nb>& lower, std::vector<Nb>& upper) {
  lower.clear();
  upper.clear();
  const int c = g.C(i, j);
  const double cf = g.coef[c];
  auto scaled = [&](const M4& A, double s) {
    M4 B;
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) B[r][k] = s * A[r][k];
    return B;
  };
  auto order = [&](int nc) { return nc < c; };  // lexicographic j-major index
  // west: -c A+ of face (i,j); east: +c A- of face (i+1,j)
  if (i > 0) lower.push_back({g.C(i - 1, j), scaled(g.Axp[g.FX(i, j)], -cf)});
  if (i < g.ni - 1) upper.push_back({g.C(i + 1, j), scaled(g.Axm[g.FX(i + 1, j)], cf)});
  // south: -c B+ of face (i,j) (also across the wake cut); north: +c B- of face (i,j+1)
  if (j > 0) {
    lower.push_back({g.C(i, j - 1), scaled(g.Aep[g.FE(i, j)], -cf)});
  } else if (g.cut(i)) {
    const int nc = g.C(g.mirror(i), 0);
    Nb nb{nc, scaled(g.Aep[g.FE(i, 0)], -cf)};
    if (order(nc)) lower.push_back(nb); else upper.push_back(nb);
  }
  if (j < g.nj - 1) upper.push_back({g.C(i, j + 1), scaled(g.Aem[g.FE(i, j + 1)], cf)});
}

// z = P^{-1} r with P = (D+L) D^{-1} (D+U) (eq. sgs-precon, G20):
// forward (D+L) y = r, backward (D+U) z = D y; lexicographic order.
static void sgs_apply(const Level& g, const std::vector<V4>& r, std::vector<V4>& z) {
  const int ni = g.ni, nj = g.nj, n = ni * nj;
  std::vector<V4> y(n);
  std::vector<Nb> lo, up;
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      const int c = g.C(i, j);
      neighbours(g, i, j, lo, up);
      V4 t = r[c];
      for (const Nb& nb : lo) {
        const V4 m = matvec(nb.B, y[nb.c]);
        for (int k = 0; k < 4; ++k) t[k] -= m[k];
      }
      y[c] = solve4(g.D[c], t);
    }
  z.assign(n, V4{});
  for (int j = nj - 1; j >= 0; --j)
    for (int i = ni - 1; i >= 0; --i) {
      const int c = g.C(i, j);
      neighbours(g, i, j, lo, up);
      V4 t{0.0, 0.0, 0.0, 0.0};
      for (const Nb& nb : up) {
        const V4 m = matvec(nb.B, z[nb.c]);
        for (int k = 0; k < 4; ++k) t[k] += m[k];
      }
      const V4 q = solve4(g.D[c], t);
      for (int k = 0; k < 4; ++k) z[c][k] = y[c][k] - q[k];
    }
}

// Independent dense application: assemble N x N matrices and solve with partial pivoting.
static void dense_apply(const Level& g, const std::vector<V4>& r, std::vector<V4>& z) {
  const int n = g.ni * g.nj, N = 4 * n;
  std::vector<double> Dm(N * N, 0.0), Lm(N * N, 0.0), Um(N * N, 0.0);
  std::vector<Nb> lo, up;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i) {
      const int c = g.C(i, j);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) Dm[(4 * c + a) * N + 4 * c + b] = g.D[c][a][b];
      neighbours(g, i, j, lo, up);
      for (const Nb& nb : lo)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) Lm[(4 * c + a) * N + 4 * nb.c + b] += nb.B[a][b];
      for (const Nb& nb : up)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) Um[(4 * c + a) * N + 4 * nb.c + b] += nb.B[a][b];
    }
  // D^{-1} (block diagonal) by dense Gauss-Jordan on each block
  std::vector<double> Dinv(N * N, 0.0);
  for (int c = 0; c < n; ++c) {
    double A[4][8];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 8; ++b) A[a][b] = b < 4 ? Dm[(4 * c + a) * N + 4 * c + b] : (b - 4 == a ? 1.0 : 0.0);
    for (int k = 0; k < 4; ++k) {
      int p = k;
      for (int a = k + 1; a < 4; ++a)
        if (std::fabs(A[a][k]) > std::fabs(A[p][k])) p = a;
      for (int b = 0; b < 8; ++b) std::swap(A[k][b], A[p][b]);
      const double piv = A[k][k];
      for (int b = 0; b < 8; ++b) A[k][b] /= piv;
      for (int a = 0; a < 4; ++a)
        if (a != k) {
          const double m = A[a][k];
          for (int b = 0; b < 8; ++b) A[a][b] -= m * A[k][b];
        }
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) Dinv[(4 * c + a) * N + 4 * c + b] = A[a][b + 4];
  }
  // P = (D+L) Dinv (D+U)
  std::vector<double> DL(N * N), DU(N * N), T(N * N, 0.0), Pm(N * N, 0.0);
  for (int k = 0; k < N * N; ++k) {
    DL[k] = Dm[k] + Lm[k];
    DU[k] = Dm[k] + Um[k];
  }
  for (int a = 0; a < N; ++a)
    for (int k = 0; k < N; ++k) {
      const double v = DL[a * N + k];
      if (v == 0.0) continue;
      for (int b = 0; b < N; ++b) T[a * N + b] += v * Dinv[k * N + b];
    }
  for (int a = 0; a < N; ++a)
    for (int k = 0; k < N; ++k) {
      const double v = T[a * N + k];
      if (v == 0.0) continue;
      for (int b = 0; b < N; ++b) Pm[a * N + b] += v * DU[k * N + b];
    }
  // solve P z = r, partial pivoting
  std::vector<double> rhs(N);
  for (int c = 0; c < n; ++c)
    for (int a = 0; a < 4; ++a) rhs[4 * c + a] = r[c][a];
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int a = k + 1; a < N; ++a)
      if (std::fabs(Pm[a * N + k]) > std::fabs(Pm[p * N + k])) p = a;
    if (p != k) {
      for (int b = 0; b < N; ++b) std::swap(Pm[k * N + b], Pm[p * N + b]);
      std::swap(rhs[k], rhs[p]);
    }
    for (int a = k + 1; a < N; ++a) {
      const double m = Pm[a * N + k] / Pm[k * N + k];
      if (m == 0.0) continue;
      for (int b = k; b < N; ++b) Pm[a * N + b] -= m * Pm[k * N + b];
      rhs[a] -= m * rhs[k];
    }
  }
  std::vector<double> sol(N);
  for (int a = N - 1; a >= 0; --a) {
    double s = rhs[a];
    for (int b = a + 1; b < N; ++b) s -= Pm[a * N + b] * sol[b];
    sol[a] = s / Pm[a * N + a];
  }
  z.assign(n, V4{});
  for (int c = 0; c < n; ++c)
    for (int a = 0; a < 4; ++a) z[c][a] = sol[4 * c + a];
}

// y = (D + L + U) x: the block operator of eq. (steadylinearized) / (form1) with the blocks of
// the current build (the same neighbour sets the sweeps use).  With the ARK scaling (1/Omega)
// and a_t = 0 it is the first-order flux-vector-split residual linearized at frozen face states.
static void block_apply(const Level& g, const std::vector<V4>& x, std::vector<V4>& y) {
  const int n = g.ni * g.nj;
  y.assign(n, V4{});
  std::vector<Nb> lo, up;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i) {
      const int c = g.C(i, j);
      V4 t = matvec(g.D[c], x[c]);
      neighbours(g, i, j, lo, up);
      for (const Nb& nb : lo) {
        const V4 m = matvec(nb.B, x[nb.c]);
        for (int k = 0; k < 4; ++k) t[k] += m[k];
      }
      for (const Nb& nb : up) {
        const V4 m = matvec(nb.B, x[nb.c]);
        for (int k = 0; k < 4; ++k) t[k] += m[k];
      }
      y[c] = t;
    }
}

// The "exact" preconditioner (the column of the same name in Table Prec-ARK-stability,
// section 5.4): z = (D + L + U)^-1 r instead of the SGS factorization, by Gaussian
// elimination with partial pivoting on the band of the lexicographic ordering (couplings reach
// one grid row, ni cells, away; the wake cut stays within row 0).  For tiny grids.
static void exact_apply(const Level& g, const std::vector<V4>& r, std::vector<V4>& z) {
  const int n = g.ni * g.nj, N = 4 * n;
  const int b = 4 * g.ni + 3;     // lower and upper bandwidth of D + L + U
  const int w = 3 * b + 1;        // stored columns: the band plus fill from row exchanges
  std::vector<double> A((size_t)N * w, 0.0);  // A(row, col) at row * w + (col - row + b)
  auto at = [&](int row, int col) -> double& { return A[(size_t)row * w + (col - row + b)]; };
  std::vector<Nb> lo, up;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i) {
      const int c = g.C(i, j);
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 4; ++q) at(4 * c + a, 4 * c + q) += g.D[c][a][q];
      neighbours(g, i, j, lo, up);
      for (const Nb& nb : lo)
        for (int a = 0; a < 4; ++a)
          for (int q = 0; q < 4; ++q) at(4 * c + a, 4 * nb.c + q) += nb.B[a][q];
      for (const Nb& nb : up)
        for (int a = 0; a < 4; ++a)
          for (int q = 0; q < 4; ++q) at(4 * c + a, 4 * nb.c + q) += nb.B[a][q];
    }
  std::vector<double> rhs(N);
  for (int c = 0; c < n; ++c)
    for (int a = 0; a < 4; ++a) rhs[4 * c + a] = r[c][a];
  for (int k = 0; k < N; ++k) {
    const int last = std::min(N - 1, k + b);
    int p = k;
    for (int a = k + 1; a <= last; ++a)
      if (std::fabs(at(a, k)) > std::fabs(at(p, k))) p = a;
    const int cmax = std::min(N - 1, k + 2 * b);  // upper band after row exchanges: b_l + b_u = 2b
    if (p != k) {
      for (int col = k; col <= cmax; ++col) std::swap(at(k, col), at(p, col));
      std::swap(rhs[k], rhs[p]);
    }
    for (int a = k + 1; a <= last; ++a) {
      const double m = at(a, k) / at(k, k);
      if (m == 0.0) continue;
      for (int col = k; col <= cmax; ++col) at(a, col) -= m * at(k, col);
      rhs[a] -= m * rhs[k];
    }
  }
  std::vector<double> sol(N);
  for (int a = N - 1; a >= 0; --a) {
    double s = rhs[a];
    const int cmax = std::min(N - 1, a + 2 * b);
    for (int col = a + 1; col <= cmax; ++col) s -= at(a, col) * sol[col];
    sol[a] = s / at(a, a);
  }
  z.assign(n, V4{});
  for (int c = 0; c < n; ++c)
    for (int a = 0; a < 4; ++a) z[c][a] = sol[4 * c + a];
}

// ---------------------------------------------------------------- stage loop
// Generic low-storage preconditioned additive RK / additive W step (sections 4.1, 4.2):
//   u^(0) = u;  u^(i) = u - alpha_i [dt* W^{-1}] (f^{c,(i-1)} + f^{v,(i-1)}),  i = 1..s
// where apply_Winv supplies the bracket (including the local pseudo time step)
//   f^{c,(i)} = f^c(u^(i));  f^{v,(0)} = f^v(u^(0));
//   f^{v,(i)} = beta_{i+1} f^v(u^(i)) + (1 - beta_{i+1}) f^{v,(i-1)}   (G15)
struct StageOps {
  virtual ~StageOps() = default;
  virtual void get_state(std::vector<V4>& u) = 0;
  virtual void residual(std::vector<V4>& fc, std::vector<V4>& fv) = 0;
  virtual void apply_Winv(const std::vector<V4>& r, std::vector<V4>& z) = 0;
  virtual void set_state(const std::vector<V4>& u0, double alpha, const std::vector<V4>& z) = 0;
  virtual void stage_residual(int stage, const std::vector<V4>& fc, const std::vector<V4>& fv) {
    (void)stage; (void)fc; (void)fv;
  }
};

static void stage_loop(StageOps& op, int s, const double* alpha, const double* beta) {
  std::vector<V4> u0, fc, fv, fvc, R, z;
  op.get_state(u0);
  for (int i = 1; i <= s; ++i) {
    op.residual(fc, fv);
    op.stage_residual(i, fc, fv);
    if (i == 1) {
      fvc = fv;
    } else {
      const double b = beta[i - 1];
      for (size_t c = 0; c < fvc.size(); ++c)
        for (int k = 0; k < 4; ++k) fvc[c][k] = b * fv[c][k] + (1.0 - b) * fvc[c][k];
    }
    R.resize(fc.size());
    for (size_t c = 0; c < fc.size(); ++c)
      for (int k = 0; k < 4; ++k) R[c][k] = fc[c][k] + fvc[c][k];
    op.apply_Winv(R, z);
    op.set_state(u0, alpha[i - 1], z);
  }
}

struct LevelOps : StageOps {
  Solver& S;
  Level& g;
  bool finest;
  bool dense;
  LevelOps(Solver& s, Level& l, bool f, bool d = false) : S(s), g(l), finest(f), dense(d) {}
  void get_state(std::vector<V4>& u) override {
    u.resize(g.ni * g.nj);
    for (int j = 0; j < g.nj; ++j)
      for (int i = 0; i < g.ni; ++i) u[g.C(i, j)] = g.u[g.G(i, j)];
  }
  void residual(std::vector<V4>& fc, std::vector<V4>& fv) override {
    bc_fill(S, g);
    orc::residual(S, g, finest, fc, fv);
  }
  void stage_residual(int stage, const std::vector<V4>& fc, const std::vector<V4>& fv) override {
    if (stage == 1 && finest && S.record_norm) {
      double acc = 0.0;
      const int nk = S.P.norm_all ? 4 : 1;
      for (size_t c = 0; c < fc.size(); ++c)
        for (int k = 0; k < nk; ++k) {
          const double v = fc[c][k] + fv[c][k];
          acc += v * v;
        }
      S.norm_first = std::sqrt(acc / (double)(fc.size() * nk));
    }
  }
  // The product "dt* W^{-1}" with local steps T = diag(dt*_i) (reading G36):
  //   AW : z = W^{-1} (T r), W = I + eta T J row-scaled as in eq. d-l-u-matrices-W,
  //        so that W^{-1} T -> (eta J)^{-1} for large dt* (the Rosenbrock step);
  //   ARK: z = T P^{-1} r, the pseudo-time step of u' = -P^{-1} F (section 4.1).
  void apply_Winv(const std::vector<V4>& r, std::vector<V4>& z) override {
    const size_t n = r.size();
    if (S.P.scheme == 0) {
      std::vector<V4> tr(n);
      for (size_t c = 0; c < n; ++c)
        for (int k = 0; k < 4; ++k) tr[c][k] = g.dts[c] * r[c][k];
      if (S.P.precond == 1) exact_apply(g, tr, z); else if (dense) dense_apply(g, tr, z); else sgs_apply(g, tr, z);
    } else {
      if (S.P.precond == 1) exact_apply(g, r, z); else if (dense) dense_apply(g, r, z); else sgs_apply(g, r, z);
      for (size_t c = 0; c < n; ++c)
        for (int k = 0; k < 4; ++k) z[c][k] = g.dts[c] * z[c][k];
    }
  }
  void set_state(const std::vector<V4>& u0, double alpha, const std::vector<V4>& z) override {
    for (int j = 0; j < g.nj; ++j)
      for (int i = 0; i < g.ni; ++i) {
        const int c = g.C(i, j);
        for (int k = 0; k < 4; ++k) g.u[g.G(i, j)][k] = u0[c][k] - alpha * z[c][k];
      }
  }
};

// One smoothing step on level l: W (and dt*) frozen at u^(0) (G19), then s stages.
static void smooth(Solver& S, int l, double cfl) {
  Level& g = S.lev[l];
  const bool finest = (l == S.L());
  bc_fill(S, g);
  pseudo_dt(S, g, cfl);
  build_blocks(S, g);
  LevelOps op(S, g, finest);
  stage_loop(op, S.P.nstages, S.P.alpha, S.P.beta);
  bc_fill(S, g);
}

// ---------------------------------------------------------------- multigrid transfer
// Volume-weighted agglomeration restriction R_{l-1,l} (section 3).
static void restrict_vec(const Level& f, const Level& c, const std::vector<V4>& vf, std::vector<V4>& vc,
                         bool ghosted_fine) {
  vc.assign(c.ni * c.nj, V4{});
  for (int J = 0; J < c.nj; ++J)
    for (int I = 0; I < c.ni; ++I) {
      V4 acc{};
      const int fi[4] = {2 * I, 2 * I + 1, 2 * I, 2 * I + 1};
      const int fj[4] = {2 * J, 2 * J, 2 * J + 1, 2 * J + 1};
      for (int q = 0; q < 4; ++q) {
        const double w = f.vol[f.C(fi[q], fj[q])];
        const V4& v = ghosted_fine ? vf[f.G(fi[q], fj[q])] : vf[f.C(fi[q], fj[q])];
        for (int k = 0; k < 4; ++k) acc[k] += w * v[k];
      }
      for (int k = 0; k < 4; ++k) vc[c.C(I, J)][k] = acc[k] / c.vol[c.C(I, J)];
    }
}

// Coarse correction value at a possibly-ghost coarse cell (G14): zero-gradient copy at
// far-field and wall boundaries, mirror across the wake cut.
static V4 coarse_delta(const Level& c, const std::vector<V4>& dl, int I, int J) {
  const int Ic = std::min(std::max(I, 0), c.ni - 1);
  if (J < 0) {
    if (c.cut(Ic)) return dl[c.C(c.mirror(Ic), 0)];
    return dl[c.C(Ic, 0)];
  }
  const int Jc = std::min(J, c.nj - 1);
  return dl[c.C(Ic, Jc)];
}

// Bilinear prolongation P_{l,l-1} (section 3): weights 9/16, 3/16, 3/16, 1/16 from the
// coarse cell containing the fine cell and its three nearest coarse neighbours.
static void prolong_add(Level& f, const Level& c, const std::vector<V4>& dl) {
  for (int j = 0; j < f.nj; ++j)
    for (int i = 0; i < f.ni; ++i) {
      const int I = i / 2, J = j / 2;
      const int I2 = (i % 2 == 0) ? I - 1 : I + 1;
      const int J2 = (j % 2 == 0) ? J - 1 : J + 1;
      const V4 a = coarse_delta(c, dl, I, J), b = coarse_delta(c, dl, I2, J);
      const V4 cc = coarse_delta(c, dl, I, J2), d = coarse_delta(c, dl, I2, J2);
      for (int k = 0; k < 4; ++k)
        f.u[f.G(i, j)][k] += (9.0 * a[k] + 3.0 * b[k] + 3.0 * cc[k] + d[k]) / 16.0;
    }
}

// ---------------------------------------------------------------- FAS cycle (section 3)
static void fas_cycle(Solver& S, int l, double cfl) {
  Level& g = S.lev[l];
  for (int k = 0; k < S.P.nu1; ++k) smooth(S, l, cfl);
  if (l == 0) return;
  Level& c = S.lev[l - 1];
  // r_l = s_l - F_l(u_l)
  std::vector<V4> Fc, Fv, r(g.ni * g.nj);
  bc_fill(S, g);
  residual(S, g, l == S.L(), Fc, Fv);
  for (int q = 0; q < g.ni * g.nj; ++q)
    for (int k = 0; k < 4; ++k) r[q][k] = -(Fc[q][k] + Fv[q][k]);  // F here already includes -s_l
  // u~_{l-1} = R u_l ; s_{l-1} = F_{l-1}(u~) + R r_l
  std::vector<V4> ut, rr;
  restrict_vec(g, c, g.u, ut, true);
  restrict_vec(g, c, r, rr, false);
  c.ut = ut;
  for (int J = 0; J < c.nj; ++J)
    for (int I = 0; I < c.ni; ++I) c.u[c.G(I, J)] = ut[c.C(I, J)];
  if (S.P.turb) {
    std::vector<V4> mv(g.ni * g.nj), mc;
    for (int q = 0; q < g.ni * g.nj; ++q) mv[q] = V4{g.mut[q], 0.0, 0.0, 0.0};
    restrict_vec(g, c, mv, mc, false);
    for (int q = 0; q < c.ni * c.nj; ++q) c.mut[q] = mc[q][0];
  }
  for (auto& v : c.s) v = V4{};
  bc_fill(S, c);
  residual(S, c, false, Fc, Fv);  // with s = 0: F_{l-1}(u~)
  for (int q = 0; q < c.ni * c.nj; ++q)
    for (int k = 0; k < 4; ++k) c.s[q][k] = (Fc[q][k] + Fv[q][k]) + rr[q][k];
  for (int it = 0; it < S.P.gamma_cycle; ++it) fas_cycle(S, l - 1, cfl);
  // u_l += P (u_{l-1} - u~_{l-1})
  std::vector<V4> dl(c.ni * c.nj);
  for (int J = 0; J < c.nj; ++J)
    for (int I = 0; I < c.ni; ++I)
      for (int k = 0; k < 4; ++k) dl[c.C(I, J)][k] = c.u[c.G(I, J)][k] - c.ut[c.C(I, J)][k];
  prolong_add(g, c, dl);
  bc_fill(S, g);
}

// ---------------------------------------------------------------- linear model (section 5)
// Linearized Euler u_t + A u_x + B u_y = 0 on a periodic nx x ny Cartesian grid (eq.
// linearized-euler), discretized as in section 5.1 with the sensor switched off (eps2 = 0,
// eps4 = r/32 per direction): H = H_c + H_v,
//   H_c u = (A (u_{i+1} - u_{i-1}) dy + B (u_{j+1} - u_{j-1}) dx) / (2 dx dy) [+ a_t u],
//   H_v u = M (eps4x (u_{i+2} - 4u_{i+1} + 6u_i - 4u_{i-1} + u_{i-2}) dy + eps4y (...) dx) / (dx dy).
// The preconditioner uses the blocks of section 5.2 (cell values, not face averages):
//   L = -(s/Omega) (dy A+ E_x^-1 + dx B+ E_y^-1),  U = (s/Omega) (dy A- E_x + dx B- E_y),
//   D = sigma I + (s/Omega) (dy (A+ - A-) + dx (B+ - B-)), Omega = dx dy,
// with s = eta dt* (AW) and sigma = 1 + eta dt* a_t, applied either as the circulant operator
// (wrap-around couplings in L and U, dense solve) or as a real lexicographic sweep in which
// wrap-around neighbours are treated like every other neighbour of lower or higher index.
struct LinModel {
  int nx, ny;
  double dx, dy, dts, eta, a_t, eps4x, eps4y;
  M4 A, B, Ap, Am, Bp, Bm, M;
  int aw;
  int circulant;
  int idx(int i, int j) const { return ((j + ny) % ny) * nx + ((i + nx) % nx); }
};

struct LinOps : StageOps {
  const LinModel& m;
  std::vector<V4> u;
  LinOps(const LinModel& mm) : m(mm) {}
  void get_state(std::vector<V4>& v) override { v = u; }
  void residual(std::vector<V4>& fc, std::vector<V4>& fv) override {
    const int n = m.nx * m.ny;
    fc.assign(n, V4{});
    fv.assign(n, V4{});
    const double om = m.dx * m.dy;
    for (int j = 0; j < m.ny; ++j)
      for (int i = 0; i < m.nx; ++i) {
        const int c = m.idx(i, j);
        V4 dxu, dyu, d4x, d4y;
        for (int k = 0; k < 4; ++k) {
          dxu[k] = u[m.idx(i + 1, j)][k] - u[m.idx(i - 1, j)][k];
          dyu[k] = u[m.idx(i, j + 1)][k] - u[m.idx(i, j - 1)][k];
          d4x[k] = u[m.idx(i + 2, j)][k] - 4.0 * u[m.idx(i + 1, j)][k] + 6.0 * u[c][k] - 4.0 * u[m.idx(i - 1, j)][k] +
                   u[m.idx(i - 2, j)][k];
          d4y[k] = u[m.idx(i, j + 2)][k] - 4.0 * u[m.idx(i, j + 1)][k] + 6.0 * u[c][k] - 4.0 * u[m.idx(i, j - 1)][k] +
                   u[m.idx(i, j - 2)][k];
        }
        const V4 ax = matvec(m.A, dxu), by = matvec(m.B, dyu);
        V4 diss;
        for (int k = 0; k < 4; ++k) diss[k] = (m.eps4x * d4x[k] * m.dy + m.eps4y * d4y[k] * m.dx) / om;
        const V4 md = matvec(m.M, diss);
        for (int k = 0; k < 4; ++k) {
          fc[c][k] = (ax[k] * m.dy + by[k] * m.dx) / (2.0 * om) + m.a_t * u[c][k];
          fv[c][k] = md[k];
        }
      }
  }
  // coupling blocks of cell c: D, and neighbour blocks with their cell index
  void blocks(M4& D, std::vector<Nb>& lower, std::vector<Nb>& upper, int i, int j) const {
    const double om = m.dx * m.dy;
    const double sc = (m.aw ? m.eta * m.dts : 1.0) / om;
    const double sigma = m.aw ? 1.0 + m.eta * m.dts * m.a_t : m.a_t;
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k)
        D[r][k] = (r == k ? sigma : 0.0) + sc * (m.dy * (m.Ap[r][k] - m.Am[r][k]) + m.dx * (m.Bp[r][k] - m.Bm[r][k]));
    lower.clear();
    upper.clear();
    const int c = m.idx(i, j);
    auto blk = [&](const M4& X, double f) {
      M4 Y;
      for (int r = 0; r < 4; ++r)
        for (int k = 0; k < 4; ++k) Y[r][k] = f * X[r][k];
      return Y;
    };
    // L couples E_x^-1 (west) and E_y^-1 (south); U couples east and north
    const Nb w{m.idx(i - 1, j), blk(m.Ap, -sc * m.dy)}, s{m.idx(i, j - 1), blk(m.Bp, -sc * m.dx)};
    const Nb e{m.idx(i + 1, j), blk(m.Am, sc * m.dy)}, n{m.idx(i, j + 1), blk(m.Bm, sc * m.dx)};
    if (m.circulant) {
      lower.push_back(w);
      lower.push_back(s);
      upper.push_back(e);
      upper.push_back(n);
    } else {
      for (const Nb* q : {&w, &s, &e, &n}) (q->c < c ? lower : upper).push_back(*q);
    }
  }
  void apply_P(const std::vector<V4>& r, std::vector<V4>& z) const {
    const int n = m.nx * m.ny;
    std::vector<Nb> lo, up;
    M4 D;
    if (!m.circulant) {  // real lexicographic sweep
      std::vector<V4> y(n);
      for (int c = 0; c < n; ++c) {
        blocks(D, lo, up, c % m.nx, c / m.nx);
        V4 t = r[c];
        for (const Nb& b : lo) {
          const V4 v = matvec(b.B, y[b.c]);
          for (int k = 0; k < 4; ++k) t[k] -= v[k];
        }
        y[c] = solve4(D, t);
      }
      z.assign(n, V4{});
      for (int c = n - 1; c >= 0; --c) {
        blocks(D, lo, up, c % m.nx, c / m.nx);
        V4 t{};
        for (const Nb& b : up) {
          const V4 v = matvec(b.B, z[b.c]);
          for (int k = 0; k < 4; ++k) t[k] += v[k];
        }
        const V4 q = solve4(D, t);
        for (int k = 0; k < 4; ++k) z[c][k] = y[c][k] - q[k];
      }
      return;
    }
    // circulant: dense (D+L) D^-1 (D+U), solved with partial pivoting
    const int N = 4 * n;
    std::vector<double> DL(N * N, 0.0), DU(N * N, 0.0), Dinv(N * N, 0.0);
    for (int c = 0; c < n; ++c) {
      blocks(D, lo, up, c % m.nx, c / m.nx);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          DL[(4 * c + a) * N + 4 * c + b] += D[a][b];
          DU[(4 * c + a) * N + 4 * c + b] += D[a][b];
        }
      for (const Nb& q : lo)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) DL[(4 * c + a) * N + 4 * q.c + b] += q.B[a][b];
      for (const Nb& q : up)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) DU[(4 * c + a) * N + 4 * q.c + b] += q.B[a][b];
      for (int col = 0; col < 4; ++col) {
        V4 e{};
        e[col] = 1.0;
        const V4 x = solve4(D, e);
        for (int a = 0; a < 4; ++a) Dinv[(4 * c + a) * N + 4 * c + col] = x[a];
      }
    }
    std::vector<double> T(N * N, 0.0), P(N * N, 0.0);
    for (int a = 0; a < N; ++a)
      for (int k = 0; k < N; ++k) {
        const double v = DL[a * N + k];
        if (v != 0.0)
          for (int b = 0; b < N; ++b) T[a * N + b] += v * Dinv[k * N + b];
      }
    for (int a = 0; a < N; ++a)
      for (int k = 0; k < N; ++k) {
        const double v = T[a * N + k];
        if (v != 0.0)
          for (int b = 0; b < N; ++b) P[a * N + b] += v * DU[k * N + b];
      }
    std::vector<double> rhs(N);
    for (int c = 0; c < n; ++c)
      for (int a = 0; a < 4; ++a) rhs[4 * c + a] = r[c][a];
    for (int k = 0; k < N; ++k) {
      int piv = k;
      for (int a = k + 1; a < N; ++a)
        if (std::fabs(P[a * N + k]) > std::fabs(P[piv * N + k])) piv = a;
      if (piv != k) {
        for (int b = 0; b < N; ++b) std::swap(P[k * N + b], P[piv * N + b]);
        std::swap(rhs[k], rhs[piv]);
      }
      for (int a = k + 1; a < N; ++a) {
        const double f = P[a * N + k] / P[k * N + k];
        if (f == 0.0) continue;
        for (int b = k; b < N; ++b) P[a * N + b] -= f * P[k * N + b];
        rhs[a] -= f * rhs[k];
      }
    }
    std::vector<double> x(N);
    for (int a = N - 1; a >= 0; --a) {
      double acc = rhs[a];
      for (int b = a + 1; b < N; ++b) acc -= P[a * N + b] * x[b];
      x[a] = acc / P[a * N + a];
    }
    z.assign(n, V4{});
    for (int c = 0; c < n; ++c)
      for (int a = 0; a < 4; ++a) z[c][a] = x[4 * c + a];
  }
  // AW: z = W^-1 (dt* r); ARK: z = dt* P^-1 r (uniform dt*: the two orders coincide)
  void apply_Winv(const std::vector<V4>& r, std::vector<V4>& z) override {
    apply_P(r, z);
    for (auto& v : z)
      for (int k = 0; k < 4; ++k) v[k] *= m.dts;
  }
  void set_state(const std::vector<V4>& u0, double alpha, const std::vector<V4>& z) override {
    for (size_t c = 0; c < u.size(); ++c)
      for (int k = 0; k < 4; ++k) u[c][k] = u0[c][k] - alpha * z[c][k];
  }
};

}  // namespace orc

using namespace orc;

// ---------------------------------------------------------------- C interface
extern "C" {

void* or_create(int ni, int nj, int nw, const double* x, const double* y, const OrParams* p) {
  if (!p || ni <= 0 || nj <= 0 || p->nlevels < 1) return nullptr;
  const int f = 1 << (p->nlevels - 1);
  if (ni % f || nj % f || nw % f) return nullptr;
  auto* S = new Solver();
  S->P = *p;
  S->uinf = free_stream(p->mach, p->alpha_deg);
  S->lev.resize(p->nlevels);
  Level& fine = S->lev[p->nlevels - 1];
  fine.ni = ni;
  fine.nj = nj;
  fine.nw = nw;
  const size_t nv = (size_t)(ni + 1) * (nj + 1);
  S->x0.assign(x, x + nv);
  S->y0.assign(y, y + nv);
  fine_metrics(fine, x, y);
  for (int l = p->nlevels - 2; l >= 0; --l) agglomerate(S->lev[l + 1], S->lev[l]);
  for (auto& g : S->lev) alloc_level_state(g);
  for (auto& g : S->lev) {
    for (auto& v : g.u) v = S->uinf;
  }
  const double at = p->dt_phys > 0.0 ? (p->bdf_order == 1 ? 1.0 / p->dt_phys : 1.5 / p->dt_phys) : 0.0;
  for (auto& g : S->lev) g.a_t = at;
  return S;
}

void or_destroy(void* h) { delete static_cast<Solver*>(h); }

void or_free_stream(double mach, double alpha_deg, double* out) {
  const V4 w = free_stream(mach, alpha_deg);
  for (int k = 0; k < 4; ++k) out[k] = w[k];
}

int or_nlevels(void* h) { return (int)static_cast<Solver*>(h)->lev.size(); }

void or_level_dims(void* h, int l, int* ni, int* nj, int* nw) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  *ni = g.ni;
  *nj = g.nj;
  *nw = g.nw;
}

void or_get_metrics(void* h, int l, double* sxi_x, double* sxi_y, double* seta_x, double* seta_y, double* vol) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  std::memcpy(sxi_x, g.sxi_x.data(), g.sxi_x.size() * 8);
  std::memcpy(sxi_y, g.sxi_y.data(), g.sxi_y.size() * 8);
  std::memcpy(seta_x, g.seta_x.data(), g.seta_x.size() * 8);
  std::memcpy(seta_y, g.seta_y.data(), g.seta_y.size() * 8);
  std::memcpy(vol, g.vol.data(), g.vol.size() * 8);
}

// State arrays at the interface: 4 x nj x ni, component-major (SoA), interior cells.
void or_set_state(void* h, int l, const double* u) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  const int n = g.ni * g.nj;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i)
      for (int k = 0; k < 4; ++k) g.u[g.G(i, j)][k] = u[k * n + g.C(i, j)];
  bc_fill(*S, g);
}

void or_get_state(void* h, int l, double* u) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  const int n = g.ni * g.nj;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i)
      for (int k = 0; k < 4; ++k) u[k * n + g.C(i, j)] = g.u[g.G(i, j)][k];
}

// Ghosted state (ni+4) x (nj+4) per component, after the boundary fill.
void or_get_ghosted(void* h, int l, double* u) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  const int m = (g.ni + 4) * (g.nj + 4);
  for (int q = 0; q < m; ++q)
    for (int k = 0; k < 4; ++k) u[k * m + q] = g.u[q][k];
}

void or_set_forcing(void* h, int l, const double* s) {
  Level& g = static_cast<Solver*>(h)->lev[l];
  const int n = g.ni * g.nj;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) g.s[q][k] = s[k * n + q];
}

void or_get_forcing(void* h, int l, double* s) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  const int n = g.ni * g.nj;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) s[k * n + q] = g.s[q][k];
}

void or_set_mut(void* h, int l, const double* m) {
  Level& g = static_cast<Solver*>(h)->lev[l];
  for (int q = 0; q < g.ni * g.nj; ++q) g.mut[q] = m[q];
}

void or_get_mut(void* h, int l, double* m) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  for (int q = 0; q < g.ni * g.nj; ++q) m[q] = g.mut[q];
}

// Baldwin-Lomax on the finest level from its current state.
void or_compute_mut(void* h) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[S->L()];
  bc_fill(*S, g);
  baldwin_lomax(*S, g);
}

// Residual F = F^c + F^v (and the two parts) on level l; outputs may be null.
void or_residual(void* h, int l, double* F, double* Fc_out, double* Fv_out) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  std::vector<V4> Fc, Fv;
  residual(*S, g, l == S->L(), Fc, Fv);
  const int n = g.ni * g.nj;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) {
      if (F) F[k * n + q] = Fc[q][k] + Fv[q][k];
      if (Fc_out) Fc_out[k * n + q] = Fc[q][k];
      if (Fv_out) Fv_out[k * n + q] = Fv[q][k];
    }
}

// Complex-step directional derivative of the residual on level l: the residual functions
// evaluated at u + i hstep v (v: 4 x nj x ni, interior cells; the ghosts follow from the
// boundary conditions in complex arithmetic), F = Re F(u + i hstep v) (the residual itself, to
// rounding) and dF = Im F(u + i hstep v) / hstep = (dF/du) v with no differencing error for a
// tiny hstep (1e-30).  The eddy viscosity is held at its current value.
void or_residual_complex_step(void* h, int l, const double* v, double hstep, double* F, double* dF) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  const int ni = g.ni, nj = g.nj, n = ni * nj;
  std::vector<V4T<CX>> u(g.u.size());
  for (size_t k = 0; k < g.u.size(); ++k)
    for (int q = 0; q < 4; ++q) u[k][q] = CX(g.u[k][q], 0.0);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i)
      for (int q = 0; q < 4; ++q) u[g.G(i, j)][q] = CX(g.u[g.G(i, j)][q], hstep * v[q * n + g.C(i, j)]);
  bc_fill_t(*S, g, u);
  std::vector<V4T<CX>> Fc, Fv;
  residual_t(*S, g, u, l == S->L(), Fc, Fv);
  for (int c = 0; c < n; ++c)
    for (int q = 0; q < 4; ++q) {
      const CX f = Fc[c][q] + Fv[c][q];
      if (F) F[q * n + c] = f.real();
      dF[q * n + c] = f.imag() / hstep;
    }
}

// Force on the body through each wall face (j = 0 off the wake cut) of the finest level: the
// discrete momentum flux of the residual's j-face (central part minus dissipation minus the
// viscous part), with the opposite sign because the face vector points into the fluid.
// fx, fy: ni entries, zero on the cut.  The lift and drag objectives of the discrete adjoint
// are built from these (force coefficients from the scheme's own wall fluxes).
void or_wall_force(void* h, double* fx, double* fy) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[S->L()];
  bc_fill(*S, g);
  for (int i = 0; i < g.ni; ++i) {
    if (g.cut(i)) {
      fx[i] = fy[i] = 0.0;
      continue;
    }
    const FaceFlux f = S->P.flux == 1
                           ? fvs_face(*S, g.u[g.G(i, -1)], g.u[g.G(i, 0)], g.seta_x[g.FE(i, 0)],
                                      g.seta_y[g.FE(i, 0)], g.vfe[g.FE(i, 0)])
                           : jst_face(*S, g.u[g.G(i, -2)], g.u[g.G(i, -1)], g.u[g.G(i, 0)], g.u[g.G(i, 1)],
                                      g.seta_x[g.FE(i, 0)], g.seta_y[g.FE(i, 0)], g.vfe[g.FE(i, 0)],
                                      rtilde(g, i, -1, 1), rtilde(g, i, 0, 1), true);
    const V4 v = S->P.viscous ? visc_face(*S, g, i, 0) : V4{};
    fx[i] = -(f.hc[1] - f.hd[1] - v[1]);
    fy[i] = -(f.hc[2] - f.hd[2] - v[2]);
  }
}

void or_pseudo_dt(void* h, int l, double cfl, double* dts) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  pseudo_dt(*S, g, cfl);
  for (int q = 0; q < g.ni * g.nj; ++q) dts[q] = g.dts[q];
}

// Build dt* and the blocks from the current state, then apply the preconditioner to r.
// dense != 0 uses the independent dense assembly.  D_out (16 per cell, row-major) may be null.
void or_precond_apply(void* h, int l, double cfl, const double* r, double* z, int dense, double* D_out) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  pseudo_dt(*S, g, cfl);
  build_blocks(*S, g);
  const int n = g.ni * g.nj;
  std::vector<V4> rv(n), zv;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) rv[q][k] = r[k * n + q];
  if (dense == 2 || S->P.precond == 1) exact_apply(g, rv, zv); else if (dense) dense_apply(g, rv, zv); else sgs_apply(g, rv, zv);
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) z[k * n + q] = zv[q][k];
  if (D_out)
    for (int q = 0; q < n; ++q)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) D_out[16 * q + 4 * a + b] = g.D[q][a][b];
}

// Face blocks (A+, A- times |S|) built from the current state: i-faces then j-faces,
// 16 per block row-major.
// y = (D + L + U) x with the blocks built at level l's current state and pseudo CFL cfl.
void or_block_apply(void* h, int l, double cfl, const double* x, double* y) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  pseudo_dt(*S, g, cfl);
  build_blocks(*S, g);
  const int n = g.ni * g.nj;
  std::vector<V4> xv(n), yv;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) xv[q][k] = x[k * n + q];
  block_apply(g, xv, yv);
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) y[k * n + q] = yv[q][k];
}

void or_face_blocks(void* h, int l, double* axp, double* axm, double* aep, double* aem) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[l];
  bc_fill(*S, g);
  pseudo_dt(*S, g, 1.0);
  build_blocks(*S, g);
  for (size_t q = 0; q < g.Axp.size(); ++q)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        axp[16 * q + 4 * a + b] = g.Axp[q][a][b];
        axm[16 * q + 4 * a + b] = g.Axm[q][a][b];
      }
  for (size_t q = 0; q < g.Aep.size(); ++q)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        aep[16 * q + 4 * a + b] = g.Aep[q][a][b];
        aem[16 * q + 4 * a + b] = g.Aem[q][a][b];
      }
}

// nsteps smoothing steps on level l with pseudo CFL cfl; dense != 0 uses the dense preconditioner.
void or_smooth(void* h, int l, int nsteps, double cfl, int dense) {
  Solver* S = static_cast<Solver*>(h);
  for (int k = 0; k < nsteps; ++k) {
    Level& g = S->lev[l];
    bc_fill(*S, g);
    pseudo_dt(*S, g, cfl);
    build_blocks(*S, g);
    LevelOps op(*S, g, l == S->L(), dense != 0);
    stage_loop(op, S->P.nstages, S->P.alpha, S->P.beta);
    bc_fill(*S, g);
  }
}

// One FAS cycle from the finest level; returns the residual norm at its start.
double or_fas_cycle(void* h, int cycle_index) {
  Solver* S = static_cast<Solver*>(h);
  const double cfl = cycle_index < S->P.ramp_cycles ? std::min(S->P.cfl, S->P.cfl_ramp) : S->P.cfl;
  if (S->P.turb) {
    Level& g = S->lev[S->L()];
    bc_fill(*S, g);
    baldwin_lomax(*S, g);
  }
  S->record_norm = true;
  fas_cycle(*S, S->L(), cfl);
  S->record_norm = false;
  return S->norm_first;
}

// Cycles until norm <= drop * norm_0 or max_cycles; history[k] = norm at the start of cycle k.
int or_solve(void* h, double drop, int max_cycles, double* history) {
  double n0 = 0.0;
  for (int k = 0; k < max_cycles; ++k) {
    const double nk = or_fas_cycle(h, k);
    if (history) history[k] = nk;
    if (k == 0) n0 = nk;
    if (!(nk == nk)) return -(k + 1);
    if (nk <= drop * n0 && k > 0) return k + 1;
  }
  return max_cycles;
}

// Dual-time history source on the finest level (4 x n SoA) and a_t on every level.
void or_set_time_source(void* h, double a_t, const double* src) {
  Solver* S = static_cast<Solver*>(h);
  for (auto& g : S->lev) g.a_t = a_t;
  Level& g = S->lev[S->L()];
  const int n = g.ni * g.nj;
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k) g.src[q][k] = src ? src[k * n + q] : 0.0;
}

// ---- point functions exposed for pins
void or_conv_flux(const double* w, double sx, double sy, double* f) {
  const V4 r = conv_flux(V4{w[0], w[1], w[2], w[3]}, sx, sy);
  for (int k = 0; k < 4; ++k) f[k] = r[k];
}

void or_split_jacobians(const double* w, double sx, double sy, double d, double* Ap, double* Am) {
  M4 P, M;
  split_jacobians(V4{w[0], w[1], w[2], w[3]}, sx, sy, 0.0, d, P, M);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      Ap[4 * a + b] = P[a][b];
      Am[4 * a + b] = M[a][b];
    }
}

void or_eigvecs(const double* w, double nx, double ny, double* R, double* Ri) {
  M4 A, B;
  double vn, a;
  eigvecs(V4{w[0], w[1], w[2], w[3]}, nx, ny, A, B, vn, a);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      R[4 * r + c] = A[r][c];
      Ri[4 * r + c] = B[r][c];
    }
}

double or_cutoff(double lam, double a, double d) { return cutoff_abs(lam, a, d); }

double or_sensor(double qm, double q0, double qp) { return sensor_val(qm, q0, qp); }

void or_farfield_state(const double* wi, const double* winf, double nx, double ny, double* out) {
  const V4 b = farfield_state(V4{wi[0], wi[1], wi[2], wi[3]}, V4{winf[0], winf[1], winf[2], winf[3]}, nx, ny);
  for (int k = 0; k < 4; ++k) out[k] = b[k];
}

// The generic stage loop driven by a scalar linear problem: f^c = lc u, f^v = lv u,
// W^{-1} r = r / w.  Returns u after one step from u0 = 1 (the amplification factor).
double or_stage_scalar(int s, const double* alpha, const double* beta, double lc, double lv, double dts,
                       double w) {
  struct Scal : StageOps {
    double u, lc, lv, dts, w;
    void get_state(std::vector<V4>& v) override { v.assign(1, V4{u, 0, 0, 0}); }
    void residual(std::vector<V4>& fc, std::vector<V4>& fv) override {
      fc.assign(1, V4{lc * u, 0, 0, 0});
      fv.assign(1, V4{lv * u, 0, 0, 0});
    }
    void apply_Winv(const std::vector<V4>& r, std::vector<V4>& z) override {
      z.assign(1, V4{dts * r[0][0] / w, 0, 0, 0});
    }
    void set_state(const std::vector<V4>& u0, double al, const std::vector<V4>& z) override {
      u = u0[0][0] - al * z[0][0];
    }
  } op;
  op.u = 1.0;
  op.lc = lc;
  op.lv = lv;
  op.dts = dts;
  op.w = w;
  stage_loop(op, s, alpha, beta);
  return op.u;
}

// Restriction and prolongation exposed for pins (l = fine level index >= 1).
void or_restrict(void* h, int l, const double* vf, double* vc) {
  Solver* S = static_cast<Solver*>(h);
  const Level &f = S->lev[l], &c = S->lev[l - 1];
  const int nf = f.ni * f.nj, nc = c.ni * c.nj;
  std::vector<V4> a(nf), b;
  for (int q = 0; q < nf; ++q)
    for (int k = 0; k < 4; ++k) a[q][k] = vf[k * nf + q];
  restrict_vec(f, c, a, b, false);
  for (int q = 0; q < nc; ++q)
    for (int k = 0; k < 4; ++k) vc[k * nc + q] = b[q][k];
}

void or_prolong(void* h, int l, const double* dc, double* df) {
  Solver* S = static_cast<Solver*>(h);
  Level &f = S->lev[l], &c = S->lev[l - 1];
  const int nf = f.ni * f.nj, nc = c.ni * c.nj;
  std::vector<V4> d(nc);
  for (int q = 0; q < nc; ++q)
    for (int k = 0; k < 4; ++k) d[q][k] = dc[k * nc + q];
  std::vector<V4> save = f.u;
  for (auto& v : f.u) v = V4{};
  prolong_add(f, c, d);
  for (int j = 0; j < f.nj; ++j)
    for (int i = 0; i < f.ni; ++i)
      for (int k = 0; k < 4; ++k) df[k * nf + f.C(i, j)] = f.u[f.G(i, j)][k];
  f.u = save;
}

// Linear model: one smoothing step of the generic stage loop on u (4 x ny x nx SoA, in place).
// w: linearization state; d: cutoff; aw: 1 = AW (W blocks), 0 = ARK; circulant: 1 = wrap-around
// couplings in L and U (dense solve), 0 = real lexicographic sweep.  Mout (16, nullable): the
// dissipation matrix M used, Aout/Bout (16 each, nullable): the flux Jacobians used.
void or_linear_step(const double* w, double dx, double dy, int nx, int ny, double dts, double eta, double a_t,
                    double d, int aw, int circulant, int s, const double* alpha, const double* beta, double* u,
                    double* Aout, double* Bout, double* Mout) {
  LinModel m;
  m.nx = nx;
  m.ny = ny;
  m.dx = dx;
  m.dy = dy;
  m.dts = dts;
  m.eta = eta;
  m.a_t = a_t;
  m.aw = aw;
  m.circulant = circulant;
  const V4 st{w[0], w[1], w[2], w[3]};
  split_jacobians(st, 1.0, 0.0, 0.0, d, m.Ap, m.Am);
  split_jacobians(st, 0.0, 1.0, 0.0, d, m.Bp, m.Bm);
  for (int r = 0; r < 4; ++r)
    for (int k = 0; k < 4; ++k) {
      m.A[r][k] = m.Ap[r][k] + m.Am[r][k];
      m.B[r][k] = m.Bp[r][k] + m.Bm[r][k];
    }
  const Prim q = prim(st);
  const double a = std::sqrt(GAM * q.p / q.rho);
  m.eps4x = (std::fabs(q.u) + a) / 32.0;
  m.eps4y = (std::fabs(q.v) + a) / 32.0;
  // M of section 5.1: identity with last row (-(gamma-1)|v|^2/2, 0, 0, gamma)
  m.M = M4{};
  for (int k = 0; k < 3; ++k) m.M[k][k] = 1.0;
  m.M[3][0] = -(GAM - 1.0) * 0.5 * (q.u * q.u + q.v * q.v);
  m.M[3][3] = GAM;
  LinOps op(m);
  const int n = nx * ny;
  op.u.assign(n, V4{});
  for (int c = 0; c < n; ++c)
    for (int k = 0; k < 4; ++k) op.u[c][k] = u[k * n + c];
  stage_loop(op, s, alpha, beta);
  for (int c = 0; c < n; ++c)
    for (int k = 0; k < 4; ++k) u[k * n + c] = op.u[c][k];
  for (int r = 0; r < 4; ++r)
    for (int k = 0; k < 4; ++k) {
      if (Aout) Aout[4 * r + k] = m.A[r][k];
      if (Bout) Bout[4 * r + k] = m.B[r][k];
      if (Mout) Mout[4 * r + k] = m.M[r][k];
    }
}

// Rigid motion of the whole grid: rotation by phi about (xc, yc) at angular rate phidot
// (the pitching motion of section 6).  Metrics and face grid fluxes of every level follow.
void or_set_motion(void* h, double phi, double phidot, double xc, double yc) {
  Solver* S = static_cast<Solver*>(h);
  Level& f = S->lev[S->L()];
  const size_t nv = S->x0.size();
  std::vector<double> x(nv), y(nv);
  const double c = std::cos(phi), s = std::sin(phi);
  for (size_t k = 0; k < nv; ++k) {
    const double dx = S->x0[k] - xc, dy = S->y0[k] - yc;
    x[k] = xc + c * dx - s * dy;
    y[k] = yc + s * dx + c * dy;
  }
  fine_metrics(f, x.data(), y.data(), phidot, xc, yc);
  for (int l = S->L() - 1; l >= 0; --l) agglomerate(S->lev[l + 1], S->lev[l]);
  S->phi = phi;
  S->phidot = phidot;
  S->xc = xc;
  S->yc = yc;
  S->moving = true;
}

// One physical time step of dual time stepping (eq. nonlin-eq; section 6: implicit Euler for
// the first step, BDF2 afterwards) from the stored history to t + dt, with the grid already
// placed at t + dt by or_set_motion.  Pseudo-time FAS cycles until the residual has dropped
// by `drop` or max_cycles.  Returns the cycles run (negative on NaN); history[k] = norm of
// cycle k.  The first call takes the current state as u^n.
int or_dual_time_step(void* h, double dt, double drop, int max_cycles, double* history) {
  Solver* S = static_cast<Solver*>(h);
  Level& g = S->lev[S->L()];
  const int n = g.ni * g.nj;
  if (S->un.empty()) {
    S->un.resize(n);
    for (int j = 0; j < g.nj; ++j)
      for (int i = 0; i < g.ni; ++i) S->un[g.C(i, j)] = g.u[g.G(i, j)];
  }
  const bool bdf2 = S->steps_done > 0 && S->P.bdf_order == 2;
  const double a_t = bdf2 ? 1.5 / dt : 1.0 / dt;
  std::vector<double> src(4 * (size_t)n);
  for (int q = 0; q < n; ++q)
    for (int k = 0; k < 4; ++k)
      src[k * n + q] = bdf2 ? (-4.0 * S->un[q][k] + S->unm1[q][k]) / (2.0 * dt) : -S->un[q][k] / dt;
  or_set_time_source(h, a_t, src.data());
  const int nc = or_solve(h, drop, max_cycles, history);
  S->unm1 = S->un;
  for (int j = 0; j < g.nj; ++j)
    for (int i = 0; i < g.ni; ++i) S->un[g.C(i, j)] = g.u[g.G(i, j)];
  S->steps_done += 1;
  return nc;
}

// Face grid volume fluxes of level l (i-faces then j-faces), for pins.
void or_grid_fluxes(void* h, int l, double* vfx, double* vfe) {
  const Level& g = static_cast<Solver*>(h)->lev[l];
  std::memcpy(vfx, g.vfx.data(), g.vfx.size() * 8);
  std::memcpy(vfe, g.vfe.data(), g.vfe.size() * 8);
}

}  // extern "C"
