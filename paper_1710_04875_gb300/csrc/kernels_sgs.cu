// Flux-vector-split face Jacobians with the parabolic eigenvalue cutoff, block diagonal
// LU, and the block SGS sweeps of the preconditioner (section 4.4 of arXiv 1710.04875).
//
// Face blocks use a closed form instead of R diag(lambda) R^-1: with r0 = (1, u, v, H),
// r1 = (0, nx, ny, vn), dp = (gamma-1)(q^2/2, -u, -v, 1) (so dp.du = dp) and
// dvn = (-vn, nx, ny, 0) (so dvn.du = rho dvn), every matrix R diag(l) R^-1 with
// eigenvalue pattern (l1, l1, l3, l4) on the entropy, shear and acoustic waves equals
//   M(l) = l1 I + r0 (c1/a^2 dp + c2/a dvn)^T + r1 (c2/a dp + c1 dvn)^T,
//   c1 = (l3 + l4)/2 - l1,  c2 = (l3 - l4)/2.
// M is linear in l, so A+- = M(l+-) with l+-_k = (lambda_k +- |lambda_k|_cut)/2.
//
// The sweeps follow the hyperplane order i + j = const; on a hyperplane the cells are
// independent, and the lower/upper neighbour sets of every cell are those of the
// lexicographic ordering, so the result equals the lexicographic Gauss-Seidel sweep.
#include "fasw_internal.cuh"

namespace fasw {

namespace {

__device__ __forceinline__ int gidx(const LevelDev& L, int i, int j) { return (j + 2) * L.P + (i + 2); }
__device__ __forceinline__ bool on_cut(const LevelDev& L, int i) { return L.nw > 0 && (i < L.nw || i >= L.ni - L.nw); }

template <typename T>
__device__ __forceinline__ T cutabs(T lam, T a, T d) {
  const T al = fabs(lam);
  const T ad = a * d;
  if (d > T(0) && al <= ad) return T(0.5) * (ad + lam * lam / ad);
  return al;
}

// Writes |S| A+ and |S| A- (row-major 4x4) for state w and area vector (sx, sy).
// vf: grid volume flux of the face; the eigenvalues are those of the relative normal velocity.
template <typename T>
__device__ void split_blocks(const T w[4], T sx, T sy, T vf, T d, T Ap[16], T Am[16]) {
  const T g1 = T(GAM - 1.0);
  const T len = sqrt(sx * sx + sy * sy);
  const T nx = sx / len, ny = sy / len;
  const T rho = w[0], u = w[1] / rho, v = w[2] / rho;
  const T q2 = u * u + v * v;
  const T p = g1 * (w[3] - T(0.5) * rho * q2);
  const T a = sqrt(T(GAM) * p / rho);
  const T H = (w[3] + p) / rho;
  const T vn = u * nx + v * ny;
  const T r0[4] = {T(1), u, v, H};
  const T r1[4] = {T(0), nx, ny, vn};
  const T dp[4] = {g1 * T(0.5) * q2, -g1 * u, -g1 * v, g1};
  const T dv[4] = {-vn, nx, ny, T(0)};
  const T vr = vn - vf / len;
  const T lam1 = vr, lam3 = vr + a, lam4 = vr - a;
  const T m1 = cutabs(lam1, a, d), m3 = cutabs(lam3, a, d), m4 = cutabs(lam4, a, d);
  const T inva = T(1) / a, inva2 = inva * inva;
#pragma unroll
  for (int sgn = 0; sgn < 2; ++sgn) {
    const T s = sgn == 0 ? T(1) : T(-1);
    const T l1 = T(0.5) * (lam1 + s * m1), l3 = T(0.5) * (lam3 + s * m3), l4 = T(0.5) * (lam4 + s * m4);
    const T c1 = T(0.5) * (l3 + l4) - l1, c2 = T(0.5) * (l3 - l4);
    T g0[4], gg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g0[k] = c1 * inva2 * dp[k] + c2 * inva * dv[k];
      gg[k] = c2 * inva * dp[k] + c1 * dv[k];
    }
    T* M = sgn == 0 ? Ap : Am;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) M[4 * r + c] = len * ((r == c ? l1 : T(0)) + r0[r] * g0[c] + r1[r] * gg[c]);
  }
}

// Thin-layer viscous Jacobian of j-face (i, j) in scalar form: nu |S|^2 / Omega_f with
// nu = max(mu + mu_t, gamma (mu/Pr + mu_t/Pr_t)) / rho; added as +V I to A+ and -V I to A-.
__device__ double visc_radius(const LevelDev& L, const PhysParams& ph, int i, int j, double rho) {
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
  const double mu = ph.inv_re;
  const double nu = fmax(mu + mutf, GAM * (mu * ph.inv_pr + mutf * ph.inv_prt)) / rho;
  const int f = j * ni + i;
  const double sx = L.seta[f], sy = L.seta[L.nfe + f];
  return 2.0 * nu * (sx * sx + sy * sy) / (volL + volR);
}

template <typename T>
__global__ void k_face_blocks(LevelDev L, PhysParams ph, T* blk, T d) {
  pdl_entry();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int ni = L.ni;
  if (f >= L.nfx + L.nfe) return;
  int gL, gR;
  double sx, sy, vf;
  T *Ap, *Am;
  int stride;
  if (f < L.nfx) {
    const int i = f % (ni + 1), j = f / (ni + 1);
    gL = gidx(L, i - 1, j);
    gR = gidx(L, i, j);
    sx = L.sxi[f];
    sy = L.sxi[L.nfx + f];
    vf = L.vfx[f];
    Ap = blk + f;
    Am = blk + 16 * L.nfx + f;
    stride = L.nfx;
  } else {
    const int e = f - L.nfx;
    const int i = e % ni, j = e / ni;
    gL = gidx(L, i, j - 1);
    gR = gidx(L, i, j);
    sx = L.seta[e];
    sy = L.seta[L.nfe + e];
    vf = L.vfe[e];
    Ap = blk + 32 * L.nfx + e;
    Am = blk + 32 * L.nfx + 16 * L.nfe + e;
    stride = L.nfe;
  }
  double wd[4];
  T w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wd[k] = 0.5 * (L.u[k * L.Gn + gL] + L.u[k * L.Gn + gR]);
    w[k] = T(wd[k]);
  }
  T P[16], M[16];
  split_blocks<T>(w, T(sx), T(sy), T(vf), d, P, M);
  if (ph.viscous && f >= L.nfx) {
    const int e = f - L.nfx;
    const T V = T(visc_radius(L, ph, e % ni, e / ni, wd[0]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      P[5 * k] += V;
      M[5 * k] -= V;
    }
  }
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    Ap[e * stride] = P[e];
    Am[e * stride] = M[e];
  }
}

// D_i = sigma I + c_i (A+_e - A-_w + B+_n - B-_s), LU without pivoting (unit L below the
// diagonal, U on and above with the reciprocal of its diagonal stored on the diagonal).
template <typename T>
__global__ void k_diag_blocks(LevelDev L, const T* blk, T* dlu, int aw, double eta) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  double coef, sigma;
  if (aw) {
    coef = eta * L.dts[c] / L.vol[c];
    sigma = 1.0 + eta * L.dts[c] * L.a_t;
  } else {
    coef = 1.0 / L.vol[c];
    sigma = L.a_t;
  }
  L.coef[c] = coef;
  {  // u^(0) of the smoothing step (the state the blocks are frozen at)
    const int g = (j + 2) * L.P + (i + 2);
#pragma unroll
    for (int k = 0; k < 4; ++k) L.u0[k * L.n + c] = L.u[k * L.Gn + g];
  }
  const int fw = j * (ni + 1) + i, fe = fw + 1, fs = j * ni + i, fn = fs + ni;
  const T* Axp = blk;
  const T* Axm = blk + 16 * L.nfx;
  const T* Aep = blk + 32 * L.nfx;
  const T* Aem = blk + 32 * L.nfx + 16 * L.nfe;
  T A[16];
  const T cf = T(coef);
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const T v = (Axp[e * L.nfx + fe] - Axm[e * L.nfx + fw]) + (Aep[e * L.nfe + fn] - Aem[e * L.nfe + fs]);
    A[e] = ((e % 5 == 0) ? T(sigma) : T(0)) + cf * v;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int r = k + 1; r < 4; ++r) {
      const T m = A[4 * r + k] / A[4 * k + k];
      A[4 * r + k] = m;
#pragma unroll
      for (int cc = k + 1; cc < 4; ++cc) A[4 * r + cc] -= m * A[4 * k + cc];
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) A[5 * k] = T(1) / A[5 * k];
#pragma unroll
  for (int e = 0; e < 16; ++e) dlu[e * L.n + c] = A[e];
}

template <typename T>
__device__ __forceinline__ void lu_solve(const T* dlu, int n, int c, T b[4]) {
  T A[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) A[e] = dlu[e * n + c];
#pragma unroll
  for (int r = 1; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < r; ++k) b[r] -= A[4 * r + k] * b[k];
#pragma unroll
  for (int r = 3; r >= 0; --r) {
    T s = b[r];
#pragma unroll
    for (int k = r + 1; k < 4; ++k) s -= A[4 * r + k] * b[k];
    b[r] = s * A[5 * r];
  }
}

template <typename T>
__device__ __forceinline__ void matvec_acc(const T* B, int stride, int f, const T* y, int n, int cy, T s, T acc[4]) {
  T yv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) yv[k] = y[k * n + cy];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    T t = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) t += B[(4 * r + k) * stride + f] * yv[k];
    acc[r] += s * t;
  }
}

// Single-CTA wavefront: forward (D+L) y = r over hyperplanes k = i + j ascending, then
// backward (D+U) z = D y descending, z overwriting y; optional fused stage update.
template <typename T>
__global__ void k_sgs_single(LevelDev L, const T* blk, const T* dlu, T* yz, const double* r_in,
                             int do_update, int aw, double alpha) {
  pdl_entry();
  const int ni = L.ni, nj = L.nj, n = L.n;
  const T* Axp = blk;
  const T* Axm = blk + 16 * L.nfx;
  const T* Aep = blk + 32 * L.nfx;
  const T* Aem = blk + 32 * L.nfx + 16 * L.nfe;
  const int nk = ni + nj - 1;
  for (int k = 0; k < nk; ++k) {
    const int ilo = max(0, k - nj + 1), ihi = min(k, ni - 1);
    for (int i = ilo + (int)threadIdx.x; i <= ihi; i += blockDim.x) {
      const int j = k - i;
      const int c = j * ni + i;
      const T cf = T(L.coef[c]);
      T t[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] = T(r_in[q * n + c]);
      if (i > 0) matvec_acc<T>(Axp, L.nfx, j * (ni + 1) + i, yz, n, c - 1, cf, t);
      if (j > 0) {
        matvec_acc<T>(Aep, L.nfe, j * ni + i, yz, n, c - ni, cf, t);
      } else if (on_cut(L, i) && ni - 1 - i < i) {
        matvec_acc<T>(Aep, L.nfe, i, yz, n, ni - 1 - i, cf, t);
      }
      lu_solve<T>(dlu, n, c, t);
#pragma unroll
      for (int q = 0; q < 4; ++q) yz[q * n + c] = t[q];
    }
    __syncthreads();
  }
  for (int k = nk - 1; k >= 0; --k) {
    const int ilo = max(0, k - nj + 1), ihi = min(k, ni - 1);
    for (int i = ilo + (int)threadIdx.x; i <= ihi; i += blockDim.x) {
      const int j = k - i;
      const int c = j * ni + i;
      const T cf = T(L.coef[c]);
      T t[4] = {T(0), T(0), T(0), T(0)};
      if (i < ni - 1) matvec_acc<T>(Axm, L.nfx, j * (ni + 1) + i + 1, yz, n, c + 1, cf, t);
      if (j == 0 && on_cut(L, i) && ni - 1 - i > i) matvec_acc<T>(Aep, L.nfe, i, yz, n, ni - 1 - i, -cf, t);
      if (j < nj - 1) matvec_acc<T>(Aem, L.nfe, (j + 1) * ni + i, yz, n, c + ni, cf, t);
      lu_solve<T>(dlu, n, c, t);
      T z[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        z[q] = yz[q * n + c] - t[q];
        yz[q * n + c] = z[q];
      }
      if (do_update) {
        const double sc = aw ? alpha : alpha * L.dts[c];
        const int g = (j + 2) * L.P + (i + 2);
#pragma unroll
        for (int q = 0; q < 4; ++q) L.u[q * L.Gn + g] = L.u0[q * n + c] - sc * double(z[q]);
      }
    }
    __syncthreads();
  }
}

}  // namespace

void launch_face_blocks(const LevelDev& L, const PhysParams& ph, const SchemeParams& sc, int mixed, cudaStream_t st) {
  const int nf = L.nfx + L.nfe;
  if (mixed)
    launch_pdl(k_face_blocks<float>, (nf + 63) / 64, 64, 0, st, L, ph, L.blk32, float(sc.d_cut));
  else
    launch_pdl(k_face_blocks<double>, (nf + 63) / 64, 64, 0, st, L, ph, L.blk64, sc.d_cut);
}

void launch_diag_blocks(const LevelDev& L, const SchemeParams& sc, int mixed, cudaStream_t st) {
  if (mixed)
    launch_pdl(k_diag_blocks<float>, (L.n + 63) / 64, 64, 0, st, L, L.blk32, L.dlu32, sc.aw, sc.eta);
  else
    launch_pdl(k_diag_blocks<double>, (L.n + 63) / 64, 64, 0, st, L, L.blk64, L.dlu64, sc.aw, sc.eta);
}

void launch_sgs(const LevelDev& L, const SchemeParams& sc, int mixed, int do_update, double alpha,
                const double* r_in, double* z_out, cudaStream_t st) {
  const int threads = 128;
  if (mixed) {
    launch_pdl(k_sgs_single<float>, 1, threads, 0, st, L, L.blk32, L.dlu32, L.yz32, r_in, do_update, sc.aw, alpha);
  } else {
    launch_pdl(k_sgs_single<double>, 1, threads, 0, st, L, L.blk64, L.dlu64, L.yz64, r_in, do_update, sc.aw, alpha);
  }
  (void)z_out;
}

}  // namespace fasw
