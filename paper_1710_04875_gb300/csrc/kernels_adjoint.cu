// Discrete adjoint of the steady finest-level residual (arXiv 1710.04875 gives the primal
// method; the adjoint is the standard one of a steady residual F(u, X) = 0 with an objective
// J(u, X): (dF/du)^T lambda = (dJ/du)^T, dJ/dX = dJ/dX|_u - lambda^T dF/dX).
//
// dF/du is assembled by central differences of the library's own FP64 residual kernels on
// groups of cells of one colour (no residual stencil holds two cells of a colour), so the
// Jacobian is that of exactly the discrete operator the smoother drives to zero, with the
// eddy viscosity frozen.  The transposed product is then an exact gather over the stored
// blocks.  The adjoint system is solved by restarted GMRES, right-preconditioned by the
// transpose of the primal AW preconditioner (flux-vector-split blocks with the eigenvalue
// cutoff, symmetric Gauss-Seidel factors) scaled to approximate J: Gauss-Seidel on the
// central-difference Jacobian itself is not usable, its diagonal blocks hold only the
// artificial dissipation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/fasw.h"
#include "fasw_adjoint.cuh"
#include "fasw_sweep.cuh"

namespace fasw {

namespace {

constexpr int RED_BLOCKS = 120;  // fixed grid of the deterministic reductions
constexpr int MAXV = 256;        // most vectors in one multi-dot (Krylov basis + 1)
constexpr size_t PARTS = (size_t)RED_BLOCKS * MAXV + 2 * MAXV;  // partials, row sums, coefficients

template <typename T>
int adj_alloc(std::vector<void*>& allocs, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (count ? count : 1) * sizeof(T)) != cudaSuccess) return FASW_ERR_OOM;
  allocs.push_back(q);
  *p = static_cast<T*>(q);
  return FASW_OK;
}

__device__ __forceinline__ int gidx_of(const LevelDev& L, int i, int j) { return (j + 2) * L.P + (i + 2); }

// L.u interior = base state, plus sgn * h at component m of the cells of colour k (k < 0: none).
__global__ void k_adj_set_state(LevelDev L, const double* ub, const int* col, int k, int m, double h_rel, double sgn) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, g = gidx_of(L, c % L.ni, c / L.ni);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = ub[q * n + c];
    if (q == m && col[c] == k) v += sgn * h_rel * fmax(1.0, fabs(v));
    L.u[q * L.Gn + g] = v;
  }
}

__global__ void k_adj_get_state(LevelDev L, double* ub) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, g = gidx_of(L, c % L.ni, c / L.ni);
#pragma unroll
  for (int q = 0; q < 4; ++q) ub[q * n + c] = L.u[q * L.Gn + g];
}

// Column m of the block of the unique colour-k dependency of every cell.
__global__ void k_adj_extract(int n, const int* nbr, const int* col, int k, int m, const double* Fp,
                              const double* Fm, const double* ub, double h_rel, double* J) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int s = 0; s < ADJ_SLOTS; ++s) {
    const int d = nbr[c * ADJ_SLOTS + s];
    if (d < 0 || col[d] != k) continue;
    const double h2 = 2.0 * h_rel * fmax(1.0, fabs(ub[m * n + d]));
    double* B = J + ((size_t)c * ADJ_SLOTS + s) * 16;
#pragma unroll
    for (int r = 0; r < 4; ++r) B[4 * r + m] = (Fp[r * n + c] - Fm[r * n + c]) / h2;
    return;
  }
}

// Objective gradients: wall face i depends on cells (i, 0) and (i, 1) only.
__global__ void k_adj_extract_obj(int ni, int n, const int* col, int k, int m, const double* fw, const double* ub,
                                  double h_rel, double sa, double ca, double* g) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  int x = -1;
  if (col[i] == k) x = i;
  if (col[ni + i] == k) x = ni + i;
  if (x < 0) return;
  const double h2 = 2.0 * h_rel * fmax(1.0, fabs(ub[m * n + x]));
  const double dfx = (fw[i] - fw[2 * ni + i]) / h2, dfy = (fw[ni + i] - fw[3 * ni + i]) / h2;
  g[m * n + x] = 2.0 * (-dfx * sa + dfy * ca);
  g[4 * (size_t)n + m * n + x] = 2.0 * (dfx * ca + dfy * sa);
}

// out = J v
__global__ void k_jac_mv(int n, const int* nbr, const double* J, const double* v, double* out) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = 0; s < ADJ_SLOTS; ++s) {
    const int d = nbr[c * ADJ_SLOTS + s];
    if (d < 0) continue;
    const double* B = J + ((size_t)c * ADJ_SLOTS + s) * 16;
    double vd[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) vd[m] = v[m * n + d];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[r] += B[4 * r + m] * vd[m];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) out[r * n + c] = acc[r];
}

// out = J^T v: every cell d gathers the blocks whose column is d.
__global__ void k_jac_tmv(int n, const int* rev_ptr, const int* rev, const double* J, const double* v, double* out) {
  pdl_entry();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = rev_ptr[d]; e < rev_ptr[d + 1]; ++e) {
    const int cs = rev[e], c = cs / ADJ_SLOTS;
    const double* B = J + (size_t)cs * 16;
    double vc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) vc[r] = v[r * n + c];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[m] += B[4 * r + m] * vc[r];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m * n + d] = acc[m];
}

// Preconditioner of the adjoint system: P = S^-1 W, with W the primal AW preconditioner
// (section 4: D + L + U from the flux-vector-split blocks with the eigenvalue cutoff, applied
// as the SGS product (D+L) D^-1 (D+U)) and S = eta dt* per cell, so that P ~ I/(eta dt*) +
// J_FVS approximates J.  For the transposed system, P^-T = S M^-T with
// M = D (I - G_L)(I - H_U) in the transfer blocks (tb: D^-1, G_W, G_S, H_E, H_N):
// a = (I - H_U)^-T r (forward, i+j order), b = (I - G_L)^-T a (backward), z = S D^-T b.
// H_U^T couples d to its west and south cells (their H_E, H_N) and, on the upper wake, to its
// mirror (its G_S); G_L^T couples d to its east and north cells (their G_W, G_S) and, on the
// lower wake, to its mirror.  That is the primal sweep's own dependence pattern, so the two
// triangular solves run in the primal's FP64 strip-pipelined sweep on transfer blocks built for
// the transposed couplings:
//   D' = I, G'_W(d) = H_E(w)^T, G'_S(d) = H_N(s)^T (on the wake cut: G_S(mirror)^T),
//   H'_E(d) = G_W(e)^T, H'_N(d) = G_S(n)^T,
// with w, s, e, n the west, south, east and north cells (zero blocks where there is none).
__device__ __forceinline__ double tbT(const double* tb, int n, int blk, int r, int q, int c) {
  return tb[(blk * 16 + 4 * r + q) * n + c];  // entry (r, q) of block blk of cell c
}

__global__ void k_adj_tb_transpose(LevelDev L, double* tbt) {
  pdl_entry();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = L.n, ni = L.ni, nj = L.nj, nw = L.nw;
  if (d >= n) return;
  const int i = d % ni, j = d / ni;
  const double* tb = L.tb;
  // source (block, cell) of each transposed block; cell -1: zero block
  int src_blk[5] = {0, 3, 4, 1, 2}, src_cell[5] = {-1, -1, -1, -1, -1};
  if (i > 0) src_cell[1] = d - 1;
  if (j > 0) {
    src_cell[2] = d - ni;
  } else if (nw > 0 && (i < nw || i >= ni - nw)) {
    src_blk[2] = 2;
    src_cell[2] = ni - 1 - i;
  }
  if (i < ni - 1) src_cell[3] = d + 1;
  if (j < nj - 1) src_cell[4] = d + ni;
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 4; ++q) tbt[(4 * r + q) * n + d] = r == q ? 1.0 : 0.0;
  for (int k = 1; k < 5; ++k) {
    const int c = src_cell[k];
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q)
        tbt[(k * 16 + 4 * r + q) * n + d] = c < 0 ? 0.0 : tbT(tb, n, src_blk[k], q, r, c);
  }
}

__global__ void k_adj_wt_finish(LevelDev L, const double* b, double* z) {
  pdl_entry();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= L.n) return;
  const int n = L.n;
  const double sc = L.coef[d] * L.vol[d];
  double bd[4];
  for (int t = 0; t < 4; ++t) bd[t] = b[t * n + d];
  for (int q = 0; q < 4; ++q) {
    double s = 0.0;
    for (int t = 0; t < 4; ++t) s += tbT(L.tb, n, 0, t, q, d) * bd[t];
    z[q * n + d] = sc * s;
  }
}

// FP32 copies of the transposed transfer blocks for the FP32 sweeps: entry-major (all five
// blocks; D' = I is what k_hp_cy reads) and, with hpF, hyperplane-major G'_W, G'_S | H'_E, H'_N
// (entry h = (i + j) nj + j, 16 floats per block, row-major).
__global__ void k_adj_tb_lower(int ni, int nj, const double* tbt, float* tb32, float* hpF, float* hpB) {
  pdl_entry();
  const int n = ni * nj;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  for (int e = 0; e < 80; ++e) tb32[(size_t)e * n + d] = float(tbt[(size_t)e * n + d]);
  if (!hpF) return;
  const int i = d % ni, j = d / ni;
  const size_t h = (size_t)(i + j) * nj + j;
  for (int k = 1; k < 5; ++k) {
    float* dst = (k <= 2 ? hpF : hpB) + 32 * h + ((k - 1) & 1) * 16;
    for (int e = 0; e < 16; ++e) dst[e] = float(tbt[(size_t)(k * 16 + e) * n + d]);
  }
}

// z = S D^-T b for the FP32 sweep's output b.
__global__ void k_adj_wt_finish32(LevelDev L, const float* b, double* z) {
  pdl_entry();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= L.n) return;
  const int n = L.n;
  const double sc = L.coef[d] * L.vol[d];
  double bd[4];
  for (int t = 0; t < 4; ++t) bd[t] = double(b[t * n + d]);
  for (int q = 0; q < 4; ++q) {
    double s = 0.0;
    for (int t = 0; t < 4; ++t) s += tbT(L.tb, n, 0, t, q, d) * bd[t];
    z[q * n + d] = sc * s;
  }
}

// Partial sums of dot(V_v, w) for v < nvec (grid RED_BLOCKS x nvec), then row reduction.
__global__ void k_multi_dot(const double* V, size_t ld, const double* w, int m, double* parts) {
  pdl_entry();
  __shared__ double red[256];
  const double* a = V + (size_t)blockIdx.y * ld;
  double s = 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < m; x += gridDim.x * blockDim.x) s += a[x] * w[x];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_rows_sum(const double* parts, int nblk, int nvec, double* out) {
  pdl_entry();
  const int v = threadIdx.x;
  if (v >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += parts[v * nblk + b];
  out[v] = s;
}

// w -= sum_v coef[v] V_v
__global__ void k_multi_axpy(const double* V, size_t ld, const double* coef, int nvec, int m, double* w) {
  pdl_entry();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= m) return;
  double s = w[x];
  for (int v = 0; v < nvec; ++v) s -= coef[v] * V[(size_t)v * ld + x];
  w[x] = s;
}

// y = a x + b y
__global__ void k_axpby(int m, double a, const double* x, double b, double* y) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y[i] = a * x[i] + b * y[i];
}

// Greedy distance-2 colouring (host): no residual stencil holds two cells of one colour.
int colour_cells(const std::vector<int>& nbr, const std::vector<std::vector<int>>& users, int n,
                 std::vector<int>& col) {
  col.assign(n, -1);
  int ncol = 0;
  std::vector<char> taken;
  for (int d = 0; d < n; ++d) {
    taken.assign(ncol + 1, 0);
    for (int c : users[d])
      for (int s = 0; s < ADJ_SLOTS; ++s) {
        const int x = nbr[c * ADJ_SLOTS + s];
        if (x >= 0 && col[x] >= 0) taken[col[x]] = 1;
      }
    int k = 0;
    while (k < ncol && taken[k]) ++k;
    col[d] = k;
    if (k == ncol) ++ncol;
  }
  return ncol;
}

}  // namespace

int adj_setup(AdjointDev& A, int ni, int nj, int nw, std::vector<void*>& allocs, cudaStream_t st) {
  const int n = ni * nj;
  std::vector<int> nbr((size_t)n * ADJ_SLOTS, -1);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      int* s = &nbr[((size_t)j * ni + i) * ADJ_SLOTS];
      s[0] = j * ni + i;
      const int di[4] = {-2, -1, 1, 2};
      for (int a = 0; a < 4; ++a) {
        if (i + di[a] >= 0 && i + di[a] < ni) s[1 + a] = j * ni + i + di[a];
        if (j + di[a] >= 0 && j + di[a] < nj) s[5 + a] = (j + di[a]) * ni + i;
      }
      const bool cut = nw > 0 && (i < nw || i >= ni - nw);
      if (cut && j <= 1) s[9] = ni - 1 - i;
      if (cut && j == 0) s[10] = ni + (ni - 1 - i);
    }
  std::vector<std::vector<int>> users(n);
  for (int c = 0; c < n; ++c)
    for (int s = 0; s < ADJ_SLOTS; ++s)
      if (nbr[(size_t)c * ADJ_SLOTS + s] >= 0) users[nbr[(size_t)c * ADJ_SLOTS + s]].push_back(c);
  std::vector<int> col;
  A.ncolours = colour_cells(nbr, users, n, col);
  std::vector<int> rev_ptr(n + 1, 0), rev;
  rev.reserve((size_t)n * ADJ_SLOTS);
  for (int d = 0; d < n; ++d) {
    rev_ptr[d] = (int)rev.size();
    for (int c : users[d])
      for (int s = 0; s < ADJ_SLOTS; ++s)
        if (nbr[(size_t)c * ADJ_SLOTS + s] == d) rev.push_back(c * ADJ_SLOTS + s);
  }
  rev_ptr[n] = (int)rev.size();
  A.ni = ni;
  A.nj = nj;
  A.n = n;
  int r;
  if ((r = adj_alloc(allocs, &A.nbr, nbr.size())) || (r = adj_alloc(allocs, &A.col, (size_t)n)) ||
      (r = adj_alloc(allocs, &A.rev_ptr, (size_t)n + 1)) || (r = adj_alloc(allocs, &A.rev, rev.size())) ||
      (r = adj_alloc(allocs, &A.J, (size_t)n * ADJ_SLOTS * 16)) ||
      (r = adj_alloc(allocs, &A.g, 8 * (size_t)n)) || (r = adj_alloc(allocs, &A.ub, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.Fp, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.Fm, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.fw, 4 * (size_t)ni)) || (r = adj_alloc(allocs, &A.parts, PARTS)) ||
      (r = adj_alloc(allocs, &A.mgs, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.mgy, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.mgt, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.mgz, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.tbt, 80 * (size_t)n)))
    return r;
  if (A.fp32) {
    if ((r = adj_alloc(allocs, &A.tb32, 80 * (size_t)n)) || (r = adj_alloc(allocs, &A.yz32, 4 * (size_t)n))) return r;
    if (hp_fits(ni, nj, nw)) {
      const size_t h = hp_floats(ni, nj);
      if ((r = adj_alloc(allocs, &A.hpF, 32 * h)) || (r = adj_alloc(allocs, &A.hpB, 32 * h)) ||
          (r = adj_alloc(allocs, &A.hpC, 4 * h)) || (r = adj_alloc(allocs, &A.hpY, 4 * h)))
        return r;
    }
  }
  if (cudaMallocHost(&A.h_parts, MAXV * sizeof(double)) != cudaSuccess) return FASW_ERR_OOM;
  cudaMemcpyAsync(A.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(A.col, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(A.rev_ptr, rev_ptr.data(), rev_ptr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(A.rev, rev.data(), rev.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(A.J, 0, (size_t)n * ADJ_SLOTS * 16 * sizeof(double), st);
  // the host vectors above are freed on return: wait for the copies
  return cudaStreamSynchronize(st) == cudaSuccess ? FASW_OK : FASW_ERR_CUDA;
}

int adj_assemble(AdjointDev& A, const LevelDev& L, const PhysParams& ph, double h_rel, cudaStream_t st,
                 long long& launches) {
  const int n = A.n, nb = (n + 127) / 128, nbf = (A.ni + 127) / 128;
  const double al = ph.alpha_deg * M_PI / 180.0, sa = std::sin(al), ca = std::cos(al);
  launch_pdl(k_adj_get_state, nb, 128, 0, st, L, A.ub);
  cudaMemsetAsync(A.g, 0, 8 * (size_t)n * sizeof(double), st);
  ++launches;
  ResArgs a{};
  a.mode = RES_FULL;
  for (int k = 0; k < A.ncolours; ++k)
    for (int m = 0; m < 4; ++m) {
      for (int sgn = 0; sgn < 2; ++sgn) {
        launch_pdl(k_adj_set_state, nb, 128, 0, st, L, A.ub, A.col, k, m, h_rel, sgn == 0 ? 1.0 : -1.0);
        launch_bc_aux(L, ph, 1.0, 0, st);
        a.F = sgn == 0 ? A.Fp : A.Fm;
        launch_residual(L, ph, a, st);
        launch_wall_force(L, ph, A.fw + 2 * sgn * A.ni, A.fw + (2 * sgn + 1) * A.ni, st);
        launches += 4;
      }
      launch_pdl(k_adj_extract, nb, 128, 0, st, n, A.nbr, A.col, k, m, A.Fp, A.Fm, A.ub, h_rel, A.J);
      launch_pdl(k_adj_extract_obj, nbf, 128, 0, st, A.ni, n, A.col, k, m, A.fw, A.ub, h_rel, sa, ca, A.g);
      launches += 2;
    }
  launch_pdl(k_adj_set_state, nb, 128, 0, st, L, A.ub, A.col, -1, 0, 0.0, 0.0);
  launch_bc_aux(L, ph, 1.0, 0, st);
  launches += 2;
  A.built = true;
  return cudaGetLastError() == cudaSuccess ? FASW_OK : FASW_ERR_CUDA;
}

void adj_apply(const AdjointDev& A, const double* v, double* out, int transpose, cudaStream_t st) {
  const int nb = (A.n + 127) / 128;
  if (transpose)
    launch_pdl(k_jac_tmv, nb, 128, 0, st, A.n, A.rev_ptr, A.rev, A.J, v, out);
  else
    launch_pdl(k_jac_mv, nb, 128, 0, st, A.n, A.nbr, A.J, v, out);
}

namespace {

// z = P^-T r (y: scratch of 4n): both triangular solves in one strip-pipelined FP64 sweep on
// the transposed transfer blocks (into y), then z = S D^-T y.
void precond(const AdjointDev& A, const double* r, double* y, double* z, cudaStream_t st) {
  LevelDev T = A.Lp;
  if (A.fp32) {  // FP32 transfer blocks: the hyperplane-staged sweep where the level fits, else strips
    T.tb = reinterpret_cast<double*>(A.tb32);
    T.yz32 = A.yz32;
    T.hpF = A.hpF;
    T.hpB = A.hpB;
    T.hpC = A.hpC;
    T.hpY = A.hpY;
    launch_sweep(T, 1, A.hpF ? SWEEP_HP : SWEEP_STRIPS, 0, 1, 0.0, r, A.prog, A.err, A.spin_limit, st);
    launch_pdl(k_adj_wt_finish32, (A.n + 127) / 128, 128, 0, st, A.Lp, (const float*)A.yz32, z);
    return;
  }
  T.tb = A.tbt;
  T.yz64 = y;
  launch_sweep(T, 0, SWEEP_STRIPS, 0, 1, 0.0, r, A.prog, A.err, A.spin_limit, st);
  launch_pdl(k_adj_wt_finish, (A.n + 127) / 128, 128, 0, st, A.Lp, (const double*)y, z);
}

// One smoothing step on J^T x = r from x (in place): the transposed primal stage loop,
// x_i = x_0 + c_i P^-T (r - J^T x_{i-1}), i = 1..s.  A plain Richardson step with P^-T is not
// stable; the stage polynomial is what makes the primal AW iteration converge, and
// P^-T J^T has the spectrum of J P^-1, hence of the primal's P^-1 J.
void smooth_step(AdjointDev& A, const double* r, double* x, cudaStream_t st) {
  const int m = 4 * A.n, nb = (m + 255) / 256;
  cudaMemcpyAsync(A.mgz, x, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int i = 0; i < A.nstages; ++i) {
    adj_apply(A, x, A.mgs, 1, st);
    launch_pdl(k_axpby, nb, 256, 0, st, m, 1.0, r, -1.0, A.mgs);  // s = r - J^T x
    precond(A, A.mgs, A.mgy, A.mgt, st);                            // t = P^-T s
    cudaMemcpyAsync(x, A.mgz, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_pdl(k_axpby, nb, 256, 0, st, m, A.stage_c[i], (const double*)A.mgt, 1.0, x);
  }
}

// x = M^-1 r: A.smooth_steps smoothing steps from zero (3 unless set otherwise).  As a
// stationary iteration these steps are not convergent on their own (the primal's stability also
// rests on its beta blending of the dissipative part, and on multigrid), but as a GMRES
// preconditioner they cut the Krylov iterations several-fold against one P^-T per iteration.
void steps_apply(AdjointDev& A, int steps, const double* r, double* x, cudaStream_t st) {
  cudaMemsetAsync(x, 0, 4 * (size_t)A.n * sizeof(double), st);
  for (int it = 0; it < steps; ++it) smooth_step(A, r, x, st);
}

// out[v] = dot(V_v, w), v < nvec (host values, synchronizes)
int multi_dot(AdjointDev& A, const double* V, size_t ld, int nvec, const double* w, int m, cudaStream_t st,
              double* out) {
  launch_pdl(k_multi_dot, dim3(RED_BLOCKS, nvec), 256, 0, st, V, ld, w, m, A.parts);
  launch_pdl(k_rows_sum, 1, MAXV, 0, st, A.parts, RED_BLOCKS, nvec, A.parts + (size_t)RED_BLOCKS * MAXV);
  if (cudaMemcpyAsync(A.h_parts, A.parts + (size_t)RED_BLOCKS * MAXV, nvec * sizeof(double), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FASW_ERR_CUDA;
  for (int v = 0; v < nvec; ++v) out[v] = A.h_parts[v];
  return FASW_OK;
}

}  // namespace

void adj_lincomb(int m, const double* x, double a, const double* v, double* out, cudaStream_t st) {
  cudaMemcpyAsync(out, x, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  launch_pdl(k_axpby, (m + 255) / 256, 256, 0, st, m, a, v, 1.0, out);
}

void adj_axpby(int m, double a, const double* x, double b, double* y, cudaStream_t st) {
  launch_pdl(k_axpby, (m + 255) / 256, 256, 0, st, m, a, x, b, y);
}

int adj_dot(AdjointDev& A, const double* a, const double* b, int m, cudaStream_t st, double* out) {
  return multi_dot(A, a, 0, 1, b, m, st, out);
}

int adj_force_coefficients(AdjointDev& A, const LevelDev& L, const PhysParams& ph, cudaStream_t st, double* cl,
                           double* cd, long long& launches) {
  launch_bc_aux(L, ph, 1.0, 0, st);
  launch_wall_force(L, ph, A.fw, A.fw + A.ni, st);
  launches += 2;
  std::vector<double> f(2 * (size_t)A.ni);
  if (cudaMemcpyAsync(f.data(), A.fw, f.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FASW_ERR_CUDA;
  double Fx = 0.0, Fy = 0.0;
  for (int i = 0; i < A.ni; ++i) {
    Fx += f[i];
    Fy += f[A.ni + i];
  }
  const double al = ph.alpha_deg * M_PI / 180.0;
  *cl = 2.0 * (-Fx * std::sin(al) + Fy * std::cos(al));
  *cd = 2.0 * (Fx * std::cos(al) + Fy * std::sin(al));
  return FASW_OK;
}

// GMRES(restart), right preconditioning, classical Gram-Schmidt applied twice.
void adj_build_precond(AdjointDev& A, const LevelDev& L, const PhysParams& ph, const SchemeParams& sc, double cfl,
                       cudaStream_t st, long long& launches) {
  // the primal W (additive-W form) at the current state, FP64, with pseudo CFL cfl
  SchemeParams aw = sc;
  aw.aw = 1;
  launch_bc_aux(L, ph, cfl, 1, st);
  launch_face_blocks(L, ph, aw, 0, st);
  launch_diag_blocks(L, aw, 0, st);
  launch_sgs_prep(L, 0, SWEEP_STRIPS, st);
  launch_pdl(k_adj_tb_transpose, (A.n + 127) / 128, 128, 0, st, L, A.tbt);
  launches += 5;
  if (A.fp32) {
    launch_pdl(k_adj_tb_lower, (A.n + 127) / 128, 128, 0, st, A.ni, A.nj, (const double*)A.tbt, A.tb32, A.hpF, A.hpB);
    ++launches;
  }
  A.Lp = L;
  A.nstages = sc.nstages;
  for (int i = 0; i < 5; ++i) A.stage_c[i] = i < sc.nstages ? sc.alpha[i] / sc.eta : 0.0;
}

void adj_precond(const AdjointDev& A, const double* r, double* scratch, double* z, cudaStream_t st) {
  precond(A, r, scratch, z, st);
}

void adj_steps_apply(AdjointDev& A, int steps, const double* r, double* z, cudaStream_t st) {
  if (steps <= 0)
    precond(A, r, A.mgy, z, st);
  else
    steps_apply(A, steps, r, z, st);
}

int adj_solve(AdjointDev& A, const LevelDev& L, const PhysParams& ph, const SchemeParams& sc, double cfl,
              const double* g, double* lam, double tol, int max_iters, int restart, std::vector<void*>& allocs,
              cudaStream_t st, int* iters, double* relres, long long& launches) {
  adj_build_precond(A, L, ph, sc, cfl, st, launches);
  auto apply_m = [&](const double* rr, double* zz) {  // zz = M^-1 rr
    steps_apply(A, A.smooth_steps, rr, zz, st);
  };
  const int m = 4 * A.n;
  if (restart < 1 || restart > MAXV - 5) return FASW_ERR_ARG;
  if (A.restart < restart) {
    int r = adj_alloc(allocs, &A.kry, (size_t)(2 * restart + 5) * m);
    if (r) return r;
    A.restart = restart;
  }
  const size_t ld = m;
  double* V = A.kry;                                  // restart + 1 vectors
  double* Z = A.kry + (size_t)(A.restart + 1) * ld;   // restart preconditioned vectors
  double* w = Z + (size_t)A.restart * ld;             // work
  double* res = w + ld;
  const int nb = (m + 255) / 256;
  cudaMemsetAsync(lam, 0, m * sizeof(double), st);
  cudaMemcpyAsync(res, g, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  double beta0 = 0.0, beta = 0.0;
  int r = adj_dot(A, res, res, m, st, &beta0);
  if (r) return r;
  beta0 = std::sqrt(beta0);
  beta = beta0;
  *iters = 0;
  *relres = 0.0;
  if (beta0 == 0.0) return FASW_OK;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), s(restart + 1), h(restart + 1),
      h2(restart + 1);
  double* d_coef = A.parts + (size_t)RED_BLOCKS * MAXV + MAXV;  // up to MAXV coefficients
  while (*iters < max_iters) {
    launch_pdl(k_axpby, nb, 256, 0, st, m, 1.0 / beta, res, 0.0, V);
    std::fill(s.begin(), s.end(), 0.0);
    s[0] = beta;
    int jdone = 0;
    bool conv = false;
    for (int j = 0; j < restart && *iters < max_iters; ++j) {
      double* zj = Z + (size_t)j * ld;
      apply_m(V + (size_t)j * ld, zj);            // z_j = M^-1 v_j
      adj_apply(A, zj, w, 1, st);                  // w = J^T z_j
      launches += 3;
      for (int pass = 0; pass < 2; ++pass) {
        if ((r = multi_dot(A, V, ld, j + 1, w, m, st, pass == 0 ? h.data() : h2.data()))) return r;
        cudaMemcpyAsync(d_coef, pass == 0 ? h.data() : h2.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, st);
        launch_pdl(k_multi_axpy, nb, 256, 0, st, V, ld, d_coef, j + 1, m, w);
        launches += 3;
      }
      for (int i = 0; i <= j; ++i) H[(size_t)i * restart + j] = h[i] + h2[i];
      double hn = 0.0;
      if ((r = adj_dot(A, w, w, m, st, &hn))) return r;
      hn = std::sqrt(hn);
      H[(size_t)(j + 1) * restart + j] = hn;
      if (hn > 0.0) launch_pdl(k_axpby, nb, 256, 0, st, m, 1.0 / hn, w, 0.0, V + (size_t)(j + 1) * ld);
      ++launches;
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double a = H[(size_t)i * restart + j], b = H[(size_t)(i + 1) * restart + j];
        H[(size_t)i * restart + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * restart + j], b = H[(size_t)(j + 1) * restart + j];
      const double rho = std::hypot(a, b);
      cs[j] = rho > 0.0 ? a / rho : 1.0;
      sn[j] = rho > 0.0 ? b / rho : 0.0;
      H[(size_t)j * restart + j] = rho;
      H[(size_t)(j + 1) * restart + j] = 0.0;
      s[j + 1] = -sn[j] * s[j];
      s[j] = cs[j] * s[j];
      ++*iters;
      jdone = j + 1;
      if (std::fabs(s[j + 1]) <= tol * beta0 || hn == 0.0) {
        conv = true;
        break;
      }
    }
    // y = H^-1 s (upper triangular), lam += Z y
    std::vector<double> yv(jdone);
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = s[i];
      for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * restart + k] * yv[k];
      yv[i] = acc / H[(size_t)i * restart + i];
    }
    for (int i = 0; i < jdone; ++i) yv[i] = -yv[i];  // k_multi_axpy subtracts
    cudaMemcpyAsync(d_coef, yv.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, st);
    launch_pdl(k_multi_axpy, nb, 256, 0, st, Z, ld, d_coef, jdone, m, lam);
    // true residual g - J^T lam
    adj_apply(A, lam, res, 1, st);
    launch_pdl(k_axpby, nb, 256, 0, st, m, 1.0, g, -1.0, res);
    launches += 5;
    if ((r = adj_dot(A, res, res, m, st, &beta))) return r;
    beta = std::sqrt(beta);
    *relres = beta / beta0;
    if (beta <= tol * beta0) return FASW_OK;
    (void)conv;  // the Krylov estimate said converged but the true residual did not: restart
  }
  return *relres <= tol ? FASW_OK : FASW_ERR_NOT_CONVERGED;
}

}  // namespace fasw
