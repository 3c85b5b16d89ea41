// Discrete adjoint of the steady finest-level residual (arXiv 1710.04875 gives the primal
// method; the adjoint is the standard one of a steady residual F(u, X) = 0 with an objective
// J(u, X): (dF/du)^T lambda = (dJ/du)^T, dJ/dX = dJ/dX|_u - lambda^T dF/dX).
//
// dF/du is assembled by central differences of the library's own FP64 residual kernels on
// groups of cells of one colour (no residual stencil holds two cells of a colour), so the
// Jacobian is that of exactly the discrete operator the smoother drives to zero, with the
// eddy viscosity frozen.  The transposed product is then an exact gather over the stored
// blocks (the dissipative part's Jacobian is kept apart as well, for the smoother's beta
// blending).  The adjoint system is solved by flexible GMRES, right-preconditioned by the
// exact transpose of the primal's linearised FAS cycle: the transposed AW smoothing step (the
// primal's flux-vector-split SGS preconditioner with the eigenvalue cutoff, run transposed)
// on every level, with transposed restriction and prolongation and coarse Jacobians at the
// restricted state.  Gauss-Seidel on the central-difference Jacobian itself is not usable, its
// diagonal blocks hold only the artificial dissipation.  Also here: the vertex colouring of the
// transposed grid product (dF/dX)^T lambda.
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
  const int r = device_alloc(&q, (count ? count : 1) * sizeof(T));
  if (r != FASW_OK) return r;
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
  int r;
  if ((r = adj_alloc(allocs, &A.nbr, nbr.size())) || (r = adj_alloc(allocs, &A.col, (size_t)n)) ||
      (r = adj_alloc(allocs, &A.rev_ptr, (size_t)n + 1)) || (r = adj_alloc(allocs, &A.rev, rev.size())) ||
      (r = adj_alloc(allocs, &A.J, (size_t)n * ADJ_SLOTS * 16)) ||
      (r = adj_alloc(allocs, &A.g, 8 * (size_t)n)) || (r = adj_alloc(allocs, &A.ub, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.Fp, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.Fm, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.fw, 4 * (size_t)ni)) || (r = adj_alloc(allocs, &A.parts, PARTS)) ||
      (r = adj_alloc(allocs, &A.mgs, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.mgy, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.mgt, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.mgz, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.tbt, 80 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.Jv, (size_t)n * ADJ_SLOTS * 16)) || (r = adj_alloc(allocs, &A.Fvp, 4 * (size_t)n)) ||
      (r = adj_alloc(allocs, &A.Fvm, 4 * (size_t)n)) || (r = adj_alloc(allocs, &A.mgw, 32 * (size_t)n)))
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
  cudaMemsetAsync(A.Jv, 0, (size_t)n * ADJ_SLOTS * 16 * sizeof(double), st);
  // the host vectors above are freed on return: wait for the copies
  if (cudaStreamSynchronize(st) != cudaSuccess) return FASW_ERR_CUDA;
  A.n = n;  // published last: a failed set-up is redone by the next call
  return FASW_OK;
}

int adj_assemble(AdjointDev& A, const LevelDev& L, const PhysParams& ph, double h_rel, cudaStream_t st,
                 long long& launches) {
  const int n = A.n, nb = (n + 127) / 128, nbf = (A.ni + 127) / 128;
  const double al = ph.alpha_deg * M_PI / 180.0, sa = std::sin(al), ca = std::cos(al);
  launch_pdl(k_adj_get_state, nb, 128, 0, st, L, A.ub);
  cudaMemsetAsync(A.g, 0, 8 * (size_t)n * sizeof(double), st);
  ++launches;
  if (A.jac_mode == 1 && A.tan.u) {
    // Forward mode: one tangent evaluation per colour and component, seeded with
    // 2 h max(1, |u|) so that the central-difference extraction (F+ - F-) / (2 h max(1, |u|))
    // with F- = 0 reads the exact Jacobian columns.
    cudaMemsetAsync(A.Fm, 0, 4 * (size_t)n * sizeof(double), st);
    cudaMemsetAsync(A.Fvm, 0, 4 * (size_t)n * sizeof(double), st);
    cudaMemsetAsync(A.fw + 2 * A.ni, 0, 2 * (size_t)A.ni * sizeof(double), st);
    launch_bc_aux(L, ph, 1.0, 0, st);
    ++launches;
    for (int k = 0; k < A.ncolours; ++k)
      for (int m = 0; m < 4; ++m) {
        launch_tangent(L, A.tan, ph, nullptr, A.col, k, m, 2.0 * h_rel, A.Fp, A.Fvp, nullptr,
                       A.finest ? A.fw : nullptr, A.finest ? A.fw + A.ni : nullptr, st);
        launches += A.finest ? 6 : 5;
        launch_pdl(k_adj_extract, nb, 128, 0, st, n, A.nbr, A.col, k, m, A.Fp, A.Fm, A.ub, h_rel, A.J);
        launch_pdl(k_adj_extract, nb, 128, 0, st, n, A.nbr, A.col, k, m, (const double*)A.Fvp, (const double*)A.Fvm,
                   (const double*)A.ub, h_rel, A.Jv);
        launches += 2;
        if (A.finest) {
          launch_pdl(k_adj_extract_obj, nbf, 128, 0, st, A.ni, n, A.col, k, m, A.fw, A.ub, h_rel, sa, ca, A.g);
          ++launches;
        }
      }
    A.built = true;
    return cudaGetLastError() == cudaSuccess ? FASW_OK : FASW_ERR_CUDA;
  }
  ResArgs a{};
  a.mode = RES_FULL;
  for (int k = 0; k < A.ncolours; ++k)
    for (int m = 0; m < 4; ++m) {
      for (int sgn = 0; sgn < 2; ++sgn) {
        launch_pdl(k_adj_set_state, nb, 128, 0, st, L, A.ub, A.col, k, m, h_rel, sgn == 0 ? 1.0 : -1.0);
        launch_bc_aux(L, ph, 1.0, 0, st);
        a.F = sgn == 0 ? A.Fp : A.Fm;
        a.Fv = sgn == 0 ? A.Fvp : A.Fvm;
        launch_residual(L, ph, a, st);
        launches += 3;
        if (A.finest) {
          launch_wall_force(L, ph, A.fw + 2 * sgn * A.ni, A.fw + (2 * sgn + 1) * A.ni, st);
          ++launches;
        }
      }
      launch_pdl(k_adj_extract, nb, 128, 0, st, n, A.nbr, A.col, k, m, A.Fp, A.Fm, A.ub, h_rel, A.J);
      launch_pdl(k_adj_extract, nb, 128, 0, st, n, A.nbr, A.col, k, m, (const double*)A.Fvp, (const double*)A.Fvm,
                 (const double*)A.ub, h_rel, A.Jv);
      launches += 2;
      if (A.finest) {
        launch_pdl(k_adj_extract_obj, nbf, 128, 0, st, A.ni, n, A.col, k, m, A.fw, A.ub, h_rel, sa, ca, A.g);
        ++launches;
      }
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
  for (int i = 0; i < 5; ++i) {
    A.stage_c[i] = i < sc.nstages ? sc.alpha[i] / sc.eta : 0.0;
    A.stage_b[i] = i < sc.nstages ? sc.beta[i] : 1.0;
  }
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

namespace {

// ---------------------------------------------------------------- transposed smoother and cycle
// The primal's smoothing step, linearised at a converged state, is a linear solver for J x = b
// (x from 0; c_i = alpha_i / eta, P^-1 t = W^-1 (eta dt* t), J = J^c + J^v with J^v the
// Jacobian of the dissipative part F^v, whose stage value is blended with beta_i as in the
// primal's stage residual):
//   f_i = beta_i J^v x_(i-1) + (1 - beta_i) f_(i-1),   x_i = c_i P^-1 (b - J^c x_(i-1) - f_i).
// Its transpose is this recurrence run backwards (reverse mode), with P^-T, J^T and J^v^T.
// The linearised FAS cycle on level l (nu1 smoothing steps, residual restriction R, gamma
// coarse cycles on J_(l-1) from zero, bilinear prolongation P of the correction) is
//   x1 = S b,  x = x1 + P A_(l-1) R (b - J x1),   A = C_(l-1) (gamma 1) or 2C - C J C (gamma 2),
// and its transpose C^T v = R^T r + S^T (v - J^T R^T r) with r = A^T P^T v.

__global__ void k_lc(int m, double a0, const double* x0, double a1, const double* x1, double a2, const double* x2,
                     double a3, const double* x3, double* out) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  double s = a0 * x0[t];
  if (x1) s += a1 * x1[t];
  if (x2) s += a2 * x2[t];
  if (x3) s += a3 * x3[t];
  out[t] = s;
}

// out = eta dt* t per cell (eta dt* = coef vol)
__global__ void k_scale_dts(int n, const double* coef, const double* vol, const double* t, double* out) {
  pdl_entry();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const double s = coef[d] * vol[d];
  for (int k = 0; k < 4; ++k) out[(size_t)k * n + d] = s * t[(size_t)k * n + d];
}

// out[o] = sum over entries e of row o: w[e] in[idx[e]], all four components
__global__ void k_csr_apply(int nout, int nin, const int* ptr, const int* idx, const double* w, const double* in,
                            double* out) {
  pdl_entry();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = ptr[o]; e < ptr[o + 1]; ++e) {
    const int c = idx[e];
    for (int k = 0; k < 4; ++k) s[k] += w[e] * in[(size_t)k * nin + c];
  }
  for (int k = 0; k < 4; ++k) out[(size_t)k * nout + o] = s[k];
}

// residual restriction of the FAS cycle: volume-weighted average of the four children
__global__ void k_restrict_res(LevelDev F, LevelDev C, const double* in, double* out) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C.n) return;
  const int I = t % C.ni, J = t / C.ni;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < 4; ++q) {
    const int fc = (2 * J + (q >> 1)) * F.ni + 2 * I + (q & 1);
    const double w = F.vol[fc];
    for (int k = 0; k < 4; ++k) s[k] += w * in[(size_t)k * F.n + fc];
  }
  for (int k = 0; k < 4; ++k) out[(size_t)k * C.n + t] = s[k] / C.vol[t];
}

// its transpose: child c of coarse cell t receives vol_c / vol_t of it
__global__ void k_restrict_res_T(LevelDev F, LevelDev C, const double* in, double* out) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= F.n) return;
  const int t = (c / F.ni / 2) * C.ni + (c % F.ni) / 2;
  const double w = F.vol[c] / C.vol[t];
  for (int k = 0; k < 4; ++k) out[(size_t)k * F.n + c] = w * in[(size_t)k * C.n + t];
}

}  // namespace

struct TransferMap {
  int* fptr = nullptr;  // fine-major: the coarse cells (and weights) each fine cell reads
  int* fidx = nullptr;
  double* fw = nullptr;
  int* cptr = nullptr;  // coarse-major: the same entries grouped by coarse cell (the transpose)
  int* cidx = nullptr;
  double* cw = nullptr;
};

struct AdjointMG {
  int L = 0, gamma = 1, nu1 = 1;
  std::vector<AdjointDev> lv;          // coarse levels 0 .. L-1 (the finest is the outer AdjointDev)
  std::vector<LevelDev> lev;           // the context's levels (volumes and sizes)
  std::vector<TransferMap> pm;         // pm[l]: prolongation from level l-1 to level l
  std::vector<std::vector<double*>> wk;  // per level: 8 work vectors of 4 n_l
};

namespace {

AdjointDev& level_of(AdjointDev& A, int l) { return l == A.mg->L ? A : A.mg->lv[l]; }

// The prolongation of k_prolong as a matrix: fine cell (i, j) takes 9/16, 3/16, 3/16, 1/16 of
// the coarse cells (I, J), (I2, J), (I, J2), (I2, J2), I = i/2, I2 = I -+ 1 by the parity of i
// (likewise J), a coarse index outside the grid standing for the clamped cell, or below the
// wake cut for the mirror cell of row 0.
int build_prolong_map(const LevelDev& F, const LevelDev& C, TransferMap& T, std::vector<void*>& allocs,
                      cudaStream_t st) {
  const int nf = F.n, nc = C.n;
  auto target = [&](int I, int J) {
    int Ic = std::min(std::max(I, 0), C.ni - 1);
    int Jc;
    if (J < 0) {
      if (C.nw > 0 && (Ic < C.nw || Ic >= C.ni - C.nw)) Ic = C.ni - 1 - Ic;
      Jc = 0;
    } else {
      Jc = std::min(J, C.nj - 1);
    }
    return Jc * C.ni + Ic;
  };
  std::vector<int> fptr(nf + 1, 0), fidx;
  std::vector<double> fw;
  for (int c = 0; c < nf; ++c) {
    const int i = c % F.ni, j = c / F.ni, I = i / 2, J = j / 2;
    const int I2 = (i % 2 == 0) ? I - 1 : I + 1, J2 = (j % 2 == 0) ? J - 1 : J + 1;
    const int tg[4] = {target(I, J), target(I2, J), target(I, J2), target(I2, J2)};
    const double wt[4] = {9.0 / 16.0, 3.0 / 16.0, 3.0 / 16.0, 1.0 / 16.0};
    const int start = (int)fidx.size();
    for (int q = 0; q < 4; ++q) {
      bool merged = false;
      for (int e = start; e < (int)fidx.size(); ++e)
        if (fidx[e] == tg[q]) {
          fw[e] += wt[q];
          merged = true;
        }
      if (!merged) {
        fidx.push_back(tg[q]);
        fw.push_back(wt[q]);
      }
    }
    fptr[c + 1] = (int)fidx.size();
  }
  const int ne = (int)fidx.size();
  std::vector<int> cptr(nc + 1, 0), cidx(ne);
  std::vector<double> cw(ne);
  for (int e = 0; e < ne; ++e) ++cptr[fidx[e] + 1];
  for (int t = 0; t < nc; ++t) cptr[t + 1] += cptr[t];
  std::vector<int> fill(cptr.begin(), cptr.end() - 1);
  for (int c = 0; c < nf; ++c)  // fine cells in increasing order: a fixed summation order
    for (int e = fptr[c]; e < fptr[c + 1]; ++e) {
      const int k = fill[fidx[e]]++;
      cidx[k] = c;
      cw[k] = fw[e];
    }
  int r;
  if ((r = adj_alloc(allocs, &T.fptr, fptr.size())) || (r = adj_alloc(allocs, &T.fidx, (size_t)ne)) ||
      (r = adj_alloc(allocs, &T.fw, (size_t)ne)) || (r = adj_alloc(allocs, &T.cptr, cptr.size())) ||
      (r = adj_alloc(allocs, &T.cidx, (size_t)ne)) || (r = adj_alloc(allocs, &T.cw, (size_t)ne)))
    return r;
  cudaMemcpyAsync(T.fptr, fptr.data(), fptr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(T.fidx, fidx.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(T.fw, fw.data(), ne * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(T.cptr, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(T.cidx, cidx.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(T.cw, cw.data(), ne * sizeof(double), cudaMemcpyHostToDevice, st);
  return cudaStreamSynchronize(st) == cudaSuccess ? FASW_OK : FASW_ERR_CUDA;  // host vectors die here
}

void lc(int m, double a0, const double* x0, double a1, const double* x1, double a2, const double* x2, double a3,
        const double* x3, double* out, cudaStream_t st) {
  launch_pdl(k_lc, (m + 255) / 256, 256, 0, st, m, a0, x0, a1, x1, a2, x2, a3, x3, out);
}

void jac(const AdjointDev& A, const double* blocks, const double* v, double* out, int transpose, cudaStream_t st) {
  const int nb = (A.n + 127) / 128;
  if (transpose)
    launch_pdl(k_jac_tmv, nb, 128, 0, st, A.n, A.rev_ptr, A.rev, blocks, v, out);
  else
    launch_pdl(k_jac_mv, nb, 128, 0, st, A.n, A.nbr, blocks, v, out);
}

// x = c P^-1 t (forward: the level's own FP64 blocks; scratch s)
void precond_fwd(const AdjointDev& A, double c, const double* t, double* s, double* x, cudaStream_t st) {
  launch_pdl(k_scale_dts, (A.n + 127) / 128, 128, 0, st, A.n, (const double*)A.Lp.coef, (const double*)A.Lp.vol, t,
             s);
  LevelDev T = A.Lp;
  T.yz64 = x;
  launch_sweep(T, 0, SWEEP_STRIPS, 0, 1, 0.0, s, A.prog, A.err, A.spin_limit, st);
  const int m = 4 * A.n;
  lc(m, c, x, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, x, st);
}

// x = S b: one linearised smoothing step from zero.  Work: A.mgw vectors 0-3.
void smooth_fwd(AdjointDev& A, const double* b, double* x, cudaStream_t st) {
  const int m = 4 * A.n;
  double* f = A.mgw;
  double* t = A.mgw + (size_t)m;
  double* jv = A.mgw + 2 * (size_t)m;
  double* jx = A.mgw + 3 * (size_t)m;
  for (int i = 0; i < A.nstages; ++i) {
    const double be = A.stage_b[i], c = A.stage_c[i];
    if (i == 0) {  // x_0 = 0: f_1 = 0, t = b
      precond_fwd(A, c, b, t, x, st);
      continue;
    }
    jac(A, A.Jv, x, jv, 0, st);
    if (i == 1)
      lc(m, be, jv, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, f, st);
    else
      lc(m, be, jv, 1.0 - be, f, 0.0, nullptr, 0.0, nullptr, f, st);
    jac(A, A.J, x, jx, 0, st);
    lc(m, 1.0, b, -1.0, jx, 1.0, jv, -1.0, f, t, st);  // b - J^c x - f
    precond_fwd(A, c, t, jx, x, st);
  }
}

// out = S^T v (reverse of smooth_fwd).  Work: A.mgw vectors 0-4, A.mgy.
void smooth_T(AdjointDev& A, const double* v, double* out, cudaStream_t st) {
  const int m = 4 * A.n;
  double* xb = A.mgw;
  double* fb = A.mgw + (size_t)m;
  double* w = A.mgw + 2 * (size_t)m;
  double* s = A.mgw + 3 * (size_t)m;
  double* tmp = A.mgw + 4 * (size_t)m;
  cudaMemcpyAsync(xb, v, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int i = A.nstages - 1; i >= 0; --i) {
    const double be = A.stage_b[i], c = A.stage_c[i];
    precond(A, xb, A.mgy, w, st);
    lc(m, c, w, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, w, st);  // w = c P^-T xbar_i
    if (i == A.nstages - 1) {
      cudaMemcpyAsync(out, w, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
      lc(m, -1.0, w, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, fb, st);  // fbar_s = -w
    } else {
      lc(m, 1.0, out, 1.0, w, 0.0, nullptr, 0.0, nullptr, out, st);
      lc(m, 1.0, fb, -1.0, w, 0.0, nullptr, 0.0, nullptr, fb, st);
    }
    if (i == 0) break;  // x_0 = 0 is no input
    // xbar_(i-1) = -J^T w + J^v^T (w + beta_i fbar_i);  fbar_(i-1) = (1 - beta_i) fbar_i
    lc(m, 1.0, w, be, fb, 0.0, nullptr, 0.0, nullptr, s, st);
    jac(A, A.Jv, s, tmp, 1, st);
    jac(A, A.J, w, xb, 1, st);
    lc(m, -1.0, xb, 1.0, tmp, 0.0, nullptr, 0.0, nullptr, xb, st);
    lc(m, 1.0 - be, fb, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, fb, st);
  }
}

// `steps` smoothing steps as a solver of J x = b from zero (transpose: of J^T), x_k = x_(k-1) +
// S (b - J x_(k-1)); out = sum_k S^T y_k with y_0 = v, y_(k+1) = y_k - J^T S^T y_k.
// Work: A.mgw vectors 5-7 (plus those of the single step).
void smooth_steps(AdjointDev& A, int steps, int transpose, const double* v, double* out, cudaStream_t st) {
  const int m = 4 * A.n;
  double* y = A.mgw + 5 * (size_t)m;
  double* mv = A.mgw + 6 * (size_t)m;
  double* jt = A.mgw + 7 * (size_t)m;
  if (steps <= 1) {
    if (transpose)
      smooth_T(A, v, out, st);
    else
      smooth_fwd(A, v, out, st);
    return;
  }
  cudaMemcpyAsync(y, v, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(out, 0, m * sizeof(double), st);
  for (int k = 0; k < steps; ++k) {
    if (transpose) {
      smooth_T(A, y, mv, st);
      lc(m, 1.0, out, 1.0, mv, 0.0, nullptr, 0.0, nullptr, out, st);
      if (k + 1 < steps) {
        jac(A, A.J, mv, jt, 1, st);
        lc(m, 1.0, y, -1.0, jt, 0.0, nullptr, 0.0, nullptr, y, st);
      }
    } else {  // y = b - J x, x += S y
      if (k > 0) {
        jac(A, A.J, out, jt, 0, st);
        lc(m, 1.0, v, -1.0, jt, 0.0, nullptr, 0.0, nullptr, y, st);
      }
      smooth_fwd(A, y, mv, st);
      lc(m, 1.0, out, 1.0, mv, 0.0, nullptr, 0.0, nullptr, out, st);
    }
  }
}

// out = C_l v (transpose = 0) or C_l^T v, recursively over the coarse levels.
void mg_cycle(AdjointDev& A, int l, int transpose, const double* v, double* out, cudaStream_t st) {
  AdjointMG& G = *A.mg;
  AdjointDev& Al = level_of(A, l);
  if (l == 0) {
    smooth_steps(Al, G.nu1, transpose, v, out, st);
    return;
  }
  AdjointDev& Ac = level_of(A, l - 1);
  const LevelDev &F = G.lev[l], &Cl = G.lev[l - 1];
  const int mf = 4 * F.n, mc = 4 * Cl.n;
  double** wc = G.wk[l - 1].data();
  double** wf = G.wk[l].data();
  double *xH = wc[0], *t = wc[1], *u = wc[2], *rH = wc[3], *jt = wc[4];
  double *rb = wf[5], *x1 = wf[6], *sm = wf[7];
  const TransferMap& T = G.pm[l];
  if (transpose) {
    launch_pdl(k_csr_apply, (Cl.n + 127) / 128, 128, 0, st, Cl.n, F.n, (const int*)T.cptr, (const int*)T.cidx,
               (const double*)T.cw, v, xH);  // P^T v
    if (G.gamma == 1) {
      mg_cycle(A, l - 1, 1, xH, rH, st);
    } else {  // (2C - C J C)^T = 2C^T - C^T J^T C^T
      mg_cycle(A, l - 1, 1, xH, t, st);
      jac(Ac, Ac.J, t, jt, 1, st);
      lc(mc, 1.0, xH, -1.0, jt, 0.0, nullptr, 0.0, nullptr, u, st);
      mg_cycle(A, l - 1, 1, u, rH, st);
      lc(mc, 1.0, rH, 1.0, t, 0.0, nullptr, 0.0, nullptr, rH, st);
    }
    launch_pdl(k_restrict_res_T, (F.n + 127) / 128, 128, 0, st, F, Cl, (const double*)rH, rb);  // R^T
    jac(Al, Al.J, rb, x1, 1, st);
    lc(mf, 1.0, v, -1.0, x1, 0.0, nullptr, 0.0, nullptr, x1, st);
    smooth_steps(Al, G.nu1, 1, x1, sm, st);
    lc(mf, 1.0, rb, 1.0, sm, 0.0, nullptr, 0.0, nullptr, out, st);
  } else {
    smooth_steps(Al, G.nu1, 0, v, x1, st);
    jac(Al, Al.J, x1, rb, 0, st);
    lc(mf, 1.0, v, -1.0, rb, 0.0, nullptr, 0.0, nullptr, rb, st);  // b - J x1
    launch_pdl(k_restrict_res, (Cl.n + 127) / 128, 128, 0, st, F, Cl, (const double*)rb, rH);
    if (G.gamma == 1) {
      mg_cycle(A, l - 1, 0, rH, xH, st);
    } else {
      mg_cycle(A, l - 1, 0, rH, t, st);
      jac(Ac, Ac.J, t, jt, 0, st);
      lc(mc, 1.0, rH, -1.0, jt, 0.0, nullptr, 0.0, nullptr, u, st);
      mg_cycle(A, l - 1, 0, u, xH, st);
      lc(mc, 1.0, xH, 1.0, t, 0.0, nullptr, 0.0, nullptr, xH, st);
    }
    launch_pdl(k_csr_apply, (F.n + 127) / 128, 128, 0, st, F.n, Cl.n, (const int*)T.fptr, (const int*)T.fidx,
               (const double*)T.fw, (const double*)xH, sm);  // P x_H
    lc(mf, 1.0, x1, 1.0, sm, 0.0, nullptr, 0.0, nullptr, out, st);
  }
}

}  // namespace

// ---------------------------------------------------------------- vertex gradient
namespace {

__global__ void k_vertex_lengths(int ni, int nj, const double* x, const double* y, double* len) {
  pdl_entry();
  const int V = ni + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V * (nj + 1)) return;
  const int I = v % V, J = v / V;
  double best = 1e300;
  const int nb[4][2] = {{I - 1, J}, {I + 1, J}, {I, J - 1}, {I, J + 1}};
  for (int q = 0; q < 4; ++q) {
    const int a = nb[q][0], b = nb[q][1];
    if (a < 0 || a > ni || b < 0 || b > nj) continue;
    const double dx = x[b * V + a] - x[v], dy = y[b * V + a] - y[v];
    const double d = sqrt(dx * dx + dy * dy);
    if (d > 0.0 && d < best) best = d;  // coincident wake-cut vertices have no length between them
  }
  len[v] = best < 1e300 ? best : 1.0;
}

__global__ void k_vertex_perturb(int nv, const int* col, int k, int dir, double h, const double* len,
                                 const double* x0, const double* y0, double* xo, double* yo) {
  pdl_entry();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double d = col[v] == k ? h * len[v] : 0.0;
  xo[v] = x0[v] + (dir == 0 ? d : 0.0);
  yo[v] = y0[v] + (dir == 1 ? d : 0.0);
}

__global__ void k_vertex_accum(int nv, int n, int ni, const int* col, int k, const int* ptr, const int* idx,
                               int which, double sa, double ca, const double* lam, const double* Fp,
                               const double* Fm, const double* fw, double h, const double* len, double* g) {
  pdl_entry();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv || col[v] != k) return;
  double dl = 0.0, dc = 0.0;
  for (int e = ptr[v]; e < ptr[v + 1]; ++e) {
    const int t = idx[e];
    if (t < n) {
      for (int q = 0; q < 4; ++q) dl += lam[(size_t)q * n + t] * (Fp[(size_t)q * n + t] - Fm[(size_t)q * n + t]);
    } else {
      const int i = t - n;
      const double dfx = fw[i] - fw[2 * ni + i], dfy = fw[ni + i] - fw[3 * ni + i];
      dc += which == 0 ? 2.0 * (-dfx * sa + dfy * ca) : 2.0 * (dfx * ca + dfy * sa);
    }
  }
  g[v] = (dc - dl) / (2.0 * h * len[v]);
}

}  // namespace

int adj_vertex_setup(AdjointDev& A, int nw, std::vector<void*>& allocs, cudaStream_t st) {
  if (A.nvcolours > 0) return FASW_OK;  // set last, on success
  const int ni = A.ni, nj = A.nj, n = A.n, V = ni + 1, nv = (ni + 1) * (nj + 1);
  auto on_cut = [&](int i) { return nw > 0 && (i < nw || i >= ni - nw); };
  std::vector<std::vector<int>> infl(nv);
  for (int J = 0; J <= nj; ++J)
    for (int I = 0; I <= ni; ++I) {
      std::vector<int>& t = infl[J * V + I];
      for (int j = std::max(0, J - 3); j <= std::min(nj - 1, J + 2); ++j)
        for (int i = std::max(0, I - 3); i <= std::min(ni - 1, I + 2); ++i) {
          t.push_back(j * ni + i);
          if (j <= 2 && on_cut(i))  // cells on the other side of the cut see this cell through ghosts
            for (int jj = 0; jj <= std::min(2, nj - 1); ++jj)
              for (int d = -2; d <= 2; ++d) {
                const int m = ni - 1 - i + d;
                if (m >= 0 && m < ni) t.push_back(jj * ni + m);
              }
        }
      if (J <= 3)
        for (int i = std::max(0, I - 3); i <= std::min(ni - 1, I + 2); ++i)
          if (!on_cut(i)) t.push_back(n + i);  // wall faces
      std::sort(t.begin(), t.end());
      t.erase(std::unique(t.begin(), t.end()), t.end());
    }
  // greedy colouring: no target reached by two vertices of one colour
  std::vector<std::vector<int>> reached_by(n + ni);
  std::vector<int> col(nv, -1);
  int ncol = 0;
  std::vector<char> used;
  for (int v = 0; v < nv; ++v) {
    used.assign(ncol + 1, 0);
    for (int t : infl[v])
      for (int u : reached_by[t]) used[col[u]] = 1;
    int c = 0;
    while (c < ncol && used[c]) ++c;
    col[v] = c;
    if (c == ncol) ++ncol;
    for (int t : infl[v]) reached_by[t].push_back(v);
  }
  std::vector<int> ptr(nv + 1, 0), idx;
  for (int v = 0; v < nv; ++v) {
    idx.insert(idx.end(), infl[v].begin(), infl[v].end());
    ptr[v + 1] = (int)idx.size();
  }
  int r;
  if ((r = adj_alloc(allocs, &A.vcol, (size_t)nv)) || (r = adj_alloc(allocs, &A.vinfl_ptr, ptr.size())) ||
      (r = adj_alloc(allocs, &A.vinfl, idx.size())) || (r = adj_alloc(allocs, &A.vx, 2 * (size_t)nv)) ||
      (r = adj_alloc(allocs, &A.vlen, (size_t)nv)))
    return r;
  cudaMemcpyAsync(A.vcol, col.data(), nv * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(A.vinfl_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(A.vinfl, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return FASW_ERR_CUDA;  // host vectors die here
  A.nvcolours = ncol;
  return FASW_OK;
}

void adj_vertex_lengths(const AdjointDev& A, const double* x0, const double* y0, cudaStream_t st) {
  const int nv = (A.ni + 1) * (A.nj + 1);
  launch_pdl(k_vertex_lengths, (nv + 127) / 128, 128, 0, st, A.ni, A.nj, x0, y0, A.vlen);
}

void adj_vertex_perturb(const AdjointDev& A, int k, int dir, double h, const double* x0, const double* y0,
                        double* xo, double* yo, cudaStream_t st) {
  const int nv = (A.ni + 1) * (A.nj + 1);
  launch_pdl(k_vertex_perturb, (nv + 127) / 128, 128, 0, st, nv, (const int*)A.vcol, k, dir, h,
             (const double*)A.vlen, x0, y0, xo, yo);
}

void adj_vertex_accumulate(const AdjointDev& A, int k, int which, double sa, double ca, const double* lam,
                           const double* Fp, const double* Fm, const double* fw, double h_rel, double* g,
                           cudaStream_t st) {
  const int nv = (A.ni + 1) * (A.nj + 1);
  launch_pdl(k_vertex_accum, (nv + 127) / 128, 128, 0, st, nv, A.n, A.ni, (const int*)A.vcol, k,
             (const int*)A.vinfl_ptr, (const int*)A.vinfl, which, sa, ca, lam, Fp, Fm, fw, h_rel,
             (const double*)A.vlen, g);
}

int adj_mg_setup(AdjointDev& A, const std::vector<LevelDev>& lev, int gamma, int nu1, std::vector<void*>& allocs,
                 cudaStream_t st) {
  const int L = (int)lev.size() - 1;
  if (A.mg && A.mg->L == L) {
    A.mg->gamma = gamma == 2 ? 2 : 1;
    return FASW_OK;
  }
  if (A.mg) return FASW_ERR_ARG;
  AdjointMG* G = new AdjointMG;
  G->L = L;
  G->gamma = gamma == 2 ? 2 : 1;
  G->nu1 = nu1 < 1 ? 1 : nu1;
  G->lev = lev;
  G->lv.resize(L);
  G->pm.resize(L + 1);
  G->wk.resize(L + 1);
  // published in A only when complete (device memory of a failed attempt stays in allocs)
  auto fail = [&](int r) {
    for (auto& C : G->lv) adj_release(C);
    delete G;
    return r;
  };
  int r;
  for (int l = 0; l < L; ++l) {
    AdjointDev& C = G->lv[l];
    C.finest = false;
    C.fp32 = A.fp32;
    C.prog = A.prog;
    C.err = A.err;
    C.spin_limit = A.spin_limit;
    if ((r = adj_setup(C, lev[l].ni, lev[l].nj, lev[l].nw, allocs, st))) return fail(r);
  }
  for (int l = 1; l <= L; ++l)
    if ((r = build_prolong_map(lev[l], lev[l - 1], G->pm[l], allocs, st))) return fail(r);
  for (int l = 0; l <= L; ++l) {
    G->wk[l].assign(8, nullptr);
    for (int k = 0; k < 8; ++k)
      if ((r = adj_alloc(allocs, &G->wk[l][k], 4 * (size_t)lev[l].n))) return fail(r);
  }
  A.mg = G;
  return FASW_OK;
}

int adj_mg_assemble(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph, int turb, double h_rel,
                    cudaStream_t st, long long& launches) {
  if (!A.mg) return FASW_ERR_ARG;
  const int L = A.mg->L;
  for (int l = L; l >= 1; --l) {
    launch_restrict(lev[l], lev[l - 1], turb, st);
    ++launches;
  }
  for (int l = L - 1; l >= 0; --l) {
    // The forcing is constant in the differences but enters their rounding; what the last
    // primal cycle left there must not make the Jacobian depend on history (the primal
    // recomputes it every cycle).
    cudaMemsetAsync(lev[l].s, 0, 4 * (size_t)lev[l].n * sizeof(double), st);
    int r = adj_assemble(A.mg->lv[l], lev[l], ph, h_rel, st, launches);
    if (r) return r;
  }
  return FASW_OK;
}

void adj_mg_build_precond(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph,
                          const SchemeParams& sc, double cfl, cudaStream_t st, long long& launches) {
  if (!A.mg) return;
  for (int l = 0; l < A.mg->L; ++l) adj_build_precond(A.mg->lv[l], lev[l], ph, sc, cfl, st, launches);
}

void adj_mg_apply(AdjointDev& A, int transpose, const double* r, double* z, cudaStream_t st) {
  if (A.mg)
    mg_cycle(A, A.mg->L, transpose, r, z, st);
  else
    smooth_steps(A, 1, transpose, r, z, st);
}

void adj_smoother_apply(AdjointDev& A, int steps, int transpose, const double* r, double* z, cudaStream_t st) {
  smooth_steps(A, steps, transpose, r, z, st);
}

void adj_release(AdjointDev& A) {
  if (A.h_parts) cudaFreeHost(A.h_parts);
  A.h_parts = nullptr;
  if (A.mg) {
    for (auto& C : A.mg->lv) adj_release(C);
    delete A.mg;
    A.mg = nullptr;
  }
}

int adj_solve(AdjointDev& A, const std::vector<LevelDev>& lev, const PhysParams& ph, const SchemeParams& sc,
              double cfl, const double* g, double* lam, double tol, int max_iters, int restart,
              std::vector<void*>& allocs, cudaStream_t st, int* iters, double* relres, long long& launches) {
  adj_build_precond(A, lev.back(), ph, sc, cfl, st, launches);
  const bool cycle = (A.precond_kind == ADJ_FAS_CYCLE_T || A.precond_kind == ADJ_FAS_VCYCLE_T) && A.mg;
  if (cycle) adj_mg_build_precond(A, lev, ph, sc, cfl, st, launches);
  const int m = 4 * A.n;
  if (restart < 1 || restart > MAXV - 5) return FASW_ERR_ARG;
  if (A.restart < restart) {
    int r = adj_alloc(allocs, &A.kry, (size_t)(2 * restart + 7) * m);
    if (r) return r;
    A.restart = restart;
  }
  const size_t ld = m;
  double* V = A.kry;                                  // restart + 1 vectors
  double* Z = A.kry + (size_t)(A.restart + 1) * ld;   // restart preconditioned vectors
  double* w = Z + (size_t)A.restart * ld;             // work
  double* res = w + ld;
  double* gin = res + ld;                             // input and output of the captured cycle
  double* gout = gin + ld;
  // The transposed cycle is the same launch sequence every iteration: captured once into a CUDA
  // graph that reads gin and writes gout (not on the legacy default stream, where capture is not
  // possible; an eager cycle first, so that one-time kernel attributes are set outside capture).
  cudaGraphExec_t gexec = nullptr;
  if (cycle && st != nullptr) {
    cudaMemsetAsync(gin, 0, ld * sizeof(double), st);
    mg_cycle(A, A.mg->L, 1, gin, gout, st);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      mg_cycle(A, A.mg->L, 1, gin, gout, st);
      cudaGraph_t graph = nullptr;
      if (cudaStreamEndCapture(st, &graph) == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) gexec = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();  // a failed capture leaves the eager path
  }
  struct GraphGuard {
    cudaGraphExec_t& g;
    ~GraphGuard() {
      if (g) cudaGraphExecDestroy(g);
    }
  } guard{gexec};
  auto apply_m = [&](const double* rr, double* zz) {  // zz = M^-1 rr
    if (gexec) {
      cudaMemcpyAsync(gin, rr, ld * sizeof(double), cudaMemcpyDeviceToDevice, st);
      cudaGraphLaunch(gexec, st);
      cudaMemcpyAsync(zz, gout, ld * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else if (cycle) {
      mg_cycle(A, A.mg->L, 1, rr, zz, st);
    } else if (A.precond_kind != ADJ_STAGE_LOOP) {
      smooth_steps(A, A.smooth_steps, 1, rr, zz, st);
    } else {
      steps_apply(A, A.smooth_steps, rr, zz, st);
    }
  };
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
