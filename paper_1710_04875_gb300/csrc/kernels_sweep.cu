// Block SGS sweeps of the preconditioner (eq. sgs-precon, section 4.4 of arXiv 1710.04875)
// in the form used on the GPU.
//
// Once per smoothing step (W frozen, reading G19) k_sgs_prep turns the blocks of every cell c
// into transfer blocks, so that the recurrence of each sweep has the shortest possible chain
// of dependent operations:
//   forward  (D+L) y = r:   y_c = D_c^-1 r_c + G_W y_W + G_S y_S,
//   backward (D+U) z = D y: z_c = y_c + H_E z_E + H_N z_N (+ G_S z_mirror on the lower wake),
// with G_W = c D^-1 A+_w, G_S = c D^-1 B+_s, H_E = -c D^-1 A-_e, H_N = -c D^-1 B-_n (the
// wake-cut coupling uses B+ of the cell's south face in both sweeps).  The lower/upper
// neighbour sets are those of the lexicographic ordering, so the result is the paper's
// Gauss-Seidel sweep; it is evaluated on the i+j hyperplanes.
//
// Two sweep kernels:
//  * k_sweep_cta: one CTA walks all hyperplanes of a level, 4 lanes per cell (one per row
//    of the 4x4 blocks), the previous hyperplane held in shared memory.  Used for FP32.
//  * k_sweep_strips: FP64.  On GB300 a dependent FP64 FMA costs ~64 clock cycles and FP64
//    issue is per warp instruction, so one SM cannot keep up with a wide hyperplane.  Rows
//    are split into strips of H, one CTA each, pipelined along i: strip b may process its
//    local anti-diagonal s once strip b-1 has finished s + H (forward; mirrored for the
//    backward sweep).  16 lanes per cell (row q, term t) keep the FP64 chain to one FMA
//    pair plus a two-level shuffle reduction.  Progress is published in global memory
//    every CHUNK steps (fence + flag); the consumer copies the boundary row of a whole
//    chunk at once.  Every wait is bounded; on timeout the kernel raises an error flag and
//    all strips return.
#include <atomic>
#include "fasw_internal.cuh"
#include "fasw_sweep.cuh"

namespace fasw {

namespace {

__device__ __forceinline__ bool on_cut(const LevelDev& L, int i) { return L.nw > 0 && (i < L.nw || i >= L.ni - L.nw); }

// Transfer blocks, entry-major: tb[(blk*16 + e) * n + c], blk 0 = D^-1, 1 = G_W, 2 = G_S,
// 3 = H_E, 4 = H_N.  Blocks of absent neighbours are zero.  MODE 1 (HP, FP32 only): blocks 1-4
// go to the hyperplane-major arrays of k_sweep_hp instead: entry h = (i + j) * nj + j holds
// hpF[32h..] = G_W, G_S and hpB[32h..] = H_E, H_N (row-major 4x4 each); D^-1 stays in tb.
// MODE 2 (WS): tb as MODE 0, and blocks 1-4 also in FP32 in the skewed layout of the warp-strip
// sweep (kernels_sweep_ws.cu): forward rows G_W, G_S at strip j / 32, step i + j % 32, lane j % 32
// (G_S zero on row 0 except the upper wake, whose mirror precedes it), backward rows H_E, H_N at
// step Mp - 1 - i - j % 32; the lower wake's G_S (the backward coupling to its mirror) to wsCut.
template <typename T, int MODE>
__global__ void k_sgs_prep(LevelDev L, const T* blk, const T* dlu, T* tb) {
  constexpr bool HP = MODE == 1;
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, nj = L.nj, n = L.n, i = c % ni, j = c / ni;
  T A[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) A[e] = dlu[e * n + c];
  // D^-1 column by column from the LU factors (unit lower, reciprocal pivots on the diagonal)
  T Di[16];
#pragma unroll
  for (int col = 0; col < 4; ++col) {
    T b[4] = {T(0), T(0), T(0), T(0)};
    b[col] = T(1);
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
#pragma unroll
    for (int r = 0; r < 4; ++r) Di[4 * r + col] = b[r];
  }
  const T cf = T(L.coef[c]);
  const T* Axp = blk;
  const T* Axm = blk + 16 * L.nfx;
  const T* Aep = blk + 32 * L.nfx;
  const T* Aem = blk + 32 * L.nfx + 16 * L.nfe;
  const int fw = j * (ni + 1) + i, fe = fw + 1, fs = j * ni + i, fn = fs + ni;
  const bool hasW = i > 0, hasE = i < ni - 1, hasN = j < nj - 1;
  const bool hasS = j > 0 || on_cut(L, i);
#pragma unroll
  for (int e = 0; e < 16; ++e) tb[e * n + c] = Di[e];
  const size_t h = (size_t)(i + j) * nj + j;
  // MODE 2: this cell's forward / backward rows in the warp-strip layout
  const int jl = j % WS_ROWS, Mp = ws_steps(ni, nj);
  const bool cut = on_cut(L, i);
  float4* wf = reinterpret_cast<float4*>(L.wsF) + ((size_t)(j / WS_ROWS) * Mp + (i + jl)) * WS_F4_STEP + jl;
  float4* wb = reinterpret_cast<float4*>(L.wsB) + ((size_t)(j / WS_ROWS) * Mp + (Mp - 1 - i - jl)) * WS_F4_STEP + jl;
  const bool gs_fwd = j > 0 || (cut && ni - 1 - i < i);
  const bool cut_lower = j == 0 && cut && ni - 1 - i > i;
  // product helper: out = s * Di * B (B entry-major with stride sb at face f)
  auto prod = [&](int slot, const T* B, int sb, int f, T s, bool present) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T row[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        T acc = T(0);
        if (present) {
#pragma unroll
          for (int k = 0; k < 4; ++k) acc += Di[4 * r + k] * B[(4 * k + cc) * sb + f];
          acc *= s;
        }
        row[cc] = acc;
      }
      if constexpr (HP) {
        float* dst = (slot <= 2 ? L.hpF : L.hpB) + 32 * h + ((slot - 1) & 1) * 16 + 4 * r;
        *reinterpret_cast<float4*>(dst) = make_float4(row[0], row[1], row[2], row[3]);
      } else {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) tb[(slot * 16 + 4 * r + cc) * n + c] = row[cc];
      }
      if constexpr (MODE == 2) {
        const float4 f = make_float4(float(row[0]), float(row[1]), float(row[2]), float(row[3]));
        if (slot == 1) wf[r * WS_ROWS] = f;
        if (slot == 2) {
          wf[(4 + r) * WS_ROWS] = gs_fwd ? f : make_float4(0.f, 0.f, 0.f, 0.f);
          if (cut_lower) *reinterpret_cast<float4*>(L.wsCut + 16 * i + 4 * r) = f;
        }
        if (slot == 3) wb[r * WS_ROWS] = f;
        if (slot == 4) wb[(4 + r) * WS_ROWS] = f;
      }
    }
  };
  prod(1, Axp, L.nfx, fw, cf, hasW);
  prod(2, Aep, L.nfe, fs, cf, hasS);
  prod(3, Axm, L.nfx, fe, -cf, hasE);
  prod(4, Aem, L.nfe, fn, -cf, hasN);
}

template <typename T>
__device__ __forceinline__ void stage_update(const LevelDev& L, int c, int i, int j, int q, T z, int aw, double alpha) {
  const double sc = aw ? alpha : alpha * L.dts[c];
  L.u[q * L.Gn + (j + 2) * L.P + (i + 2)] = L.u0[q * L.n + c] - sc * double(z);
}

// ---------------------------------------------------------------- one CTA, 4 lanes per cell
// The data of each lane's cell on hyperplane k+2 is loaded while hyperplane k is computed
// (three register sets, loop unrolled by three), so global-load latency stays off the
// wavefront's critical path.
template <typename T>
struct CtaPre {
  T a[4], b[4], d[4], r[4];  // forward: G_W row, G_S row, D^-1 row, rhs;  backward: H_E, H_N, G_S, (y in r[0])
  T m[4];                    // wake-cut mirror value
};

template <typename T>
__global__ void __launch_bounds__(512) k_sweep_cta(LevelDev L, const T* tb, T* yz, const double* rhs, int do_update, int aw, double alpha) {
  pdl_entry();
  extern __shared__ unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);  // 2 x ni x 4
  const int ni = L.ni, nj = L.nj, n = L.n;
  const int q = threadIdx.x & 3;
  const int slot = threadIdx.x >> 2;
  const int K = ni + nj - 1;
  auto cell_of = [&](int k, int& i, int& j) -> bool {
    if (k < 0 || k >= K) return false;
    i = max(0, k - nj + 1) + slot;
    j = k - i;
    return i <= min(k, ni - 1);
  };
  auto fload = [&](int k, CtaPre<T>& P) {
    int i, j;
    if (!cell_of(k, i, j)) return;
    const int c = j * ni + i;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      P.d[m] = tb[(4 * q + m) * n + c];
      P.a[m] = tb[(16 + 4 * q + m) * n + c];
      P.b[m] = tb[(32 + 4 * q + m) * n + c];
      P.r[m] = T(rhs[m * n + c]);
      P.m[m] = T(0);
    }
    if (j == 0 && on_cut(L, i) && ni - 1 - i < i) {
#pragma unroll
      for (int m = 0; m < 4; ++m) P.m[m] = yz[m * n + (ni - 1 - i)];
    }
  };
  auto fstep = [&](int k, const CtaPre<T>& P) {
    if (k >= K) return;
    T* prev = buf + ((k + 1) & 1) * ni * 4;
    T* cur = buf + (k & 1) * ni * 4;
    int i, j;
    if (cell_of(k, i, j)) {
      const int c = j * ni + i;
      T a = T(0), b = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) a += P.d[m] * P.r[m];
      if (i > 0) {
#pragma unroll
        for (int m = 0; m < 4; ++m) a += P.a[m] * prev[(i - 1) * 4 + m];
      }
      if (j > 0) {
#pragma unroll
        for (int m = 0; m < 4; ++m) b += P.b[m] * prev[i * 4 + m];
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) b += P.b[m] * P.m[m];
      }
      const T y = a + b;
      cur[i * 4 + q] = y;
      yz[q * n + c] = y;
    }
    __syncthreads();
  };
  CtaPre<T> A, B, C;
  fload(0, A);
  fload(1, B);
  for (int k = 0; k < K; k += 3) {
    fload(k + 2, C);
    fstep(k, A);
    fload(k + 3, A);
    fstep(k + 1, B);
    fload(k + 4, B);
    fstep(k + 2, C);
  }
  // backward (z overwrites y); hyperplanes in descending order, index kk = K-1-k
  auto bload = [&](int kk, CtaPre<T>& P) {
    int i, j;
    if (!cell_of(K - 1 - kk, i, j)) return;
    const int c = j * ni + i;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      P.a[m] = tb[(48 + 4 * q + m) * n + c];
      P.b[m] = tb[(64 + 4 * q + m) * n + c];
      P.d[m] = tb[(32 + 4 * q + m) * n + c];
      P.m[m] = T(0);
    }
    P.r[0] = yz[q * n + c];
    if (j == 0 && on_cut(L, i) && ni - 1 - i > i) {
#pragma unroll
      for (int m = 0; m < 4; ++m) P.m[m] = yz[m * n + (ni - 1 - i)];
    }
  };
  auto bstep = [&](int kk, const CtaPre<T>& P) {
    if (kk >= K) return;
    const int k = K - 1 - kk;
    T* prev = buf + ((k + 1) & 1) * ni * 4;  // hyperplane k+1
    T* cur = buf + (k & 1) * ni * 4;
    int i, j;
    if (cell_of(k, i, j)) {
      const int c = j * ni + i;
      T a = P.r[0], b = T(0);
      if (i < ni - 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) a += P.a[m] * prev[(i + 1) * 4 + m];
      }
      if (j < nj - 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) b += P.b[m] * prev[i * 4 + m];
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) b += P.d[m] * P.m[m];
      const T z = a + b;
      cur[i * 4 + q] = z;
      yz[q * n + c] = z;
      if (do_update) stage_update(L, c, i, j, q, z, aw, alpha);
    }
    __syncthreads();
  };
  CtaPre<T> D0, D1, D2;
  bload(0, D0);
  bload(1, D1);
  for (int kk = 0; kk < K; kk += 3) {
    bload(kk + 2, D2);
    bstep(kk, D0);
    bload(kk + 3, D0);
    bstep(kk + 1, D1);
    bload(kk + 4, D1);
    bstep(kk + 2, D2);
  }
}

// ---------------------------------------------------------------- strips, 16 lanes per cell
constexpr int CHUNK = 8;      // steps between progress publications
constexpr int RING = 4 * CHUNK;

__device__ __forceinline__ long long ld_acquire(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(long long* p, long long v) {
  asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T quad_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// Per step, a thread of row jl handles cell (i = s - jl, j) (forward) or (i = M-1-s-jl, j)
// (backward), so the transfer-block entries it needs over CHUNK consecutive steps are CHUNK
// consecutive words of one array: they are loaded one chunk ahead into registers, and D^-1 r
// is formed for the whole chunk before its steps start.  What remains on each step's path is
// one FMA pair, a two-level shuffle sum and one barrier.
template <typename T, int SH>  // SH rows per strip
__global__ void __launch_bounds__(16 * SH) k_sweep_strips(LevelDev L, const T* tb, T* yz, const double* rhs,
                                                           long long* prog, int* err, long long limit,
                                                           int do_update, int aw, double alpha) {
  pdl_entry();
  __shared__ T buf[2][SH][4];
  __shared__ T ring[RING][4];
  __shared__ int abort_flag;
  const int ni = L.ni, nj = L.nj, n = L.n;
  const int b = blockIdx.x, nb = gridDim.x;
  const int j0 = b * SH;
  const int jl = threadIdx.x >> 4, q = (threadIdx.x >> 2) & 3, t = threadIdx.x & 3;
  const int j = j0 + jl;
  const bool rowok = j < nj;
  const int M = ni + SH - 1;  // local steps per sweep
  long long* pf = prog;       // forward progress per strip (flags cleared by the host before launch)
  long long* pb = prog + nb;  // backward progress per strip
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  const size_t row = (size_t)j * ni;
  const T* tD = tb + (size_t)(4 * q + t) * n + row;
  const T* tW = tb + (size_t)(16 + 4 * q + t) * n + row;
  const T* tS = tb + (size_t)(32 + 4 * q + t) * n + row;
  const T* tE = tb + (size_t)(48 + 4 * q + t) * n + row;
  const T* tN = tb + (size_t)(64 + 4 * q + t) * n + row;
  const double* rr = rhs + (size_t)t * n + row;

  // bounded wait of thread 0 for a neighbour strip's progress; false on timeout
  auto wait_for = [&](const long long* flag, long long need) -> bool {
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (ld_acquire(flag) < need) {
        if (*((volatile int*)err) != 0 || ++spins > limit) {
          atomicExch(err, 1);
          abort_flag = 1;
          break;
        }
      }
    }
    __syncthreads();
    return abort_flag == 0;
  };

  // ---------------- forward
  {
    T cy[CHUNK], ca[CHUNK], cb[CHUNK];   // current chunk: D^-1 r term, G_W and G_S entries
    T nd[CHUNK], nr[CHUNK], na[CHUNK], nbv[CHUNK];  // next chunk, raw
    auto load_chunk = [&](int s0) {
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        const int i = s0 + k - jl;
        const bool ok = rowok && i >= 0 && i < ni;
        nd[k] = ok ? tD[i] : T(0);
        nr[k] = ok ? T(rr[i]) : T(0);
        na[k] = ok ? tW[i] : T(0);
        nbv[k] = ok ? tS[i] : T(0);
      }
    };
    load_chunk(0);
    for (int s0 = 0; s0 < M; s0 += CHUNK) {
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        cy[k] = nd[k] * nr[k];
        ca[k] = na[k];
        cb[k] = nbv[k];
      }
      if (s0 + CHUNK < M) load_chunk(s0 + CHUNK);
      // boundary row of strip b-1 for the columns of this chunk
      if (b > 0 && s0 < ni) {
        const long long need = min((long long)s0 + SH + CHUNK - 1, (long long)M);
        if (!wait_for(pf + b - 1, need)) return;
        const int hi = min(ni, s0 + CHUNK);
        for (int x = threadIdx.x; x < (hi - s0) * 4; x += blockDim.x) {
          const int col = s0 + x / 4, m = x % 4;
          ring[col % RING][m] = __ldcg(&yz[(size_t)m * n + (size_t)(j0 - 1) * ni + col]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        const int s = s0 + k;
        if (s < M) {  // uniform
          const T* prev = &buf[(s + 1) & 1][0][0];
          T* cur = &buf[s & 1][0][0];
          const int i = s - jl;
          const bool valid = rowok && i >= 0 && i < ni;
          T part = T(0);
          if (valid) {
            part = cy[k];
            if (i > 0) part += ca[k] * prev[jl * 4 + t];
            if (jl > 0) {
              part += cb[k] * prev[(jl - 1) * 4 + t];
            } else if (j > 0) {
              part += cb[k] * ring[i % RING][t];
            } else if (on_cut(L, i) && ni - 1 - i < i) {
              part += cb[k] * yz[(size_t)t * n + (ni - 1 - i)];
            }
          }
          const T y = quad_sum(part);  // all lanes take part in the shuffles
          if (valid && t == 0) {
            cur[jl * 4 + q] = y;
            yz[(size_t)q * n + row + i] = y;
          }
          __syncthreads();
        }
      }
      // publish this chunk: the writers of the row strip b+1 reads fence their stores first
      if (b < nb - 1) {
        if (jl == SH - 1 && t == 0) __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(pf + b, (long long)min(s0 + CHUNK, M));
      }
    }
  }
  // ---------------- backward: step s handles local anti-diagonal M-1-s; the top row needs
  // strip b+1's row 0
  {
    T cy[CHUNK], ce[CHUNK], cn[CHUNK];  // current chunk: own y (lane t == q), H_E and H_N entries
    T ny[CHUNK], ne[CHUNK], nn[CHUNK];
    double cu[CHUNK], nu[CHUNK];        // u^(0) of component q (writer lanes t == 0), scaled step
    double cs_[CHUNK], ns_[CHUNK];      // dt* factor of the update (ARK), 1 for AW
    const double* u0q = L.u0 + (size_t)q * n + row;
    const double* dtr = L.dts + row;
    auto load_chunk = [&](int s0) {
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        const int i = M - 1 - (s0 + k) - jl;
        const bool ok = rowok && i >= 0 && i < ni;
        ny[k] = (ok && q == t) ? yz[(size_t)q * n + row + i] : T(0);
        ne[k] = ok ? tE[i] : T(0);
        nn[k] = ok ? tN[i] : T(0);
        nu[k] = (ok && do_update && t == 0) ? u0q[i] : 0.0;
        ns_[k] = (ok && do_update && t == 0 && !aw) ? dtr[i] : 1.0;
      }
    };
    load_chunk(0);
    for (int s0 = 0; s0 < M; s0 += CHUNK) {
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        cy[k] = ny[k];
        ce[k] = ne[k];
        cn[k] = nn[k];
        cu[k] = nu[k];
        cs_[k] = ns_[k];
      }
      if (s0 + CHUNK < M) load_chunk(s0 + CHUNK);
      const int icol_hi = (M - 1 - s0) - (SH - 1);  // top-row column at the chunk's first step
      if (b < nb - 1 && icol_hi >= 0) {
        const long long need = min((long long)s0 + SH + CHUNK - 1, (long long)M);
        if (!wait_for(pb + b + 1, need)) return;
        const int hi = min(icol_hi, ni - 1);
        const int lo = max(0, icol_hi - CHUNK + 1);
        for (int x = threadIdx.x; x < (hi - lo + 1) * 4; x += blockDim.x) {
          const int col = lo + x / 4, m = x % 4;
          ring[col % RING][m] = __ldcg(&yz[(size_t)m * n + (size_t)(j0 + SH) * ni + col]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int k = 0; k < CHUNK; ++k) {
        const int s = s0 + k;
        if (s < M) {  // uniform
          const T* prev = &buf[(s + 1) & 1][0][0];
          T* cur = &buf[s & 1][0][0];
          const int i = (M - 1 - s) - jl;
          const bool valid = rowok && i >= 0 && i < ni;
          T part = T(0);
          if (valid) {
            part = cy[k];
            if (i < ni - 1) part += ce[k] * prev[jl * 4 + t];
            if (j < nj - 1) part += cn[k] * (jl < SH - 1 ? prev[(jl + 1) * 4 + t] : ring[i % RING][t]);
            if (j == 0 && on_cut(L, i) && ni - 1 - i > i)
              part += tS[i] * yz[(size_t)t * n + (ni - 1 - i)];
          }
          const T z = quad_sum(part);  // all lanes take part; the shuffle orders the y read before the z write
          if (valid && t == 0) {
            const int c = j * ni + i;
            cur[jl * 4 + q] = z;
            yz[(size_t)q * n + c] = z;
            if (do_update) L.u[(size_t)q * L.Gn + (j + 2) * L.P + (i + 2)] = cu[k] - alpha * cs_[k] * double(z);
          }
          __syncthreads();
        }
      }
      if (b > 0) {  // strip b-1 reads this strip's first row
        if (jl == 0 && t == 0) __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(pb + b, (long long)min(s0 + CHUNK, M));
      }
    }
  }
}

// ---------------------------------------------------------------- hyperplane-staged, FP32
// For the FP32 preconditioner the sweep is bound by how fast one SM can bring in the blocks
// of the next hyperplane (36 floats per cell and direction) and by the per-step barrier, not
// by arithmetic.  Cells are therefore stored hyperplane-major (entry h = (i+j)*nj + j, see
// k_sgs_prep<float, 1>), so that the data of one step of all rows are contiguous, and
// each thread (row j, block row q) copies its own 16-byte pieces with cp.async into a
// per-thread ring of shared memory STAGES steps ahead of use.  The previous hyperplane's
// vectors are exchanged through shared memory (one barrier per step); row 0 keeps its values
// for the wake-cut coupling, which in the forward sweep reads the mirror cell processed
// earlier on the same row, and in the backward sweep the mirror cell processed earlier there.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int sz = valid ? 16 : 0;  // 0: zero-fill without reading
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int sz = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w);
}
__device__ __forceinline__ void set_comp(float4& v, int q, float x) { reinterpret_cast<float*>(&v)[q] = x; }

// cy = D^-1 rhs per cell, written hyperplane-major (the forward sweep's constant term).
__global__ void k_hp_cy(LevelDev L, const float* dinv, const double* rhs) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, i = c % L.ni, j = c / L.ni;
  float r[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) r[t] = float(rhs[t * n + c]);
  float y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) a += dinv[(4 * q + t) * n + c] * r[t];
    y[q] = a;
  }
  *reinterpret_cast<float4*>(L.hpC + 4 * ((size_t)(i + j) * L.nj + j)) = make_float4(y[0], y[1], y[2], y[3]);
}

// Shared memory: ring of STAGES steps, each [2][nt] float4 block rows + [nt] floats (the
// thread's D^-1 r or y component); exchange [2][njp+1] float4; row 0 [ni] float4; lower-wake
// G_S rows [nw][4] float4.
inline size_t hp_smem_bytes(int stages, int nt, int njp, int ni, int nw) {
  return (size_t)stages * 36 * nt + 16 * (2 * (size_t)(njp + 1) + (size_t)ni + 4 * (size_t)nw);
}

// The sweep proper: y (forward) and z (backward, written over y in hpY).  No FP64 work and
// no per-cell update inside the recurrence; k_hp_finish applies the stage update afterwards.
// The step loop is unrolled by the ring depth, so ring slots and exchange buffers are fixed
// shared-memory offsets, and the global sources advance by one hyperplane per issue.
template <int STAGES>
__global__ void __launch_bounds__(1024) k_sweep_hp(LevelDev L) {
  pdl_entry();
  static_assert((STAGES & (STAGES - 1)) == 0 && STAGES >= 4, "ring depth: power of two, at least 4");
  extern __shared__ float4 sm4[];
  const int nt = blockDim.x, tid = threadIdx.x;
  const int j = tid >> 2, q = tid & 3, njp = nt >> 2;
  const int ni = L.ni, nj = L.nj, nw = L.nw;
  const int K = ni + nj - 1;
  const int stage_f4 = 2 * nt + nt / 4;  // float4 units per ring stage (nt is a multiple of 32)
  float4* ring = sm4;
  float4* xb = ring + (size_t)STAGES * stage_f4;
  float4* row0 = xb + 2 * (njp + 1);
  float4* gsm = row0 + ni;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int x = tid; x < 2 * (njp + 1); x += nt) xb[x] = zero4;

  float4* myA = ring + tid;       // block row q of the first block of this thread's cell
  float4* myB = ring + nt + tid;  // of the second block
  float* myC = reinterpret_cast<float*>(ring + 2 * nt) + tid;
  const int cstride = 4 * stage_f4;  // floats per ring stage
  float4* xj = xb + j;               // exchange entries of this row (buffer 0; buffer 1 at + njp + 1)
  const int xo = njp + 1;

  // Hyperplane k holds entry (k, j) = k * nj + j.  Padding threads (j >= nj) point at the
  // array start and only ever zero-fill.
  const bool rowok = j < nj;
  const size_t e0 = rowok ? (size_t)j : 0;
  const size_t s32 = 32 * (size_t)nj, s4 = 4 * (size_t)nj;
  auto valid_at = [&](int k) { return rowok && (unsigned)(k - j) < (unsigned)ni; };

  // ---------------- forward: y = D^-1 r + G_W y_W + G_S y_S
  {
    const float* bW = L.hpF + 32 * e0 + 4 * q;
    const float* bC = L.hpC + 4 * e0 + q;
    const float* iW = bW;
    const float* iC = bC;
    int ki = 0;
    auto issue = [&](int u) {
      const bool v = valid_at(ki);
      const float* w = v ? iW : bW;
      cp_async16(myA + u * stage_f4, w, v);
      cp_async16(myB + u * stage_f4, w + 16, v);
      cp_async4(myC + u * cstride, v ? iC : bC, v);
      cp_commit();
      ++ki;
      iW += s32;
      iC += s4;
    };
    // steps 0 .. STAGES-2 in flight; step k refills the slot step k-1 used with step
    // k + STAGES - 1, right after its own operands are read, so the issue overlaps their latency
#pragma unroll
    for (int u = 0; u < STAGES - 1; ++u) issue(u);
    __syncthreads();
    float* pY = L.hpY + 4 * e0 + q;
    const bool mirror_row = j == 0 && nw > 0;
    for (int k0 = 0; k0 < K; k0 += STAGES) {
#pragma unroll
      for (int u = 0; u < STAGES; ++u) {
        const int k = k0 + u;
        if (k < K) {  // uniform
          cp_wait<STAGES - 2>();
          const float4 ga = myA[u * stage_f4], gb = myB[u * stage_f4];
          const float cy = myC[u * cstride];
          const int pv = ((u + 1) & 1) * xo, cu = (u & 1) * xo;  // k0 is even
          const float4 yw = xj[pv];
          float4 ys = zero4;
          if (j > 0) {
            ys = xj[pv - 1];
          } else if (mirror_row && k >= ni - nw && k < ni) {  // row 0, i = k: lower-half mirror
            ys = row0[ni - 1 - k];
          }
          issue((u + STAGES - 1) & (STAGES - 1));
          const float y = cy + (dot4(ga, yw) + dot4(gb, ys));
          set_comp(xj[cu], q, y);
          if (valid_at(k)) {
            *pY = y;
            if (j == 0) set_comp(row0[k], q, y);
          }
          __syncthreads();
          pY += s4;
        }
      }
    }
    cp_wait<0>();
  }
  __threadfence_block();

  // ---------------- backward: z = y + H_E z_E + H_N z_N (+ G_S z_mirror on the lower wake)
  for (int x = tid; x < 2 * (njp + 1); x += nt) xb[x] = zero4;
  for (int x = tid; x < 4 * nw; x += nt) {
    const int i = x >> 2, r = x & 3;  // cell (i, 0) is entry h = i * nj
    gsm[x] = *reinterpret_cast<const float4*>(L.hpF + 32 * (size_t)i * nj + 16 + 4 * r);
  }
  __syncthreads();  // the forward's y (same thread) and the shared arrays are in place
  {
    const float* bE = L.hpB + 32 * e0 + 4 * q;
    const float* bY = L.hpY + 4 * e0 + q;
    const float* iE = bE + s32 * (size_t)(K - 1);
    const float* iY = bY + s4 * (size_t)(K - 1);
    int ki = K - 1;
    auto issue = [&](int u) {
      const bool v = valid_at(ki);
      const float* e = v ? iE : bE;
      cp_async16(myA + u * stage_f4, e, v);
      cp_async16(myB + u * stage_f4, e + 16, v);
      cp_async4(myC + u * cstride, v ? iY : bY, v);
      cp_commit();
      --ki;
      iE -= s32;
      iY -= s4;
    };
#pragma unroll
    for (int u = 0; u < STAGES - 1; ++u) issue(u);
    __syncthreads();
    float* pZ = L.hpY + 4 * e0 + q + s4 * (size_t)(K - 1);
    for (int kk0 = 0; kk0 < K; kk0 += STAGES) {
#pragma unroll
      for (int u = 0; u < STAGES; ++u) {
        const int kk = kk0 + u;
        if (kk < K) {  // uniform
          cp_wait<STAGES - 2>();
          const float4 he = myA[u * stage_f4], hn = myB[u * stage_f4];
          const float yv = myC[u * cstride];
          const int pv = ((u + 1) & 1) * xo, cu = (u & 1) * xo;
          const int k = K - 1 - kk;
          const float4 ze = xj[pv], zn = xj[pv + 1];
          float4 gm = zero4, zm = zero4;
          if (j == 0 && k < nw) {  // row 0, i = k: upper-half mirror
            gm = gsm[4 * k + q];
            zm = row0[ni - 1 - k];
          }
          issue((u + STAGES - 1) & (STAGES - 1));
          const float z = yv + (dot4(he, ze) + dot4(hn, zn)) + dot4(gm, zm);
          set_comp(xj[cu], q, z);
          if (valid_at(k)) {
            *pZ = z;
            if (j == 0) set_comp(row0[k], q, z);
          }
          __syncthreads();
          pZ -= s4;
        }
      }
    }
    cp_wait<0>();
  }
}

// After the sweep: the stage update u = u^(0) - alpha z (AW) or u^(0) - alpha dt* z (ARK) in
// FP64, or (no update) z to the natural-layout FP32 vector.
__global__ void k_hp_finish(LevelDev L, int do_update, int aw, double alpha) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, i = c % L.ni, j = c / L.ni;
  const float4 z = *reinterpret_cast<const float4*>(L.hpY + 4 * ((size_t)(i + j) * L.nj + j));
  const float zz[4] = {z.x, z.y, z.z, z.w};
  if (do_update) {
    const double sc = aw ? alpha : alpha * L.dts[c];
    const size_t g = (size_t)(j + 2) * L.P + (i + 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) L.u[q * (size_t)L.Gn + g] = L.u0[q * (size_t)n + c] - sc * double(zz[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) L.yz32[q * (size_t)n + c] = zz[q];
  }
}

}  // namespace

void launch_sgs_prep(const LevelDev& L, int mixed, int kind, cudaStream_t st) {
  if (is_ws(kind) && L.wsF) {
    if (mixed)
      launch_pdl(k_sgs_prep<float, 2>, (L.n + 63) / 64, 64, 0, st, L, L.blk32, L.dlu32, reinterpret_cast<float*>(L.tb));
    else
      launch_pdl(k_sgs_prep<double, 2>, (L.n + 63) / 64, 64, 0, st, L, L.blk64, L.dlu64, L.tb);
    return;
  }
  if (mixed && is_hp(kind) && L.hpF)
    launch_pdl(k_sgs_prep<float, 1>, (L.n + 63) / 64, 64, 0, st, L, L.blk32, L.dlu32, reinterpret_cast<float*>(L.tb));
  else if (mixed)
    launch_pdl(k_sgs_prep<float, 0>, (L.n + 63) / 64, 64, 0, st, L, L.blk32, L.dlu32, reinterpret_cast<float*>(L.tb));
  else
    launch_pdl(k_sgs_prep<double, 0>, (L.n + 63) / 64, 64, 0, st, L, L.blk64, L.dlu64, L.tb);
}

namespace {
// The dynamic shared-memory limit is a per-device attribute of a kernel: set it once on each
// device that launches the kernel (slot: which kernel).  Two host threads may both set it the
// first time; the call is idempotent.
constexpr int kAttrDevices = 64;
std::atomic<unsigned long long> g_attr_done[4];

template <typename Kernel>
void smem_attr_once(Kernel k, int bytes, int slot) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return;
  const unsigned long long bit = dev < kAttrDevices ? 1ull << dev : 0ull;
  if (bit && (g_attr_done[slot].load(std::memory_order_acquire) & bit)) return;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && bit)
    g_attr_done[slot].fetch_or(bit, std::memory_order_acq_rel);
}

int hp_threads(int nj) { return 4 * ((nj + 7) / 8 * 8); }
int hp_stages(int nt) { return nt <= 256 ? 8 : 4; }  // 512 and 1024 threads: ring of 4 keeps shared memory < 227 KB
constexpr size_t kHpSmemMax = 227 * 1024;
}  // namespace

size_t hp_floats(int ni, int nj) { return (size_t)(ni + nj - 1) * nj; }

bool hp_fits(int ni, int nj, int nw) {
  if (nj > 256) return false;  // one CTA of 4 nj threads
  const int nt = hp_threads(nj);
  return hp_smem_bytes(hp_stages(nt), nt, nt / 4, ni, nw) <= kHpSmemMax;
}

int launch_sweep(const LevelDev& L, int mixed, int kind, int do_update, int aw, double alpha, const double* rhs,
                 long long* prog, int* err, long long limit, cudaStream_t st, int exact_iters) {
  if (is_ws(kind) && L.wsF)
    return launch_ws_sweep(L, mixed, 1, do_update, aw, alpha, rhs, prog, err, limit, st, exact_iters,
                           kind == SWEEP_WS8 ? 8 : WS_K);
  if (is_ws(kind)) kind = mixed ? SWEEP_AUTO : SWEEP_STRIPS;
  if (is_hp(kind) && mixed && L.hpF) {
    launch_pdl(k_hp_cy, (L.n + 127) / 128, 128, 0, st, L, reinterpret_cast<const float*>(L.tb), rhs);
    const int nt = hp_threads(L.nj);
    int stages = kind == SWEEP_HP4 ? 4 : kind == SWEEP_HP8 ? 8 : hp_stages(nt);
    if (hp_smem_bytes(stages, nt, nt / 4, L.ni, L.nw) > kHpSmemMax) stages = 4;  // hp_fits checked 4 or 8
    const size_t sm = hp_smem_bytes(stages, nt, nt / 4, L.ni, L.nw);
    if (stages == 8) {
      smem_attr_once(k_sweep_hp<8>, (int)kHpSmemMax, 0);
      launch_pdl(k_sweep_hp<8>, 1, nt, sm, st, L);
    } else {
      smem_attr_once(k_sweep_hp<4>, (int)kHpSmemMax, 1);
      launch_pdl(k_sweep_hp<4>, 1, nt, sm, st, L);
    }
    launch_pdl(k_hp_finish, (L.n + 63) / 64, 64, 0, st, L, do_update, aw, alpha);
    return 3;
  }
  if (is_hp(kind)) kind = mixed ? SWEEP_CTA : SWEEP_STRIPS;
  const int cells = L.ni < L.nj ? L.ni : L.nj;  // longest hyperplane
  const bool cta_fits = 4 * cells <= 512;       // one thread slot per cell of a hyperplane
  const bool strips = kind == SWEEP_STRIPS || kind == SWEEP_STRIPS16 || kind == SWEEP_STRIPS4;
  if ((kind == SWEEP_CTA || (mixed && !strips)) && cta_fits) {
    int threads = 4 * cells;
    threads = threads < 64 ? 64 : threads;
    threads = (threads + 31) / 32 * 32;
    if (mixed) {
      const size_t sm = 2 * (size_t)L.ni * 4 * sizeof(float);
      smem_attr_once(k_sweep_cta<float>, 200 * 1024, 2);
      launch_pdl(k_sweep_cta<float>, 1, threads, sm, st, L, reinterpret_cast<const float*>(L.tb), L.yz32, rhs, do_update, aw,
                                                 alpha);
    } else {
      const size_t sm = 2 * (size_t)L.ni * 4 * sizeof(double);
      smem_attr_once(k_sweep_cta<double>, 200 * 1024, 3);
      launch_pdl(k_sweep_cta<double>, 1, threads, sm, st, L, L.tb, L.yz64, rhs, do_update, aw, alpha);
    }
    return 1;
  }
  // Strips wait on one another: at most ceil(nj / SH) CTAs of 16*SH threads, launched on the
  // library's single stream after the previous kernel has finished, so all of them are
  // resident at once on the 152 SMs; every wait is bounded in any case.
  const int sh = kind == SWEEP_STRIPS16 ? 16 : kind == SWEEP_STRIPS4 ? 4 : 8;
  const int nb = (L.nj + sh - 1) / sh;
  cudaMemsetAsync(prog, 0, 2 * (size_t)nb * sizeof(long long), st);
  if (sh == 4) {
    if (mixed)
      launch_pdl(k_sweep_strips<float, 4>, nb, 64, 0, st, L, reinterpret_cast<const float*>(L.tb), L.yz32, rhs, prog, err,
                                                   limit, do_update, aw, alpha);
    else
      launch_pdl(k_sweep_strips<double, 4>, nb, 64, 0, st, L, L.tb, L.yz64, rhs, prog, err, limit, do_update, aw, alpha);
  } else if (sh == 16) {
    if (mixed)
      launch_pdl(k_sweep_strips<float, 16>, nb, 256, 0, st, L, reinterpret_cast<const float*>(L.tb), L.yz32, rhs, prog, err,
                                                    limit, do_update, aw, alpha);
    else
      launch_pdl(k_sweep_strips<double, 16>, nb, 256, 0, st, L, L.tb, L.yz64, rhs, prog, err, limit, do_update, aw, alpha);
  } else {
    if (mixed)
      launch_pdl(k_sweep_strips<float, 8>, nb, 128, 0, st, L, reinterpret_cast<const float*>(L.tb), L.yz32, rhs, prog, err,
                                                   limit, do_update, aw, alpha);
    else
      launch_pdl(k_sweep_strips<double, 8>, nb, 128, 0, st, L, L.tb, L.yz64, rhs, prog, err, limit, do_update, aw, alpha);
  }
  return 1;
}

int sweep_strips(const LevelDev& L) { return (L.nj + 3) / 4; }  // the most strips any kind uses

}  // namespace fasw
