// Warp-strip SGS sweep with bulk-copy staging (FP32 recurrence), and the FP64 defect correction
// that turns two such sweeps into an FP64-accurate application of the preconditioner.
//
// The sweeps apply P^-1 = ((D+L) D^-1 (D+U))^-1 of eq. (sgs-precon) (section 4.4) in the
// transfer-block form of kernels_sweep.cu:
//   forward  y_c = D_c^-1 r_c + G_W y_W + G_S y_S            (y_S: the wake-cut mirror on row 0
//                                                             of the upper wake),
//   backward z_c = y_c + H_E z_E + H_N z_N (+ G_S z_mirror on row 0 of the lower wake).
// Rows are cut into strips of 32, one warp each (lane = row); a lane holds all four components
// of its cell, so a step of the recurrence is its own previous vector (the west / east
// neighbour), the neighbour row's previous vector by one shuffle (south / north), and 32 FMAs.
// There is no barrier inside a step: a strip is one warp.  A strip's operands are laid out in
// the order the warp consumes them (strip-major, step by step; "skewed" so that lane jl at
// step s holds cell i = s - jl, with zero padding where that cell does not exist), so that the
// operands of CHUNK steps are one contiguous block: one elected lane moves it into shared
// memory with one cp.async.bulk per chunk and array, completion tracked by an mbarrier, double
// buffered, the first step's operands of the next chunk loaded before the last step of this one.
// The strips of a sweep form one thread-block cluster.  Strip b follows strip b-1 (forward; b+1
// backward) through the neighbour's boundary row: the neighbour's out lane stores its vector of
// every step straight into this strip's shared memory (a remote store inside the cluster), into
// a buffer that holds a sentinel bit pattern until the value lands; this strip polls its own
// shared memory once per chunk.  No fence or flag is needed: each 32-bit word arrives whole, and
// the sentinel (a NaN payload that no arithmetic produces) marks the words not yet written.
// Every wait is bounded; on timeout the kernel sets the error word, waits (bounded) for its own
// copies in flight, and still meets the cluster's barriers, so that no strip waits forever.
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "fasw_internal.cuh"
#include "fasw_sweep.cuh"

namespace fasw {

namespace {

constexpr int WS_STAGES = 2;   // chunk buffers (one in use, one in flight)
constexpr int WS_U = 8;        // steps unrolled together (a chunk of KC steps is KC / WS_U such blocks)
constexpr unsigned WS_SENT = 0xFFFFFFFFu;  // "not yet written": a NaN payload no FP32 operation returns

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// address of the same shared-memory variable in CTA `rank` of this cluster
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}

// predicated in the instruction itself (no branch around it: one lane of the warp stores)
__device__ __forceinline__ void st_cluster4_if(bool pred, unsigned addr, float4 v) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %5, 0;\n"
      " @p st.relaxed.cluster.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};\n}\n" ::"r"(addr),
      "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((unsigned)pred)
      : "memory");
}

__device__ __forceinline__ uint4 ld_cluster4(const float4* p) {
  uint4 v;
  asm volatile("ld.relaxed.cluster.shared::cta.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(smem_addr(p))
               : "memory");
  return v;
}

__device__ __forceinline__ bool unwritten(uint4 v) {
  return v.x == WS_SENT || v.y == WS_SENT || v.z == WS_SENT || v.w == WS_SENT;
}

// A lone strip (a cluster of one CTA, one warp) shares its shared memory with no one: a warp
// barrier orders its own accesses, and the cluster barrier is skipped.
__device__ __forceinline__ void cluster_sync() {
  __syncwarp();
  if (gridDim.x > 1)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  else
    __syncwarp();
}

__device__ __forceinline__ float4 shfl_up4(float4 v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_up_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_up_sync(0xffffffffu, v.w, 1);
  return v;
}

__device__ __forceinline__ float4 shfl_down4(float4 v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_down_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
  return v;
}

// out = c + A x + B w for row-major 4x4 blocks given as block rows A[0..3], B[0..3]
__device__ __forceinline__ float4 two_blocks(float4 c, const float4* A, float4 x, const float4* B, float4 w) {
  float o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // x (this lane's previous vector) is ready a shuffle earlier than w: one chain of eight FMAs,
    // the A-part first (measured faster than splitting the w-part into two shorter chains joined
    // by an add: four instructions fewer per step outweigh one FMA more of latency after the
    // shuffle; 64x16 sweep pair 20.6 -> 18.6 us, 1024x256 243.8 -> 237.7 us)
    const float4 a = A[q], b = B[q];
    float s = (q == 0 ? c.x : q == 1 ? c.y : q == 2 ? c.z : c.w);
    s = fmaf(a.x, x.x, s);
    s = fmaf(a.y, x.y, s);
    s = fmaf(a.z, x.z, s);
    s = fmaf(a.w, x.w, s);
    o[q] = fmaf(b.w, w.w, fmaf(b.z, w.z, fmaf(b.y, w.y, fmaf(b.x, w.x, s))));
  }
  return make_float4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ float4 add_block(float4 v, const float* G, float4 x) {
  v.x += G[0] * x.x + G[1] * x.y + G[2] * x.z + G[3] * x.w;
  v.y += G[4] * x.x + G[5] * x.y + G[6] * x.z + G[7] * x.w;
  v.z += G[8] * x.x + G[9] * x.y + G[10] * x.z + G[11] * x.w;
  v.w += G[12] * x.x + G[13] * x.y + G[14] * x.z + G[15] * x.w;
  return v;
}

// Shared memory of the sweep: [mbarriers][ring of blocks][ring of vectors][stage][edge][cut vectors][cut blocks]
struct WsSmem {
  uint64_t* bar;
  float4* ringF;  // WS_STAGES x KC x WS_F4_STEP
  float4* ringC;  // WS_STAGES x KC x 32
  float4* stage;  // KC: the neighbour's boundary vectors of the current chunk, checked
  float4* edge;   // Mp + 32: the neighbour's out-lane vector of its step t (t >= Mp: zero)
  float4* cutv;   // nw
  float* cutG;    // nw x 16
};

template <int KC>
__device__ __forceinline__ WsSmem ws_carve(unsigned char* base, int Mp, int nw) {
  WsSmem S;
  S.bar = reinterpret_cast<uint64_t*>(base);
  S.ringF = reinterpret_cast<float4*>(base + 128);
  S.ringC = S.ringF + WS_STAGES * KC * WS_F4_STEP;
  S.stage = S.ringC + WS_STAGES * KC * WS_ROWS;
  S.edge = S.stage + KC;
  S.cutv = S.edge + Mp + 32;
  S.cutG = reinterpret_cast<float*>(S.cutv + (nw > 0 ? nw : 1));
  return S;
}

}  // namespace

int ws_strips(int nj) { return (nj + WS_ROWS - 1) / WS_ROWS; }

size_t ws_smem_bytes(int ni, int nj, int nw, int KC) {
  const int m = nw > 0 ? nw : 1;
  return 128 + 16 * ((size_t)WS_STAGES * KC * (WS_F4_STEP + WS_ROWS) + KC + ws_steps(ni, nj) + 32 + m) +
         64 * (size_t)m;
}

namespace {

// Skewed index of cell (i, j) in the backward order (the layout of y as the backward pass reads
// it and of its result z): strip j / 32, step Mp - 1 - i - jl, lane jl.
__device__ __forceinline__ size_t ws_bpos(int i, int j, int Mp) {
  const int jl = j & (WS_ROWS - 1);
  return ((size_t)(j / WS_ROWS) * Mp + (Mp - 1 - i - jl)) * WS_ROWS + jl;
}

// One pass (forward: FWD, else backward) of one strip.  Returns false on a timeout.
// F: blocks of the pass, C: its right-hand side vectors (forward: D^-1 r; backward: y), both
// skewed; Out: the pass's result, skewed in the backward order (forward: y; backward: z).
// has_in: a neighbour strip feeds this one's edge lane (below forward, above backward) through
// S.edge; redge: the cluster address of the edge buffer of the strip this one feeds (0: none).
// Lane jl at step s holds cell i = s - jl (forward) or Mp - 1 - s - jl (backward); the edge lane
// needs the neighbour's out-lane vector of the same column, which the neighbour computed at its
// step s + 31: edge entry s + 31 (entries Mp .. Mp + 31 are zero).
template <bool FWD, int KC>
__device__ bool ws_pass(const LevelDev& L, const WsSmem& S, int b, const float4* F, const float4* C, float4* Out,
                        bool has_in, unsigned redge, int* err, long long limit, unsigned& phase_bits) {
  const int lane = threadIdx.x;
  const int ni = L.ni, nw = L.nw;
  const int Mp = ws_steps(ni, L.nj);        // steps that hold a cell, padded to whole chunks
  const int nch = Mp / KC;
  const int edge_lane = FWD ? 0 : WS_ROWS - 1;      // lane that reads the neighbour's row
  const int out_lane = FWD ? WS_ROWS - 1 : 0;       // lane whose row the other neighbour reads
  const float4* Fs = F + (size_t)b * Mp * WS_F4_STEP;
  const float4* Cs = C + (size_t)b * Mp * WS_ROWS;
  float4* Os = Out + (size_t)b * Mp * WS_ROWS + lane;
  const unsigned bytesF = KC * WS_F4_STEP * 16, bytesC = KC * WS_ROWS * 16;
  const bool feeds = redge != 0 && lane == out_lane;

  // Refill of a slot by the async proxy: the slot's previous contents were only read (no generic
  // writes), and every one of those reads has completed, its value used by an earlier step of
  // this warp, so no proxy fence is needed before the copy overwrites them.
  auto issue = [&](int ch) {  // lane 0 only
    const int slot = ch % WS_STAGES;
    mbar_expect_tx(&S.bar[slot], bytesF + bytesC);
    bulk_copy(S.ringF + (size_t)slot * KC * WS_F4_STEP, Fs + (size_t)ch * KC * WS_F4_STEP, bytesF, &S.bar[slot]);
    bulk_copy(S.ringC + (size_t)slot * KC * WS_ROWS, Cs + (size_t)ch * KC * WS_ROWS, bytesC, &S.bar[slot]);
  };
  int waited = 0;  // chunks whose copies have landed (and been accounted for)
  // bounded wait for the chunk in a slot; false on timeout
  auto wait_slot = [&](int slot) -> bool {
    const unsigned par = (phase_bits >> slot) & 1u;
    long long spins = 0;
    bool ok = true;
    while (!mbar_test(&S.bar[slot], par)) {
      if (++spins > limit) {
        ok = false;
        break;
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      phase_bits ^= 1u << slot;
      ++waited;
    }
    return ok;
  };
  int issued = 0;
  // after a timeout: wait for every copy still in flight into this CTA's shared memory before
  // returning.  These copies depend on no other CTA and finish within microseconds, so their
  // bound is fixed and generous, independent of the caller's (possibly tiny) spin limit.
  auto fail = [&]() {
    if (lane == 0) atomicExch(err, 1);
    for (int ch = waited; ch < issued; ++ch) {
      const int slot = ch % WS_STAGES;
      const unsigned par = (phase_bits >> slot) & 1u;
      long long spins = 0;
      while (!mbar_test(&S.bar[slot], par) && ++spins <= (1LL << 26)) {
      }
      phase_bits ^= 1u << slot;
    }
    __syncwarp();
    return false;
  };
  // the neighbour's boundary vectors of steps s0 .. s0 + KC - 1 into S.stage: lane k polls
  // edge entry s0 + 31 + k until the neighbour's store has landed (bounded; a neighbour that
  // gave up has set the error word)
  // The loop is warp-uniform (a vote decides whether any lane still waits), so that the warp
  // leaves it converged.
  auto poll_edge = [&](int s0) -> bool {
    const float4* e = S.edge + s0 + (WS_ROWS - 1) + (lane & (KC - 1));
    uint4 v = ld_cluster4(e);
    long long spins = 0;
    while (__any_sync(0xffffffffu, unwritten(v))) {
      if (++spins > limit || ((spins & 255) == 0 && *((volatile int*)err) != 0)) return false;
      v = ld_cluster4(e);
    }
    if (lane < KC)
      S.stage[lane] = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                  __uint_as_float(v.w));
    __syncwarp();
    return true;
  };

  if (lane == 0)
    for (int ch = 0; ch < WS_STAGES && ch < nch; ++ch) issue(ch);
  __syncwarp();
  issued = nch < WS_STAGES ? nch : WS_STAGES;
  if (!has_in && lane < KC) S.stage[lane] = make_float4(0.f, 0.f, 0.f, 0.f);  // no neighbour: zero
  __syncwarp();

  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);  // this lane's vector at the previous step
  // Operands of one step: this lane's rows of the two blocks and its right-hand side vector,
  // loaded one step ahead of their use (across chunk boundaries too: the next chunk's first
  // step is loaded before this chunk's last), and the edge value, loaded one step ahead inside
  // a chunk, so that shared-memory latency stays off the chain.
  struct Ops {
    float4 A[4], B[4], c;
  };
  auto load = [&](Ops& o, int slot, int k) {
    const float4* rF = S.ringF + (size_t)slot * KC * WS_F4_STEP;
    const float4* rC = S.ringC + (size_t)slot * KC * WS_ROWS;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      o.A[q] = rF[k * WS_F4_STEP + q * WS_ROWS + lane];
      o.B[q] = rF[k * WS_F4_STEP + (4 + q) * WS_ROWS + lane];
    }
    o.c = rC[k * WS_ROWS + lane];
  };
  // One step.  Padded positions (no cell) carry zero blocks and vectors, so they compute zero
  // and need no test: every step writes its result.  Only the wake-cut coupling of row 0
  // (strip 0, lane 0) is special, and chunks that hold no cut cell run the step without it
  // (CUT false).
  auto step = [&](const Ops& o, float4 e, int s, auto cut_tag) {
    constexpr bool CUT = decltype(cut_tag)::value;
    float4 w = FWD ? shfl_up4(v) : shfl_down4(v);  // the row below (forward) / above (backward)
    if (lane == edge_lane) w = e;                   // neighbour strip's row, or zero
    const int i = FWD ? s - lane : Mp - 1 - s - lane;  // this lane's cell (i, j)
    if constexpr (CUT && FWD)
      if (lane == 0 && i >= ni - nw && i < ni) w = S.cutv[ni - 1 - i];  // upper wake: its mirror
    float4 y = two_blocks(o.c, o.A, v, o.B, w);
    if constexpr (CUT && !FWD)
      if (lane == 0 && i >= 0 && i < nw) y = add_block(y, S.cutG + 16 * i, S.cutv[i]);  // lower wake
    if constexpr (CUT) {
      if (lane == 0 && FWD && i >= 0 && i < nw) S.cutv[i] = y;                   // read by its mirror
      if (lane == 0 && !FWD && i >= ni - nw && i < ni) S.cutv[ni - 1 - i] = y;   // read by its mirror
    }
    Os[(size_t)(FWD ? Mp - 1 - s : s) * WS_ROWS] = y;
    st_cluster4_if(feeds, redge + 16u * (unsigned)s, y);  // the fed strip's edge entry s
    v = y;
  };
  // o[0] holds the next step's operands between chunks: the last step of a chunk loads the next
  // chunk's first step into it.  A chunk runs as KC / WS_U blocks of WS_U unrolled steps, which
  // keeps the code of a pass small enough for the instruction cache.
  Ops o[2];
  float4 e[2];
  bool late = false;  // the next chunk's wait gave up
  auto run_chunk = [&](int slot, int ch, int s0, auto cut_tag) {
    e[0] = S.stage[0];
#pragma unroll 1
    for (int kk = 0; kk < KC; kk += WS_U) {
#pragma unroll
      for (int u = 0; u < WS_U; ++u) {
        const int k = kk + u;
        if (u + 1 < WS_U || kk + WS_U < KC) {
          load(o[(u + 1) & 1], slot, k + 1);
          e[(u + 1) & 1] = S.stage[k + 1];
        } else if (ch + 1 < nch) {
          if (wait_slot((ch + 1) % WS_STAGES))
            load(o[0], (ch + 1) % WS_STAGES, 0);
          else
            late = true;
        }
        step(o[u & 1], e[u & 1], s0 + k, cut_tag);
      }
    }
  };

  if (!wait_slot(0)) return fail();
  load(o[0], 0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    const int s0 = ch * KC;
    if (has_in && !poll_edge(s0)) return fail();
    const int slot = ch % WS_STAGES;
    // does lane 0 of strip 0 meet a wake-cut cell in this chunk?
    const int ilo = FWD ? s0 : Mp - s0 - KC, ihi = FWD ? s0 + KC - 1 : Mp - 1 - s0;
    const bool cut = b == 0 && nw > 0 && (ilo < nw || ihi >= ni - nw);
    if (cut)
      run_chunk(slot, ch, s0, std::true_type{});
    else
      run_chunk(slot, ch, s0, std::false_type{});
    __syncwarp();
    if (late) return fail();
    // this chunk's slot is free again (its operands are all in registers or consumed)
    if (lane == 0 && issued < nch) issue(issued);
    if (issued < nch) ++issued;
    __syncwarp();
  }
  return true;
}

// the edge buffer before a pass: entries the neighbour will write hold the sentinel, the
// entries past the last step zero
__device__ __forceinline__ void ws_clear_edge(const WsSmem& S, int Mp) {
  const float sent = __uint_as_float(WS_SENT);
  for (int t = threadIdx.x; t < Mp + 32; t += 32)
    S.edge[t] = t < Mp ? make_float4(sent, sent, sent, sent) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// One launch: forward then backward pass of strip b (one warp per CTA, the nb strips one
// cluster).  Every strip meets the cluster barriers (set-up, between the passes, at the end)
// whatever happened in its passes, so that a strip that gave up leaves no other one waiting on
// a barrier; the last barrier also keeps every strip's shared memory alive until the
// neighbours' remote stores into it have completed.
template <int KC>
__global__ void __launch_bounds__(32) k_sweep_ws(LevelDev L, const float4* Fb, const float4* Bb, const float4* C,
                                                 float4* Y, const float* cutG, float4* Z, int* err, long long limit) {
  pdl_entry();
  extern __shared__ __align__(128) unsigned char ws_raw[];
  const int nw = L.nw;
  const int Mp = ws_steps(L.ni, L.nj);
  WsSmem S = ws_carve<KC>(ws_raw, Mp, nw);
  const int b = blockIdx.x, nb = gridDim.x, lane = threadIdx.x;
  if (lane == 0) {
    for (int k = 0; k < WS_STAGES; ++k) mbar_init(&S.bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (b == 0)
    for (int x = lane; x < 16 * nw; x += 32) S.cutG[x] = cutG[x];
  ws_clear_edge(S, Mp);
  // every strip's edge buffer holds its sentinels before any neighbour stores into it
  cluster_sync();
  unsigned phase_bits = 0;
  // forward: strip b feeds b + 1 (lane 31) and is fed by b - 1; backward the other way round
  const unsigned up = b < nb - 1 ? cluster_addr(S.edge, (unsigned)(b + 1)) : 0u;
  const unsigned down = b > 0 ? cluster_addr(S.edge, (unsigned)(b - 1)) : 0u;
  bool ok = ws_pass<true, KC>(L, S, b, Fb, C, Y, b > 0, up, err, limit, phase_bits);
  // the backward pass reads, through the async proxy, the y this warp has just written
  asm volatile("fence.proxy.async.global;" ::: "memory");
  // every strip has read its edge buffer to the end before it is cleared for the backward pass,
  // and cleared before a neighbour stores into it again
  cluster_sync();
  ws_clear_edge(S, Mp);
  cluster_sync();
  if (ok) ws_pass<false, KC>(L, S, b, Bb, Y, Z, b < nb - 1, down, err, limit, phase_bits);
  cluster_sync();
}

// ---------------------------------------------------------------- operand layout
// Skewed position of cell (i, j): strip b = j / 32, lane jl = j % 32, forward step s = i + jl,
// backward step Mp - 1 - i - jl (Mp: the ni + R - 1 steps that hold a cell, R = min(nj, 32), padded to whole chunks).

// Forward right-hand side D^-1 r (FP32), skewed.
// The FP64 kernels of one application, written per row q of their block products: a thread
// takes one cell and all four rows (SPLIT false: the loads of a warp coalesce along the cells, for
// levels whose time is their memory traffic), or one cell and one row (SPLIT true: a quarter of
// the FP64 chain per thread, for the small levels whose time is that chain).  Every row is summed
// in the same order either way.
constexpr int WS_SPLIT_CELLS = 16384;  // levels up to this many cells take one thread per row

template <bool SPLIT>
__device__ __forceinline__ bool ws_thread(const LevelDev& L, int& c, int& q0, int& q1) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (SPLIT) {
    c = g >> 2;
    q0 = g & 3;
    q1 = q0 + 1;
  } else {
    c = g;
    q0 = 0;
    q1 = 4;
  }
  return c < L.n;
}

// row q of D^-1 r
template <typename T>
__device__ __forceinline__ double rhs_row(const LevelDev& L, const T* tb, const double* rhs, int c, int q) {
  const int n = L.n;
  double a = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) a += double(tb[(size_t)(4 * q + t) * n + c]) * rhs[(size_t)t * n + c];
  return a;
}

template <typename T, bool SPLIT>
__global__ void k_ws_rhs(LevelDev L, const T* tb, const double* rhs, float4* C) {
  pdl_entry();
  int c, q0, q1;
  if (!ws_thread<SPLIT>(L, c, q0, q1)) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  const int b = j / WS_ROWS, jl = j % WS_ROWS, Mp = ws_steps(ni, L.nj);
  float* out = reinterpret_cast<float*>(C + ((size_t)b * Mp + (i + jl)) * WS_ROWS + jl);
  for (int q = q0; q < q1; ++q) out[q] = float(rhs_row(L, tb, rhs, c, q));
}

// ---------------------------------------------------------------- FP64 defect correction
// t = (I + U~) z0: the vector the backward sweep would have started from to reach z0,
//   t_c = z0_c - H_E z0_E - H_N z0_N (- G_S z0_mirror on row 0 of the lower wake).
__device__ __forceinline__ double defect_t_row(const LevelDev& L, const double* tb, const float4* z0, int c, int q) {
  const int ni = L.ni, nj = L.nj, n = L.n, i = c % ni, j = c / ni;
  const int Mp = ws_steps(ni, nj);
  const float4 zc = z0[ws_bpos(i, j, Mp)];
  double acc = q == 0 ? zc.x : q == 1 ? zc.y : q == 2 ? zc.z : zc.w;
  auto sub = [&](int blk, int cn) {
    const float4 zn = z0[ws_bpos(cn % ni, cn / ni, Mp)];
    const double x[4] = {zn.x, zn.y, zn.z, zn.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) acc -= tb[(size_t)(blk * 16 + 4 * q + k) * n + c] * x[k];
  };
  if (i < ni - 1) sub(3, c + 1);
  if (j < nj - 1) sub(4, c + ni);
  if (j == 0 && L.nw > 0 && i < L.nw && ni - 1 - i > i) sub(2, ni - 1 - i);
  return acc;
}

template <bool SPLIT>
__global__ void k_ws_defect_t(LevelDev L, const double* tb, const float4* z0, double* t) {
  pdl_entry();
  int c, q0, q1;
  if (!ws_thread<SPLIT>(L, c, q0, q1)) return;
  for (int q = q0; q < q1; ++q) t[(size_t)q * L.n + c] = defect_t_row(L, tb, z0, c, q);
}

// d = D^-1 r - (I + L~) t = D^-1 r - t_c + G_W t_W + G_S t_S (t_S: the mirror on row 0 of the
// upper wake, none elsewhere on row 0), written as the next forward right-hand side (FP32).
__device__ __forceinline__ double defect_d_row(const LevelDev& L, const double* tb, const double* rhs,
                                               const double* t, int c, int q) {
  const int ni = L.ni, n = L.n, i = c % ni, j = c / ni;
  double a = -t[(size_t)q * n + c];
#pragma unroll
  for (int k = 0; k < 4; ++k) a += tb[(size_t)(4 * q + k) * n + c] * rhs[(size_t)k * n + c];
  auto add = [&](int blk, int cn) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a += tb[(size_t)(blk * 16 + 4 * q + k) * n + c] * t[(size_t)k * n + cn];
  };
  if (i > 0) add(1, c - 1);
  if (j > 0) add(2, c - ni);
  else if (L.nw > 0 && i >= ni - L.nw && ni - 1 - i < i) add(2, ni - 1 - i);
  return a;
}

template <bool SPLIT>
__global__ void k_ws_defect_d(LevelDev L, const double* tb, const double* rhs, const double* t, float4* C) {
  pdl_entry();
  int c, q0, q1;
  if (!ws_thread<SPLIT>(L, c, q0, q1)) return;
  const int ni = L.ni, i = c % ni, j = c / ni;
  const int b = j / WS_ROWS, jl = j % WS_ROWS, Mp = ws_steps(ni, L.nj);
  float* out = reinterpret_cast<float*>(C + ((size_t)b * Mp + (i + jl)) * WS_ROWS + jl);
  for (int q = q0; q < q1; ++q) out[q] = float(defect_d_row(L, tb, rhs, t, c, q));
}

// z = z0 (+ dz): the stage update u = u0 - alpha z (scaled by dt* for ARK), or z to the level's
// sweep vector (FP64 contexts: yz64; mixed: yz32).
__global__ void k_ws_finish(LevelDev L, const float4* z0, const float4* dz, int do_update, int aw, double alpha,
                            int mixed) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, i = c % L.ni, j = c / L.ni;
  const size_t zp = ws_bpos(i, j, ws_steps(L.ni, L.nj));
  const float4 a = z0[zp];
  double z[4] = {a.x, a.y, a.z, a.w};
  if (dz) {
    const float4 d = dz[zp];
    z[0] += d.x;
    z[1] += d.y;
    z[2] += d.z;
    z[3] += d.w;
  }
  if (do_update) {
    const double sc = aw ? alpha : alpha * L.dts[c];
    const size_t g = (size_t)(j + 2) * L.P + (i + 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) L.u[q * (size_t)L.Gn + g] = L.u0[q * (size_t)n + c] - sc * z[q];
  } else if (mixed) {
#pragma unroll
    for (int q = 0; q < 4; ++q) L.yz32[q * (size_t)n + c] = float(z[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) L.yz64[q * (size_t)n + c] = z[q];
  }
}

// ---------------------------------------------------------------- the exact preconditioner
// Block Gauss-Seidel iterations on the full first-order operator A = D + L + U (the "exact"
// preconditioner of section 5.4's tables is A^-1): x <- x + P^-1 (r - A x), each P^-1 one
// warp-strip sweep pair, converging to A^-1 r.  x accumulates in FP64 (cell-major, 4 per cell).

// x = (init ? 0 : x) + z0 (+ dz), z0 / dz skewed in the backward order
__global__ void k_ws_accum(LevelDev L, const float4* z0, const float4* dz, double* x, int init) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int i = c % L.ni, j = c / L.ni;
  const size_t zp = ws_bpos(i, j, ws_steps(L.ni, L.nj));
  const float4 a = z0[zp];
  double v[4] = {a.x, a.y, a.z, a.w};
  if (dz) {
    const float4 d = dz[zp];
    v[0] += d.x;
    v[1] += d.y;
    v[2] += d.z;
    v[3] += d.w;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) x[4 * (size_t)c + q] = (init ? 0.0 : x[4 * (size_t)c + q]) + v[q];
}

// D^-1 (r - A x) = D^-1 r - x + G_W x_W + G_S x_S + H_E x_E + H_N x_N (+ G_S x_mirror on row 0 of
// the wake cut, either side), as the next sweep's right-hand side (skewed, FP32)
template <typename T>
__global__ void k_ws_exact_defect(LevelDev L, const T* tb, const double* rhs, const double* x, float4* C) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int ni = L.ni, nj = L.nj, n = L.n, i = c % ni, j = c / ni;
  double r[4], acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = rhs[(size_t)k * n + c];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double a = -x[4 * (size_t)c + q];
#pragma unroll
    for (int k = 0; k < 4; ++k) a += double(tb[(size_t)(4 * q + k) * n + c]) * r[k];
    acc[q] = a;
  }
  auto add = [&](int blk, int cn) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[q] += double(tb[(size_t)(blk * 16 + 4 * q + k) * n + c]) * x[4 * (size_t)cn + k];
  };
  if (i > 0) add(1, c - 1);
  if (j > 0) add(2, c - ni);
  else if (L.nw > 0 && (i < L.nw || i >= ni - L.nw)) add(2, ni - 1 - i);
  if (i < ni - 1) add(3, c + 1);
  if (j < nj - 1) add(4, c + ni);
  const int b = j / WS_ROWS, jl = j % WS_ROWS, Mp = ws_steps(ni, L.nj);
  C[((size_t)b * Mp + (i + jl)) * WS_ROWS + jl] = make_float4(float(acc[0]), float(acc[1]), float(acc[2]), float(acc[3]));
}

// the stage update (or the result vector) from the accumulated x
__global__ void k_ws_finish_x(LevelDev L, const double* x, int do_update, int aw, double alpha, int mixed) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  const int n = L.n, i = c % L.ni, j = c / L.ni;
  if (do_update) {
    const double sc = aw ? alpha : alpha * L.dts[c];
    const size_t g = (size_t)(j + 2) * L.P + (i + 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) L.u[q * (size_t)L.Gn + g] = L.u0[q * (size_t)n + c] - sc * x[4 * (size_t)c + q];
  } else if (mixed) {
#pragma unroll
    for (int q = 0; q < 4; ++q) L.yz32[q * (size_t)n + c] = float(x[4 * (size_t)c + q]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) L.yz64[q * (size_t)n + c] = x[4 * (size_t)c + q];
  }
}

constexpr size_t kWsSmemMax = 227 * 1024;

}  // namespace

bool ws_fits(int ni, int nj, int nw) {
  return ws_strips(nj) <= 8 && ws_smem_bytes(ni, nj, nw, WS_K) <= kWsSmemMax;  // one portable cluster per sweep
}


namespace {
template <int KC>
cudaError_t ws_sweep_launch(const LevelDev& L, float4* zout, int* err, long long limit, cudaStream_t st) {
  const int nb = ws_strips(L.nj);
  const size_t sm = ws_smem_bytes(L.ni, L.nj, L.nw, KC);
  // the shared-memory limit is a per-device attribute of each instance: set once on each device
  // (idempotent if two host threads race on the first launch)
  static std::atomic<unsigned long long> attr_done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(attr_done.load() & (1ull << dev))) {
    if (cudaFuncSetAttribute(k_sweep_ws<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemMax) ==
        cudaSuccess)
      attr_done.fetch_or(1ull << dev);
  }
  // The strips of one sweep wait on one another, so they are launched as one thread-block
  // cluster (nb <= 8 CTAs): the hardware schedules a cluster's CTAs together, so every strip is
  // resident whatever else runs beside it (concurrent cases of a batch included).
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = nb;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_sweep_ws<KC>, L, reinterpret_cast<const float4*>(L.wsF),
                            reinterpret_cast<const float4*>(L.wsB), reinterpret_cast<const float4*>(L.wsC),
                            reinterpret_cast<float4*>(L.wsY), static_cast<const float*>(L.wsCut), zout, err,
                            limit);
}
}  // namespace

int launch_ws_sweep(const LevelDev& L, int mixed, int refine, int do_update, int aw, double alpha, const double* rhs,
                    long long* prog, int* err, long long limit, cudaStream_t st, int exact_iters, int chunk) {
  (void)prog;  // the warp strips exchange their boundary rows in shared memory, not through progress words
  auto sweep = [&](float4* zout) {
    return chunk == 8 ? ws_sweep_launch<8>(L, zout, err, limit, st) : ws_sweep_launch<WS_K>(L, zout, err, limit, st);
  };
  const int g = (L.n + 127) / 128;
  float4* z0 = reinterpret_cast<float4*>(L.wsZ);
  float4* dz = z0 + ws_vec_floats(L.ni, L.nj) / 4;
  int launches = 0;
  const bool split = L.n <= WS_SPLIT_CELLS;
  const int g4 = (4 * L.n + 127) / 128;  // one thread per cell and row
  float4* wC = reinterpret_cast<float4*>(L.wsC);
  const double* tb64 = static_cast<const double*>(L.tb);
  if (mixed) {
    const float* tb32 = reinterpret_cast<const float*>(L.tb);
    if (split)
      launch_pdl(k_ws_rhs<float, true>, g4, 128, 0, st, L, tb32, rhs, wC);
    else
      launch_pdl(k_ws_rhs<float, false>, g, 128, 0, st, L, tb32, rhs, wC);
  } else if (split) {
    launch_pdl(k_ws_rhs<double, true>, g4, 128, 0, st, L, tb64, rhs, wC);
  } else {
    launch_pdl(k_ws_rhs<double, false>, g, 128, 0, st, L, tb64, rhs, wC);
  }
  sweep(z0);
  launches += 2;
  const bool corr = refine && !mixed;
  if (corr) {
    const float4* z0c = z0;
    const double* wT = L.wsT;
    if (split) {
      launch_pdl(k_ws_defect_t<true>, g4, 128, 0, st, L, tb64, z0c, L.wsT);
      launch_pdl(k_ws_defect_d<true>, g4, 128, 0, st, L, tb64, rhs, wT, wC);
    } else {
      launch_pdl(k_ws_defect_t<false>, g, 128, 0, st, L, tb64, z0c, L.wsT);
      launch_pdl(k_ws_defect_d<false>, g, 128, 0, st, L, tb64, rhs, wT, wC);
    }
    sweep(dz);
    launches += 3;
  }
  if (exact_iters > 0) {
    launch_pdl(k_ws_accum, g, 128, 0, st, L, static_cast<const float4*>(z0),
               corr ? static_cast<const float4*>(dz) : nullptr, L.wsX, 1);
    ++launches;
    for (int it = 0; it < exact_iters; ++it) {
      if (mixed)
        launch_pdl(k_ws_exact_defect<float>, g, 128, 0, st, L, reinterpret_cast<const float*>(L.tb), rhs,
                   static_cast<const double*>(L.wsX), reinterpret_cast<float4*>(L.wsC));
      else
        launch_pdl(k_ws_exact_defect<double>, g, 128, 0, st, L, static_cast<const double*>(L.tb), rhs,
                   static_cast<const double*>(L.wsX), reinterpret_cast<float4*>(L.wsC));
      sweep(z0);
      launch_pdl(k_ws_accum, g, 128, 0, st, L, static_cast<const float4*>(z0), nullptr, L.wsX, 0);
      launches += 3;
    }
    launch_pdl(k_ws_finish_x, g, 128, 0, st, L, static_cast<const double*>(L.wsX), do_update, aw, alpha, mixed);
    return launches + 1;
  }
  launch_pdl(k_ws_finish, g, 128, 0, st, L, static_cast<const float4*>(z0), corr ? static_cast<const float4*>(dz) : nullptr,
             do_update, aw, alpha, mixed);
  return launches + 1;
}

size_t ws_floats(int ni, int nj) { return (size_t)ws_strips(nj) * ws_steps(ni, nj) * WS_F4_STEP * 4; }
size_t ws_vec_floats(int ni, int nj) { return (size_t)ws_strips(nj) * ws_steps(ni, nj) * WS_ROWS * 4; }

}  // namespace fasw
