// gabp_kernels.cu -- sm_103a kernels of the synchronous broadcast GaBP sweep
// and the device-side solve controller.
//
// Every sweep kernel implements one round of Alg. 2 (broadcast GaBP) with the
// parallel schedule of Section III-C: it reads only the previous round's
// messages (buffer "in") and writes the new round (buffer "out").  Slot s of
// row i holds the incoming message m_{j->i}; a row forms
//     P~_i = A_ii + sum_k P_ki,        h~_i = b_i + sum_k eta_ki      (eta = P mu)
// and sends, to slot rev[s] of row j,
//     P_ij   = -A_ij^2 / (P~_i - P_ji),
//     eta_ij = -A_ij (h~_i - eta_ji) / (P~_i - P_ji),
// using the reverse message m_{j->i} it already holds.  Reads are contiguous;
// only the message store is a scatter.
//
// Memory pipeline: persistent CTAs walk row tiles (a few thousand slots of
// consecutive rows).  Thread 0 stages the next tile's contiguous slot and node
// arrays into shared memory with cp.async.bulk on an mbarrier while the CTA
// computes the current tile from shared memory.
//
// Work mapping inside a tile (FP32 sweeps): slot-parallel.  Threads take slots
// tid, tid + blockDim, ...; the tile-local row id of each slot (staged with the
// slots) drives a warp-segmented sum whose run heads add into per-row totals
// in shared memory; after one barrier every slot sends its message and one
// thread per row does the node work.  Lanes stay busy whatever the degree
// distribution.  The FP64 sweep keeps a G-lanes-per-row mapping (its row sums
// cost one FP64 add per slot; a segmented scan would cost five on GB300's
// 1/64-rate FP64 pipe).
//
// Control: kernels take their buffer parities and flags from the control
// block (Ctl).  The last block to finish a launch (detected with an atomic
// counter, no waiting) runs `control`, which reads the reductions, decides the
// next phase, and -- inside a solve graph -- sets the graph's WHILE and SWITCH
// conditions.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>
#include <unordered_map>

namespace gabp {
namespace {

// Warp sum by key over 32 consecutive slots whose keys (tile-local row ids)
// do not decrease along the lanes: a doubling scan that only adds a partner
// with the same key, so after five steps the first lane of every run of
// equal keys holds the run's total.  Sets `head` in those lanes.
__device__ __forceinline__ float shfl_down(float v, int off) {
  return __shfl_down_sync(0xffffffffu, v, off);
}
__device__ __forceinline__ float2 shfl_down(float2 v, int off) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
}
__device__ __forceinline__ void add_to(float &a, float b) { a += b; }
__device__ __forceinline__ void add_to(float2 &a, float2 b) { a.x += b.x; a.y += b.y; }

template <class V>
__device__ __forceinline__ V seg_sum(V v, int key, bool &head) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const V w = shfl_down(v, off);
    const int k = __shfl_down_sync(0xffffffffu, key, off);
    if (lane + off < 32 && k == key) add_to(v, w);
  }
  const int kp = __shfl_up_sync(0xffffffffu, key, 1);
  head = lane == 0 || kp != key;
  return v;
}

// Storage type of the mean messages: FP32, or BF16 with FP32 arithmetic.
__device__ __forceinline__ float ld_eta(const float *p) { return *p; }
__device__ __forceinline__ float ld_eta(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void store_eta(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_eta(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }


// ---------------------------------------------------------------------------
// Solve set-up: ||b||_inf; in the mixed modes also x = 0 and r = b.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) init_kernel(int32_t n, double *__restrict__ r64,
                                                      Ctl *ctl, DevScalars *red,
                                                      const int32_t *__restrict__ sys_of_row,
                                                      unsigned long long *sys_bmax) {
  const double *b = ctl->b;
  double *x = ctl->x;
  const bool mixed = ctl->mode == CTL_MIXED, prec = ctl->mode == CTL_PREC;
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (prec) { r64[i] = 0.0; continue; }
    const double bi = b[i];
    m = umax(m, bits(fabs(bi)));
    if (mixed) { x[i] = 0.0; r64[i] = bi; }
    if (sys_bmax) atomicMax(&sys_bmax[sys_of_row[i]], bits(fabs(bi)));
  }
  block_max4(m, 0, 0, 0, &red->max_b, nullptr, nullptr, nullptr);
  last_block_control(ctl, red, CK_INIT);
}

// ---------------------------------------------------------------------------
// Shared-memory staging of row tiles.
//
// A tile is a run of consecutive rows [r0, r1) whose slots [s0, s1) number
// at most TS (and rows at most TR); a row with more than TS slots is a tile
// of its own ("long tile") that the whole CTA processes straight from global
// memory.  Every wait is bounded; a wait that gives up sets `timeout` in the
// reductions (the controller then stops the solve with GABP_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
constexpr int kTileSlotsBig = 1024, kTileRowsBig = 256;     // FP32 sweeps, residual
constexpr int kTileSlotsSmall = 1024, kTileRowsSmall = 256; // FP64 sweep
constexpr int kTileBlock = 128;                             // threads of the FP32 / residual tile kernels
constexpr int kNoRow = 0xFFFF;                              // key of lanes past the tile's end

// Scattered message stores, kept in L2 (evict-last).
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(__nv_bfloat16 *p, float v, uint64_t pol) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const unsigned short u = *reinterpret_cast<const unsigned short *>(&h);
  asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(u), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float2 *p, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
               "l"(pol)
               : "memory");
}

struct TileBounds {
  int32_t r0, r1, s0, s1;
};
__device__ __forceinline__ TileBounds tile_at(const int2 *__restrict__ tiles, int32_t t) {
  const int2 a = tiles[t], b = tiles[t + 1];
  return TileBounds{a.x, b.x, a.y, b.y};
}

// Persistent two-stage loop over the tiles.  `issue(t, stage, bar)` is called
// by thread 0 and must arrive once on `bar` with the bytes it copies.
// `work(t, stage, st, got)` is called by all threads once thread-local waits
// returned (`got` = this thread saw the stage land); it must pass
// __syncthreads_or(!got) before any side effect outside shared memory and
// return that value (true = abort).  Returns false if a wait gave up (after
// draining the copy in flight).
template <class Issue, class Work>
__device__ bool run_tiles(int32_t ntiles, unsigned char *smem, uint32_t stage_bytes,
                          uint64_t *bars, Issue issue, Work work) {
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  int32_t t = blockIdx.x;
  if (t < ntiles && threadIdx.x == 0) issue(t, smem, bar0);
  bool ok = true;
  for (int j = 0; t < ntiles; ++j, t += gridDim.x) {
    const int st = j & 1;
    const uint32_t bar_cur = st ? bar1 : bar0, bar_next = st ? bar0 : bar1;
    const int32_t tn = t + gridDim.x;
    if (tn < ntiles && threadIdx.x == 0) {
      fence_proxy_async();   // stage st^1 was last read by generic loads
      issue(tn, smem + (st ^ 1) * stage_bytes, bar_next);
    }
    const bool got = mbar_wait(bar_cur, (j >> 1) & 1);
    if (work(t, smem + st * stage_bytes, st, got)) {
      ok = false;
      if (tn < ntiles) mbar_wait(bar_next, ((j + 1) >> 1) & 1);
      __syncthreads();
      break;
    }
    __syncthreads();
  }
  return ok;
}


// ---------------------------------------------------------------------------
// FP64 full sweep: new (P, eta) for every directed edge, plus (when asked)
// the tentative means x_i = h~_i / P~_i of the messages read (Alg. 2 step 4).
// Staged per tile: (P, eta) in, A_ij, rev, row pointers, A_ii.  G lanes per
// row.
// ---------------------------------------------------------------------------
struct Layout64 {
  static constexpr int TS = kTileSlotsSmall, TR = kTileRowsSmall;
  static constexpr uint32_t m = 0, a = m + region(TS, 16), rev = a + region(TS, 8),
                            rp = rev + region(TS, 4), dg = rp + region(TR + 1, 4),
                            bytes = dg + region(TR, 8);
};

template <int G>
__global__ void __launch_bounds__(kBlock)
sweep64_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red) {
  using L = Layout64;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  const int par = ctl->par_m;
  const bool first = ctl->first != 0;
  // incoming messages known to be zero (skip reading them): the first sweep of
  // a synchronous solve; an in-place colour schedule reads its zeroed buffer
  const bool zin = first && !g.in_place;
  bool write_x, write_msgs;
  if (ctl->mode == CTL_ROUNDS) {
    const bool infer_only = ctl->sweeps >= ctl->rounds_target;
    write_x = infer_only || ctl->write_x != 0;
    write_msgs = !infer_only;
  } else {
    write_x = ctl->write_x != 0;
    write_msgs = true;
  }
  const double *__restrict__ b = ctl->b;
  double *__restrict__ x = ctl->xw;   // x itself, or a slot of the Aitken ring
  const double2 *__restrict__ min = (par ? B.m64[1] : B.m64[0]);
  double2 *__restrict__ mout = (par ? B.m64[0] : B.m64[1]);
  const int gl = threadIdx.x % G;
  bool brk = false;

  auto issue = [&](int32_t t, unsigned char *stage, uint32_t bar) {
    const TileBounds tb = tile_at(g.tiles_small, t);
    const int64_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) { mbar_expect_tx(bar, 0); return; }
    const uint32_t tx = (zin ? 0 : Seg<double2>::bytes(tb.s0, ns)) +
                        Seg<double>::bytes(tb.s0, ns) + Seg<int32_t>::bytes(tb.s0, ns) +
                        Seg<int32_t>::bytes(tb.r0, nr + 1) + Seg<double>::bytes(tb.r0, nr);
    mbar_expect_tx(bar, tx);
    const uint32_t base = smem_u32(stage);
    if (!zin) Seg<double2>::copy(base + L::m, min, tb.s0, ns, bar);
    Seg<double>::copy(base + L::a, g.a64, tb.s0, ns, bar);
    Seg<int32_t>::copy(base + L::rev, g.rev, tb.s0, ns, bar);
    Seg<int32_t>::copy(base + L::rp, g.rp, tb.r0, nr + 1, bar);
    Seg<double>::copy(base + L::dg, g.diag64, tb.r0, nr, bar);
  };

  const double gam = g.no_damp ? 0.0 : ctl->damping;
  auto emit = [&](double a, double2 m, int32_t dst, double TP, double Th) {
    const double d = TP - m.x;   // P_{i\j} = P~_i - P_ji
    brk |= zero_or_nonfinite(d);
    const double inv = recip64(d);
    double eta = -a * (Th - m.y) * inv;
    // damping: blend with this message's previous value (slot dst of "in")
    if (gam > 0.0) eta = gam * (zin ? 0.0 : min[dst].y) + (1.0 - gam) * eta;
    mout[dst] = make_double2(-(a * a) * inv, eta);
  };

  auto work = [&](int32_t t, unsigned char *stage, int, bool got) {
    if (__syncthreads_or(!got)) return true;
    const TileBounds tb = tile_at(g.tiles_small, t);
    const int32_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) {
      // one long row, straight from global memory, the whole CTA on it
      const int32_t i = tb.r0;
      double sP = 0.0, sH = 0.0;
      if (!zin)
        for (int32_t s = tb.s0 + threadIdx.x; s < tb.s1; s += blockDim.x) {
          const double2 m = min[s];
          sP += m.x;
          sH += m.y;
        }
      sP = block_sum(sP);
      sH = block_sum(sH);
      const double TP = g.diag64[i] + sP, Th = b[i] + sH;
      if (write_x && threadIdx.x == 0) x[i] = Th / TP;
      if (write_msgs)
        for (int32_t s = tb.s0 + threadIdx.x; s < tb.s1; s += blockDim.x)
          emit(g.a64[s], zin ? make_double2(0.0, 0.0) : min[s], g.rev[s], TP, Th);
      return false;
    }
    const double2 *ms = Seg<double2>::at(stage + L::m, tb.s0);
    const double *as = Seg<double>::at(stage + L::a, tb.s0);
    const int32_t *rv = Seg<int32_t>::at(stage + L::rev, tb.s0);
    const int32_t *rp = Seg<int32_t>::at(stage + L::rp, tb.r0);
    const double *dg = Seg<double>::at(stage + L::dg, tb.r0);
    for (int32_t base_r = 0; base_r < nr; base_r += kBlock / G) {
      const int32_t lr = base_r + static_cast<int32_t>(threadIdx.x) / G;
      const bool valid = lr < nr;
      const int32_t rs = valid ? rp[lr] - tb.s0 : 0, re = valid ? rp[lr + 1] - tb.s0 : 0;
      double sP = 0.0, sH = 0.0;
      if (!zin)
        for (int32_t s = rs + gl; s < re; s += G) {
          sP += ms[s].x;
          sH += ms[s].y;
        }
      sP = group_sum<G>(sP);
      sH = group_sum<G>(sH);
      if (!valid) continue;
      const int32_t i = tb.r0 + lr;
      const double TP = dg[lr] + sP, Th = b[i] + sH;
      if (write_x && gl == 0) x[i] = Th / TP;
      if (!write_msgs) continue;
      for (int32_t s = rs + gl; s < re; s += G)
        emit(as[s], zin ? make_double2(0.0, 0.0) : ms[s], rv[s], TP, Th);
    }
    return false;
  };

  const bool ok = run_tiles(g.ntiles_small, smem, L::bytes, bars, issue, work);
  if (brk) atomicOr(&red->breakdown, 1);
  if (!ok) atomicOr(&red->timeout, 1);
  last_block_control(ctl, red, g.no_control ? 0 : CK_SWEEP64);
}

// ---------------------------------------------------------------------------
// FP32 full sweep (mixed modes, precision phase).  Messages (P, eta) and
// totals in FP32; rhs_i = r_i / ||r|| (scaled in FP64 by the first sweep of
// an inner solve, then kept in FP32).  Records (P~_i, d_i = h~_i / P~_i) per
// node and the change against the previous sweep.  When the controller has
// set pending_freeze, the sweep freezes instead: it stores the coefficient
// c_ij = -A_ij / (P~_i - P_ji) at slot s of row i, 1/P~_i, and the first
// mean-only messages eta_ij = c_ij (h~_i - eta_ji).
// Staged per tile: (P, eta) in, A_ij, rev, and row pointers (light tiles) or
// local row ids (heavy tiles).  Per-row values are read straight from global
// memory by the thread that owns the row (coalesced).
// ---------------------------------------------------------------------------
template <int TSL>
struct Layout32 {
  static constexpr int TS = TSL, TR = kTileRowsBig;
  static constexpr uint32_t m = 0, a = m + region(TS, 8), rev = a + region(TS, 4),
                            lr = rev + region(TS, 4), rp = lr + region(TS, 2),
                            ro = rp + region(TR + 1, 4), bytes = ro + region(TR, 1);
};

template <class T, int TSL>
__global__ void __launch_bounds__(kTileBlock)
sweep32_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red) {
  using L = Layout32<TSL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ float2 tot[2][L::TR];   // heavy tiles: per-row sums, double-buffered
  __shared__ float2 nd[L::TR];       // heavy tiles: (A_ii, rhs_i) of the tile's rows
  __shared__ int cont_key[L::TS / 32];      // heavy tiles: row continuing into chunk c (-1: none)
  __shared__ float2 cont_sum[L::TS / 32];   //   and its partial sum over chunk c
  const int pm = ctl->par_m, pe = ctl->par_e, pmon = ctl->par_mon;
  const bool first = ctl->first != 0;
  const bool zin = first && !g.in_place;   // incoming messages known to be zero
  const bool freeze = ctl->pending_freeze != 0;
  const double inv_rn = ctl->inv_rn;
  const float2 *__restrict__ min = (pm ? B.m32[1] : B.m32[0]);
  float2 *__restrict__ mout = (pm ? B.m32[0] : B.m32[1]);
  T *__restrict__ eta_out = static_cast<T *>((pe ? B.e[0] : B.e[1]));
  const float2 *__restrict__ mon_prev = (pmon ? B.mon32[1] : B.mon32[0]);
  float2 *__restrict__ mon_out = (pmon ? B.mon32[0] : B.mon32[1]);
  const int NT = blockDim.x, tid = threadIdx.x;
  const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
  uint32_t mdd = 0, md = 0, mdP = 0, mP = 0;
  bool brk = false;
  for (int k = tid; k < 2 * L::TR; k += NT) (&tot[0][0])[k] = make_float2(0.f, 0.f);

  auto issue = [&](int32_t t, unsigned char *stage, uint32_t bar) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int64_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) { mbar_expect_tx(bar, 0); return; }
    const bool heavy = g.heavy_big[t] != 0;
    const uint32_t tx = (zin ? 0 : Seg<float2>::bytes(tb.s0, ns)) +
                        (heavy ? Seg<uint16_t>::bytes(tb.s0, ns)
                               : Seg<int32_t>::bytes(tb.r0, nr + 1) + Seg<uint8_t>::bytes(tb.r0, nr)) +
                        Seg<float>::bytes(tb.s0, ns) + Seg<int32_t>::bytes(tb.s0, ns);
    mbar_expect_tx(bar, tx);
    const uint32_t base = smem_u32(stage);
    if (!zin) Seg<float2>::copy(base + L::m, min, tb.s0, ns, bar, pol_keep);
    if (heavy) {
      Seg<uint16_t>::copy(base + L::lr, g.lrow_big, tb.s0, ns, bar, pol_stream);
    } else {
      Seg<int32_t>::copy(base + L::rp, g.rp, tb.r0, nr + 1, bar, pol_stream);
      Seg<uint8_t>::copy(base + L::ro, g.rord, tb.r0, nr, bar, pol_stream);
    }
    Seg<float>::copy(base + L::a, g.a32, tb.s0, ns, bar, pol_stream);
    Seg<int32_t>::copy(base + L::rev, g.rev, tb.s0, ns, bar, pol_stream);
  };

  // rhs_i = r_i / ||r||: scaled once (FP64) in the first sweep of an inner
  // solve, kept in FP32 for the rest of it.
  auto rhs_at = [&](int32_t i) {
    return first ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
  };
  auto node = [&](int32_t i, float TP, float Th, float rhs) {
    const float2 prev = first ? make_float2(0.f, 0.f) : mon_prev[i];
    const float di = Th / TP;
    mon_out[i] = make_float2(TP, di);
    mdd = fmax_bits(mdd, di - prev.y);
    md = fmax_bits(md, di);
    mdP = fmax_bits(mdP, TP - prev.x);
    mP = fmax_bits(mP, TP);
    if (freeze) B.invP32[i] = 1.0f / TP;
    if (first) B.rhs32[i] = rhs;
  };
  const float gam = g.no_damp ? 0.f : static_cast<float>(ctl->damping);
  auto emit = [&](int32_t s, float a, float2 m, int32_t dst, float TP, float Th) {
    const float d = TP - m.x;   // P_{i\j} = P~_i - P_ji
    brk |= !(d != 0.0f) || !isfinite(d);
    const float inv = 1.0f / d;
    // damping: blend the information with this message's previous value
    const float old_eta = (gam > 0.f && !zin) ? min[dst].y : 0.f;
    if (freeze) {
      const float c = -a * inv;
      B.c32[s] = c;
      float eta = c * (Th - m.y);
      if (gam > 0.f) eta = gam * old_eta + (1.f - gam) * eta;
      st_keep(eta_out + dst, eta, pol_keep);
    } else {
      float eta = -a * (Th - m.y) * inv;
      if (gam > 0.f) eta = gam * old_eta + (1.f - gam) * eta;
      st_keep(mout + dst, make_float2(-(a * a) * inv, eta), pol_keep);
    }
  };

  auto work = [&](int32_t t, unsigned char *stage, int st, bool got) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int32_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    // clear the other totals buffer for the next tile, whatever this tile's kind
    float2 *tc = tot[st], *tn = tot[st ^ 1];
    for (int32_t k = tid; k < L::TR; k += NT) tn[k] = make_float2(0.f, 0.f);
    if (ns > L::TS) {
      if (__syncthreads_or(!got)) return true;
      const int32_t i = tb.r0;
      float sP = 0.f, sH = 0.f;
      if (!zin)
        for (int32_t s = tb.s0 + tid; s < tb.s1; s += NT) {
          const float2 m = min[s];
          sP += m.x;
          sH += m.y;
        }
      sP = block_sum(sP);
      sH = block_sum(sH);
      const float rhs = rhs_at(i);
      const float TP = g.diag32[i] + sP, Th = rhs + sH;
      if (tid == 0) node(i, TP, Th, rhs);
      for (int32_t s = tb.s0 + tid; s < tb.s1; s += NT)
        emit(s, g.a32[s], zin ? make_float2(0.f, 0.f) : min[s], g.rev[s], TP, Th);
      return false;
    }
    const float2 *ms = Seg<float2>::at(stage + L::m, tb.s0);
    const float *as = Seg<float>::at(stage + L::a, tb.s0);
    const int32_t *rv = Seg<int32_t>::at(stage + L::rev, tb.s0);
    if (!g.heavy_big[t]) {
      // light tile: one thread per row does the sums, the node and the sends;
      // rows taken in the tile's degree order, so a warp's rows are alike
      const int32_t *rp = Seg<int32_t>::at(stage + L::rp, tb.r0);
      const uint8_t *ro = Seg<uint8_t>::at(stage + L::ro, tb.r0);
      if (__syncthreads_or(!got)) return true;
      for (int32_t q = tid; q < nr; q += NT) {
        const int32_t k = ro[q], i = tb.r0 + k;
        const float dgi = g.diag32[i], rhs = rhs_at(i);
        const int32_t rs = rp[k] - tb.s0, re = rp[k + 1] - tb.s0;
        float sP = 0.f, sH = 0.f;
        if (!zin)
          for (int32_t s = rs; s < re; ++s) {
            sP += ms[s].x;
            sH += ms[s].y;
          }
        const float TP = dgi + sP, Th = rhs + sH;
        node(i, TP, Th, rhs);
        for (int32_t s = rs; s < re; ++s)
          emit(tb.s0 + s, as[s], zin ? make_float2(0.f, 0.f) : ms[s], rv[s], TP, Th);
      }
      return false;
    }
    // heavy tile (a row of degree > kHeavyDegree): slot-parallel sums
    const uint16_t *lrow = Seg<uint16_t>::at(stage + L::lr, tb.s0);
    for (int32_t k = tid; k < nr; k += NT) nd[k] = make_float2(g.diag32[tb.r0 + k], rhs_at(tb.r0 + k));
    // Sums in a fixed order: within a 32-slot chunk by the segmented
    // shuffle sum; a row that starts in the chunk gets its total from that
    // head alone, and the partial of a row continuing from earlier chunks
    // is added afterwards by one thread, chunk by chunk.
    if (!zin) {
      for (int32_t base = tid & ~31; base < ns; base += NT) {
        const int32_t s = base + (tid & 31);
        const bool v = s < ns;
        const int key = v ? lrow[s] : kNoRow;
        bool head;
        const float2 sum = seg_sum(v ? ms[s] : make_float2(0.f, 0.f), key, head);
        if (head && v) {
          const bool cont = (s & 31) == 0 && s > 0 && lrow[s - 1] == key;
          if (cont) { cont_key[s >> 5] = key; cont_sum[s >> 5] = sum; }
          else tc[key] = sum;
        }
        if ((tid & 31) == 0 && !(v && s > 0 && lrow[s - 1] == key)) cont_key[base >> 5] = -1;
      }
    }
    if (__syncthreads_or(!got)) return true;
    if (!zin) {
      if (tid == 0)
        for (int32_t c = 1; 32 * c < ns; ++c)
          if (cont_key[c] >= 0) {
            tc[cont_key[c]].x += cont_sum[c].x;
            tc[cont_key[c]].y += cont_sum[c].y;
          }
      __syncthreads();
    }
    for (int32_t k = tid; k < nr; k += NT)
      node(tb.r0 + k, nd[k].x + tc[k].x, nd[k].y + tc[k].y, nd[k].y);
    for (int32_t s = tid; s < ns; s += NT) {
      const int k = lrow[s];
      emit(tb.s0 + s, as[s], zin ? make_float2(0.f, 0.f) : ms[s], rv[s], nd[k].x + tc[k].x,
           nd[k].y + tc[k].y);
    }
    return false;
  };

  const bool ok = run_tiles(g.ntiles_big, smem, L::bytes, bars, issue, work);
  if (brk) atomicOr(&red->breakdown, 1);
  if (!ok) atomicOr(&red->timeout, 1);
  block_max4(widen(mdd), widen(md), widen(mdP), widen(mP), &red->max_dx, &red->max_x,
             &red->max_dP, &red->max_P);
  last_block_control(ctl, red, g.no_control ? 0 : CK_SWEEP32);
}

// ---------------------------------------------------------------------------
// FP32 full sweep, in-place form (synchronous schedule, no damping).  The
// message j -> i of round t depends on the reverse message i -> j of round
// t - 1, and that one on the node totals of i at round t - 2 and on the
// message j -> i of round t - 2 -- the value slot s of row i already holds.
// So each slot recomputes the reverse message instead of receiving it:
//     P_ij  = -A_ij^2 / (P~_i^(t-2) - P_ji^(t-2)),
//     eta_ij = -A_ij (h~_i^(t-2) - eta_ji^(t-2)) / (P~_i^(t-2) - P_ji^(t-2)),
//     P_ji  = -A_ij^2 / (P~_j^(t-1) - P_ij),
//     eta_ji = -A_ij (h~_j^(t-1) - eta_ij) / (P~_j^(t-1) - P_ij)
// (Alg. 2 applied twice, with the same expressions as the scatter form), and
// overwrites slot s with the round-t message.  The round is exactly the
// synchronous round of Section III-C; the only random access left is the
// gather of the neighbour's totals (P~_j, h~_j)^(t-1) from an n-entry table,
// where the scatter form stores every message at a random slot.
// Buffers (par = par_m): m32[par ^ 1] holds round t - 2 and receives round t
// in place; tot32[par] holds the totals of round t - 1 (gathered);
// tot32[par ^ 1] holds this row's totals of round t - 2 and receives round
// t (only the row's own lane group touches them).  Round 1 starts from zero
// messages, so its reverse messages are zero and the totals of round 0 are
// (A_jj, rhs_j); round 2 reads zero round-0 messages.
// Freeze: c_ij = -A_ij / (P~_i - P_ji) from this round's totals and
// messages, 1/P~_i, and the mean messages of round t + 1,
// eta_ij = c_ij (h~_i - eta_ji), sent to the receivers' slots as the scatter
// form's freeze sends them (once per solve), so that the next mean sweep
// reports round t + 1.
// G lanes per row; rows taken grid-stride by groups.
// ---------------------------------------------------------------------------
// One message of Alg. 2 from the sender's totals (Tx, Ty) and the reverse
// message (mx, my): (-a^2 / (Tx - mx), -a (Ty - my) / (Tx - mx)).  Every step
// is an explicitly rounded operation, so no contraction into a fused
// multiply-add can make the copy a sender recomputes differ from the copy the
// receiver stored.  The in-place form needs the two bit for bit: a difference
// would travel back and forth along the edge with gain (A_ij^2 / (P_{i\j}
// P_{j\i}))^2 per two rounds, which exceeds one on matrices that are not
// walk-summable (measured: an indefinite tree of 300 nodes diverged).
__device__ __forceinline__ float2 message32(float a, float Tx, float Ty, float mx, float my, bool &brk) {
  const float d = __fsub_rn(Tx, mx);
  brk |= !(d != 0.0f) || !isfinite(d);
  const float inv = __fdiv_rn(1.0f, d);
  return make_float2(__fmul_rn(-__fmul_rn(a, a), inv), __fmul_rn(__fmul_rn(-a, __fsub_rn(Ty, my)), inv));
}

template <class T, int G>
__global__ void __launch_bounds__(kBlock, 6)
pull32_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red) {
  const int pm = ctl->par_m, pe = ctl->par_e, pmon = ctl->par_mon;
  const bool first = ctl->first != 0;
  const bool second = !first && ctl->second != 0;   // round-0 messages are zero
  const bool freeze = ctl->pending_freeze != 0;
  const double inv_rn = ctl->inv_rn;
  float2 *__restrict__ msg = pm ? B.m32[0] : B.m32[1];
  const float2 *__restrict__ tot_prev = pm ? B.tot32[1] : B.tot32[0];
  float2 *__restrict__ tot_own = pm ? B.tot32[0] : B.tot32[1];
  T *__restrict__ eta_out = static_cast<T *>((pe ? B.e[0] : B.e[1]));
  const float2 *__restrict__ mon_prev = (pmon ? B.mon32[1] : B.mon32[0]);
  float2 *__restrict__ mon_out = (pmon ? B.mon32[0] : B.mon32[1]);
  const int gl = threadIdx.x % G;
  uint32_t mdd = 0, md = 0, mdP = 0, mP = 0;
  bool brk = false;

  // rows of the whole grid, G lanes each; every lane of a warp runs the
  // same number of iterations (the group sums shuffle across the warp)
  const int64_t groups = static_cast<int64_t>(gridDim.x) * (blockDim.x / G);
  const int64_t grp0 = static_cast<int64_t>(blockIdx.x) * (blockDim.x / G) + threadIdx.x / G;
  for (int64_t ib = grp0 - threadIdx.x % 32 / G; ib < g.n; ib += groups) {
    const int64_t i = ib + threadIdx.x % 32 / G;
    const bool valid = i < g.n;
    int32_t rs = 0, re = 0;
    float dgi = 0.f, rhs = 0.f, TP2 = 0.f, Th2 = 0.f;
    if (valid) {
      rs = g.rp[i];
      re = g.rp[i + 1];
      dgi = g.diag32[i];
      rhs = first ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
      if (second) { TP2 = dgi; Th2 = rhs; }
      else if (!first) { const float2 t2 = tot_own[i]; TP2 = t2.x; Th2 = t2.y; }
    }
    float sP = 0.f, sH = 0.f;
    for (int32_t s = rs + gl; s < re; s += G) {
      const int32_t j = g.col[s];
      const float a = g.a32[s];
      float2 Tj;
      if (first) Tj = make_float2(g.diag32[j], static_cast<float>(B.r64[j] * inv_rn));
      else Tj = tot_prev[j];
      // the reverse message i -> j of round t - 1 (zero in round 1), exactly
      // as the receiver j computed and stored it, then the message j -> i
      float2 r = make_float2(0.f, 0.f);
      if (!first) {
        const float2 m = second ? make_float2(0.f, 0.f) : msg[s];
        r = message32(a, TP2, Th2, m.x, m.y, brk);
      }
      const float2 nw = message32(a, Tj.x, Tj.y, r.x, r.y, brk);
      msg[s] = nw;
      sP += nw.x;
      sH += nw.y;
    }
    sP = group_sum<G>(sP);
    sH = group_sum<G>(sH);
    if (!valid) continue;
    const float TP = dgi + sP, Th = rhs + sH;
    if (gl == 0) {
      tot_own[i] = make_float2(TP, Th);
      const float2 prev = first ? make_float2(0.f, 0.f) : mon_prev[i];
      const float di = Th / TP;
      mon_out[i] = make_float2(TP, di);
      mdd = fmax_bits(mdd, di - prev.y);
      md = fmax_bits(md, di);
      mdP = fmax_bits(mdP, TP - prev.x);
      mP = fmax_bits(mP, TP);
      if (freeze) B.invP32[i] = 1.0f / TP;
      if (first) B.rhs32[i] = rhs;
    }
    if (freeze)
      for (int32_t s = rs + gl; s < re; s += G) {
        const float2 m = msg[s];      // written above by this thread
        const float d = TP - m.x;
        brk |= !(d != 0.0f) || !isfinite(d);
        const float c = -g.a32[s] * (1.0f / d);
        B.c32[s] = c;
        store_eta(eta_out + g.rev[s], c * (Th - m.y));
      }
  }
  if (brk) atomicOr(&red->breakdown, 1);
  block_max4(widen(mdd), widen(md), widen(mdP), widen(mP), &red->max_dx, &red->max_x,
             &red->max_dP, &red->max_P);
  last_block_control(ctl, red, CK_SWEEP32);
}

// ---------------------------------------------------------------------------
// Mean-only sweep with frozen precisions (storage T = float or bf16, FP32
// arithmetic): eta_ij = c_ij (h~_i - eta_ji), h~_i = r_i/||r|| + sum_k eta_ki,
// d_i = h~_i / P~_i.  Records d_i and its change.
// Staged per tile: eta in, c, rev, and row pointers or local row ids.
// ---------------------------------------------------------------------------
template <class T, int TSL>
struct LayoutMean {
  static constexpr int TS = TSL, TR = kTileRowsBig;
  static constexpr uint32_t e = 0, c = e + region(TS, sizeof(T)), rev = c + region(TS, 4),
                            lr = rev + region(TS, 4), rp = lr + region(TS, 2),
                            ro = rp + region(TR + 1, 4), bytes = ro + region(TR, 1);
};

template <class T, int TSL>
__global__ void __launch_bounds__(kTileBlock)
mean_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red) {
  using L = LayoutMean<T, TSL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ float tot[2][L::TR];    // heavy tiles: per-row sums, double-buffered
  __shared__ float rhs_s[L::TR];     // heavy tiles: rhs of the tile's rows
  __shared__ int cont_key[L::TS / 32];     // heavy tiles: row continuing into chunk c (-1: none)
  __shared__ float cont_sum[L::TS / 32];   //   and its partial sum over chunk c
  const int pe = ctl->par_e, pmon = ctl->par_mon;
  const bool first = ctl->first != 0;
  const bool zin = first && !g.in_place;   // incoming messages known to be zero
  const double inv_rn = ctl->inv_rn;
  const T *__restrict__ ein = static_cast<const T *>((pe ? B.e[1] : B.e[0]));
  T *__restrict__ eout = static_cast<T *>((pe ? B.e[0] : B.e[1]));
  const float2 *__restrict__ mon_prev = (pmon ? B.mon32[1] : B.mon32[0]);
  float2 *__restrict__ mon_out = (pmon ? B.mon32[0] : B.mon32[1]);
  const int NT = blockDim.x, tid = threadIdx.x;
  const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
  uint32_t mdd = 0, md = 0;
  for (int k = tid; k < 2 * L::TR; k += NT) (&tot[0][0])[k] = 0.f;

  auto issue = [&](int32_t t, unsigned char *stage, uint32_t bar) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int64_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) { mbar_expect_tx(bar, 0); return; }
    const bool heavy = g.heavy_big[t] != 0;
    const uint32_t tx = (zin ? 0 : Seg<T>::bytes(tb.s0, ns)) +
                        (heavy ? Seg<uint16_t>::bytes(tb.s0, ns)
                               : Seg<int32_t>::bytes(tb.r0, nr + 1) + Seg<uint8_t>::bytes(tb.r0, nr)) +
                        Seg<float>::bytes(tb.s0, ns) + Seg<int32_t>::bytes(tb.s0, ns);
    mbar_expect_tx(bar, tx);
    const uint32_t base = smem_u32(stage);
    if (!zin) Seg<T>::copy(base + L::e, ein, tb.s0, ns, bar, pol_keep);
    if (heavy) {
      Seg<uint16_t>::copy(base + L::lr, g.lrow_big, tb.s0, ns, bar, pol_stream);
    } else {
      Seg<int32_t>::copy(base + L::rp, g.rp, tb.r0, nr + 1, bar, pol_stream);
      Seg<uint8_t>::copy(base + L::ro, g.rord, tb.r0, nr, bar, pol_stream);
    }
    Seg<float>::copy(base + L::c, B.c32, tb.s0, ns, bar, pol_stream);
    Seg<int32_t>::copy(base + L::rev, g.rev, tb.s0, ns, bar, pol_stream);
  };

  auto rhs_at = [&](int32_t i) {
    return first ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
  };
  const float gam = g.no_damp ? 0.f : static_cast<float>(ctl->damping);
  // eta_ij sent to slot dst: damped with its previous value when gamma > 0
  auto send = [&](int32_t dst, float v) {
    if (gam > 0.f) v = gam * (zin ? 0.f : ld_eta(ein + dst)) + (1.f - gam) * v;
    st_keep(eout + dst, v, pol_keep);
  };
  auto node = [&](int32_t i, float Th, float rhs) {
    const float prev = first ? 0.f : mon_prev[i].y;
    const float di = Th * B.invP32[i];
    mon_out[i] = make_float2(0.f, di);
    mdd = fmax_bits(mdd, di - prev);
    md = fmax_bits(md, di);
    if (first) B.rhs32[i] = rhs;
  };

  auto work = [&](int32_t t, unsigned char *stage, int st, bool got) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int32_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    // clear the other totals buffer for the next tile, whatever this tile's kind
    float *tc = tot[st], *tn = tot[st ^ 1];
    for (int32_t k = tid; k < L::TR; k += NT) tn[k] = 0.f;
    if (ns > L::TS) {
      if (__syncthreads_or(!got)) return true;
      const int32_t i = tb.r0;
      float sH = 0.f;
      if (!zin)
        for (int32_t s = tb.s0 + tid; s < tb.s1; s += NT) sH += ld_eta(ein + s);
      sH = block_sum(sH);
      const float rhs = rhs_at(i), Th = rhs + sH;
      if (tid == 0) node(i, Th, rhs);
      for (int32_t s = tb.s0 + tid; s < tb.s1; s += NT) {
        const float e = zin ? 0.f : ld_eta(ein + s);
        send(g.rev[s], B.c32[s] * (Th - e));
      }
      return false;
    }
    const T *es = Seg<T>::at(stage + L::e, tb.s0);
    const float *cs = Seg<float>::at(stage + L::c, tb.s0);
    const int32_t *rv = Seg<int32_t>::at(stage + L::rev, tb.s0);
    if (!g.heavy_big[t]) {
      // light tile: one thread per row does the sum, the node and the sends;
      // rows taken in the tile's degree order, so a warp's rows are alike
      const int32_t *rp = Seg<int32_t>::at(stage + L::rp, tb.r0);
      const uint8_t *ro = Seg<uint8_t>::at(stage + L::ro, tb.r0);
      if (__syncthreads_or(!got)) return true;
      for (int32_t q = tid; q < nr; q += NT) {
        const int32_t k = ro[q], i = tb.r0 + k;
        const float rhs = rhs_at(i);
        const int32_t rs = rp[k] - tb.s0, re = rp[k + 1] - tb.s0;
        float sH = 0.f;
        if (!zin)
          for (int32_t s = rs; s < re; ++s) sH += ld_eta(es + s);
        const float Th = rhs + sH;
        node(i, Th, rhs);
        if (zin)
          for (int32_t s = rs; s < re; ++s) send(rv[s], cs[s] * Th);
        else
          for (int32_t s = rs; s < re; ++s)
            send(rv[s], cs[s] * (Th - ld_eta(es + s)));
      }
      return false;
    }
    // heavy tile (a row of degree > kHeavyDegree): slot-parallel sums
    const uint16_t *lrow = Seg<uint16_t>::at(stage + L::lr, tb.s0);
    for (int32_t k = tid; k < nr; k += NT) rhs_s[k] = rhs_at(tb.r0 + k);
    // Sums in a fixed order (as in sweep32_kernel): chunk-wise segmented
    // sums, then the partials of rows continuing across chunks in chunk order.
    if (!zin) {
      for (int32_t base = tid & ~31; base < ns; base += NT) {
        const int32_t s = base + (tid & 31);
        const bool v = s < ns;
        const int key = v ? lrow[s] : kNoRow;
        bool head;
        const float sum = seg_sum(v ? ld_eta(es + s) : 0.f, key, head);
        if (head && v) {
          const bool cont = (s & 31) == 0 && s > 0 && lrow[s - 1] == key;
          if (cont) { cont_key[s >> 5] = key; cont_sum[s >> 5] = sum; }
          else tc[key] = sum;
        }
        if ((tid & 31) == 0 && !(v && s > 0 && lrow[s - 1] == key)) cont_key[base >> 5] = -1;
      }
    }
    if (__syncthreads_or(!got)) return true;
    if (!zin) {
      if (tid == 0)
        for (int32_t c = 1; 32 * c < ns; ++c)
          if (cont_key[c] >= 0) tc[cont_key[c]] += cont_sum[c];
      __syncthreads();
    }
    for (int32_t k = tid; k < nr; k += NT) node(tb.r0 + k, rhs_s[k] + tc[k], rhs_s[k]);
    for (int32_t s = tid; s < ns; s += NT) {
      const int k = lrow[s];
      const float e = zin ? 0.f : ld_eta(es + s);
      send(rv[s], cs[s] * (rhs_s[k] + tc[k] - e));
    }
    return false;
  };

  const bool ok = run_tiles(g.ntiles_big, smem, L::bytes, bars, issue, work);
  if (!ok) atomicOr(&red->timeout, 1);
  block_max4(widen(mdd), widen(md), 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
  last_block_control(ctl, red, g.no_control ? 0 : CK_MEAN);
}

// Aitken's Delta^2 per node on the last three tentative means in the ring
// (Section IV-A, convergence acceleration): y = x0 - (x1 - x0)^2 / (x2 - 2 x1
// + x0), or the latest mean x2 where the second difference is at rounding
// level (|x2 - 2 x1 + x0| <= 64 eps max|x_k|) or fewer than three means exist.
// out = nullptr: the solve's x (read from the control block, so a recorded
// graph serves every solve).
__global__ void __launch_bounds__(kBlock) aitken_kernel(int32_t n, const Ctl *ctl, double *out) {
  const int nw = ctl->nw;
  if (nw < 1) return;
  double *__restrict__ dst = out ? out : ctl->x;
  const double *__restrict__ x2 = ctl->ring[(nw - 1) % 3];
  const double *__restrict__ x1 = ctl->ring[(nw + 1) % 3];   // (nw - 2) mod 3
  const double *__restrict__ x0 = ctl->ring[nw % 3];         // (nw - 3) mod 3
  const bool have3 = nw >= 3;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double c2 = x2[i];
    double y = c2;
    if (have3) {
      const double c0 = x0[i], c1 = x1[i];
      const double d1 = c1 - c0, den = (c2 - c1) - d1;
      const double scale = fmax(fmax(fabs(c0), fabs(c1)), fabs(c2));
      if (fabs(den) > 64.0 * DBL_EPSILON * scale) y = c0 - d1 * d1 / den;
    }
    dst[i] = y;
  }
}

// x_i += ||r|| d_i (FP64), d_i from the latest monitor.  With Aitken on a
// mixed grid solve (ait_use), d_i is extrapolated from the inner solve's last
// three records y0, y1, y2 at spacing 2^level (Section IV-A):
//     d_i = y2 - (y2 - y1)^2 / (y2 - 2 y1 + y0),
// except where the second difference is at FP32 rounding level
// (|y2 - 2 y1 + y0| <= 64 eps max |d|), which keeps the latest d_i.
// Records of an inner solve's means for Aitken on mixed solves (CSR forms;
// the grid mean sweep records its own).  The controller runs the mean sweeps
// 64, 128, ... of an inner solve as phases that add this kernel behind the
// sweep and its control step, so ctl->k counts the sweep and par_mon names
// the monitor buffer it wrote.  Each node's mean d_i goes to the ring of
// every spacing 2^j (j = 6..12) that divides k, at slot (k / 2^j) mod 3.
__global__ void __launch_bounds__(kBlock) ait_record_kernel(int32_t n, Buffers B, const Ctl *ctl) {
  const int k = ctl->k;
  if (!ctl->ait_mixed || k <= 0 || (k & ((1 << kAitMinLevel) - 1)) != 0) return;
  const float2 *__restrict__ mon = ctl->par_mon ? B.mon32[1] : B.mon32[0];
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float d = mon[i].y;
    for (int j = 0; j < kAitLevels; ++j) {
      const int lvl = kAitMinLevel + j;
      if (k & ((1 << lvl) - 1)) break;
      B.ait32[(static_cast<int64_t>(j) * 3 + (k >> lvl) % 3) * n + i] = d;
    }
  }
}

__global__ void __launch_bounds__(kBlock) refine_update_kernel(int32_t n, Buffers B, Ctl *ctl) {
  double *x = ctl->x;
  const double rn = ctl->rn;
  const float2 *mon = (ctl->par_mon ? B.mon32[1] : B.mon32[0]);
  const bool ait = ctl->ait_use != 0;
  const float *R = nullptr;
  int64_t o0 = 0, o1 = 0, o2 = 0;
  double floor_d2 = 0.0;
  if (ait) {
    const int m = ctl->ait_m;
    R = B.ait32 + static_cast<int64_t>(ctl->ait_level) * 3 * n;
    o2 = static_cast<int64_t>(m % 3) * n;
    o1 = static_cast<int64_t>((m - 1) % 3) * n;
    o0 = static_cast<int64_t>((m - 2) % 3) * n;
    floor_d2 = 64.0 * FLT_EPSILON * ctl->ait_md;
  }
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double di = static_cast<double>(mon[i].y);
    if (ait) {
      const double y0 = R[o0 + i], y1 = R[o1 + i], y2 = R[o2 + i];
      const double d2 = y2 - 2.0 * y1 + y0;
      if (fabs(d2) > floor_d2) di = y2 - (y2 - y1) * (y2 - y1) / d2;
    }
    x[i] += di * rn;
  }
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x with its infinity norm (a CSR SpMV).  Staged per
// tile: A_ij, col, row pointers, A_ii.  Phase 1 (slot-parallel): the products
// A_ij x_j, with x_j gathered from global memory, overwrite A_ij in shared
// memory.  Phase 2: one thread per row sums its products (one FP64 add per
// slot) and forms r_i.
// ---------------------------------------------------------------------------
template <int TSL>
struct LayoutRes {
  static constexpr int TS = TSL, TR = kTileRowsBig;
  static constexpr uint32_t a = 0, col = a + region(TS, 8), rp = col + region(TS, 4),
                            dg = rp + region(TR + 1, 4), ro = dg + region(TR, 8),
                            bytes = ro + region(TR, 1);
};

template <int TSL>
__global__ void __launch_bounds__(kTileBlock)
residual64_kernel(GraphView g, double *__restrict__ r_out, Ctl *ctl, DevScalars *red, int kind) {
  using L = LayoutRes<TSL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  const double *__restrict__ b = ctl->b;
  const double *__restrict__ x = ctl->x;
  const int NT = blockDim.x, tid = threadIdx.x;
  const uint64_t pol_stream = policy_evict_first();
  unsigned long long mr = 0, mrel = 0;

  auto issue = [&](int32_t t, unsigned char *stage, uint32_t bar) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int64_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) { mbar_expect_tx(bar, 0); return; }
    const uint32_t tx = Seg<double>::bytes(tb.s0, ns) + Seg<int32_t>::bytes(tb.s0, ns) +
                        Seg<int32_t>::bytes(tb.r0, nr + 1) + Seg<double>::bytes(tb.r0, nr) +
                        Seg<uint8_t>::bytes(tb.r0, nr);
    mbar_expect_tx(bar, tx);
    const uint32_t base = smem_u32(stage);
    Seg<double>::copy(base + L::a, g.a64, tb.s0, ns, bar, pol_stream);
    Seg<int32_t>::copy(base + L::col, g.col, tb.s0, ns, bar, pol_stream);
    Seg<int32_t>::copy(base + L::rp, g.rp, tb.r0, nr + 1, bar, pol_stream);
    Seg<double>::copy(base + L::dg, g.diag64, tb.r0, nr, bar, pol_stream);
    Seg<uint8_t>::copy(base + L::ro, g.rord, tb.r0, nr, bar, pol_stream);
  };

  auto node = [&](int32_t i, double dgi, double acc) {
    const double ri = b[i] - (dgi * x[i] + acc);
    if (r_out) r_out[i] = ri;
    mr = umax(mr, bits(fabs(ri)));
    if (g.sys_bmax) {
      // batched: residual relative to this row's own system
      const double bs = dv(g.sys_bmax[g.sys_of_row[i]]);
      mrel = umax(mrel, bits(bs > 0.0 ? fabs(ri) / bs : (ri == 0.0 ? 0.0 : INFINITY)));
    }
  };

  auto work = [&](int32_t t, unsigned char *stage, int, bool got) {
    const TileBounds tb = tile_at(g.tiles_big, t);
    const int32_t ns = tb.s1 - tb.s0, nr = tb.r1 - tb.r0;
    if (ns > L::TS) {
      if (__syncthreads_or(!got)) return true;
      double acc = 0.0;
      for (int32_t s = tb.s0 + tid; s < tb.s1; s += NT) acc += g.a64[s] * x[g.col[s]];
      acc = block_sum(acc);
      if (tid == 0) node(tb.r0, g.diag64[tb.r0], acc);
      return false;
    }
    double *as = Seg<double>::at(stage + L::a, tb.s0);
    const int32_t *cs = Seg<int32_t>::at(stage + L::col, tb.s0);
    const int32_t *rp = Seg<int32_t>::at(stage + L::rp, tb.r0);
    const double *dg = Seg<double>::at(stage + L::dg, tb.r0);
    const uint8_t *ro = Seg<uint8_t>::at(stage + L::ro, tb.r0);
    if (!g.heavy_big[t]) {
      // light tile: one thread per row (in the tile's degree order), gathers
      // unrolled for memory parallelism
      if (__syncthreads_or(!got)) return true;
      for (int32_t q = tid; q < nr; q += NT) {
        const int32_t k = ro[q];
        const int32_t rs = rp[k] - tb.s0, re = rp[k + 1] - tb.s0;
        double acc = 0.0;
        int32_t s = rs;
        for (; s + 4 <= re; s += 4) {
          const double x0 = x[cs[s]], x1 = x[cs[s + 1]], x2 = x[cs[s + 2]], x3 = x[cs[s + 3]];
          acc += as[s] * x0;
          acc += as[s + 1] * x1;
          acc += as[s + 2] * x2;
          acc += as[s + 3] * x3;
        }
        for (; s < re; ++s) acc += as[s] * x[cs[s]];
        node(tb.r0 + k, dg[k], acc);
      }
      return false;
    }
    // heavy tile: slot-parallel products, then one warp per row sums them
    if (got)
      for (int32_t s = tid; s < ns; s += NT) as[s] *= x[cs[s]];
    if (__syncthreads_or(!got)) return true;
    const int lane = tid & 31, nw = NT >> 5;
    for (int32_t k = tid >> 5; k < nr; k += nw) {
      double acc = 0.0;
      for (int32_t s = rp[k] - tb.s0 + lane; s < rp[k + 1] - tb.s0; s += 32) acc += as[s];
      acc = group_sum<32>(acc);
      if (lane == 0) node(tb.r0 + k, dg[k], acc);
    }
    return false;
  };

  const bool ok = run_tiles(g.ntiles_big, smem, L::bytes, bars, issue, work);
  if (!ok) atomicOr(&red->timeout, 1);
  block_max4(mr, mrel, 0, 0, &red->max_r, &red->max_rrel, nullptr, nullptr);
  last_block_control(ctl, red, kind);
}

// ---------------------------------------------------------------------------
// K right-hand sides at once (frozen precisions, FP32 mean messages, FP64
// refinement).  Mean messages are stored column-interleaved: message k of
// slot s at s * K + k, so the K messages of a slot are one contiguous run.
// One warp per row; lane l handles columns l, l + 32, ... (NC per lane), so
// every message read and every reverse-slot write moves K contiguous values.
// ---------------------------------------------------------------------------
// Per-column maxima of a block, then one atomicMax per column and block.
template <int NC>
__device__ void column_max_commit(const unsigned long long (&m)[NC], unsigned long long *dst,
                                  int K, unsigned long long *sm) {
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < K; k += blockDim.x) sm[k] = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int c = lane + 32 * j;
    if (c < K && m[j]) atomicMax(&sm[c], m[j]);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    if (sm[k]) atomicMax(&dst[k], sm[k]);
}

// X = 0, R = B and the per-column max |B|.
template <int NC>
__global__ void __launch_bounds__(kBlock)
init_multi_kernel(int32_t n, Buffers B, Ctl *ctl, DevScalars *red, int K) {
  __shared__ unsigned long long sm[32 * NC];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const double *Bm = ctl->Bm;
  double *X = ctl->Xm;
  unsigned long long m[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) m[j] = 0;
  for (int64_t i = warp; i < n; i += nwarps) {
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = lane + 32 * j;
      if (c >= K) continue;
      const int64_t idx = i * K + c;
      const double bv = Bm[idx];
      X[idx] = 0.0;
      B.rK[idx] = bv;
      m[j] = umax(m[j], bits(fabs(bv)));
    }
  }
  column_max_commit<NC>(m, ctl->cols.bmax, K, sm);
  last_block_control(ctl, red, CK_INITK);
}

// eta_ij^(k) = c_ij (h~_i^(k) - eta_ji^(k)),  h~_i^(k) = r_i^(k)/||r^(k)|| + sum eta_ki^(k)
template <int NC>
__global__ void __launch_bounds__(kBlock)
mean_multi_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red, int K) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int pe = ctl->par_e;
  const bool first = ctl->first != 0;
  // messages known to be zero (skip reading them): the first sweep of a
  // synchronous inner solve; an in-place colour pass reads its zeroed buffer
  const bool zin = first && !g.in_place;
  const float *__restrict__ ein = pe ? B.eK[1] : B.eK[0];
  float *__restrict__ eout = pe ? B.eK[0] : B.eK[1];
  const float gam = g.no_damp ? 0.f : static_cast<float>(ctl->damping);
  double irn[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int c = lane + 32 * j;
    irn[j] = (first && c < K) ? ctl->cols.inv_rn[c] : 0.0;
  }
  uint32_t mdd = 0, md = 0;
  for (int64_t i = g.row0 + warp; i < g.row1; i += nwarps) {
    const int32_t rs = g.rp[i], re = g.rp[i + 1];
    float th[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = lane + 32 * j;
      th[j] = 0.f;
      if (c >= K) continue;
      const int64_t idx = i * K + c;
      if (first) {
        th[j] = static_cast<float>(B.rK[idx] * irn[j]);
        B.rhsK[idx] = th[j];
      } else {
        th[j] = B.rhsK[idx];
      }
    }
    if (!zin) {
      // four slots' messages in flight per lane before they are added
      int32_t s = rs;
      for (; s + 4 <= re; s += 4) {
        float v[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            const int c = lane + 32 * j;
            v[u][j] = c < K ? ein[static_cast<int64_t>(s + u) * K + c] : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < NC; ++j) th[j] += v[u][j];
      }
      for (; s < re; ++s) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int c = lane + 32 * j;
          if (c < K) th[j] += ein[static_cast<int64_t>(s) * K + c];
        }
      }
    }
    const float ip = B.invP32[i];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = lane + 32 * j;
      if (c >= K) continue;
      const int64_t idx = i * K + c;
      const float d = th[j] * ip;
      const float prev = first ? 0.f : B.dK[idx];
      B.dK[idx] = d;
      mdd = fmax_bits(mdd, d - prev);
      md = fmax_bits(md, d);
    }
    int32_t s = rs;
    for (; s + 4 <= re; s += 4) {
      float cs[4], v[4][NC];
      int64_t dst[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cs[u] = B.c32[s + u];
        dst[u] = static_cast<int64_t>(g.rev[s + u]) * K;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int c = lane + 32 * j;
          v[u][j] = (zin || c >= K) ? 0.f : ein[static_cast<int64_t>(s + u) * K + c];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int c = lane + 32 * j;
          if (c >= K) continue;
          float out = cs[u] * (th[j] - v[u][j]);
          if (gam > 0.f) out = gam * (zin ? 0.f : ein[dst[u] + c]) + (1.f - gam) * out;
          eout[dst[u] + c] = out;
        }
    }
    for (; s < re; ++s) {
      const float cs = B.c32[s];
      const int64_t dst = static_cast<int64_t>(g.rev[s]) * K;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int c = lane + 32 * j;
        if (c >= K) continue;
        const float e = zin ? 0.f : ein[static_cast<int64_t>(s) * K + c];
        float out = cs * (th[j] - e);
        if (gam > 0.f) out = gam * (zin ? 0.f : ein[dst + c]) + (1.f - gam) * out;
        eout[dst + c] = out;
      }
    }
  }
  block_max4(widen(mdd), widen(md), 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
  last_block_control(ctl, red, g.no_control ? 0 : CK_MEANK);
}

// X += ||r_k|| D (FP64).
__global__ void __launch_bounds__(kBlock) refine_multi_update_kernel(int64_t total, Buffers B,
                                                                     Ctl *ctl, int K) {
  double *X = ctl->Xm;
  const double *rn = ctl->cols.rn;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x)
    X[idx] += static_cast<double>(B.dK[idx]) * rn[idx % K];
}

// R = B - A X (FP64) with per-column max |R|.
template <int NC>
__global__ void __launch_bounds__(kBlock)
residual_multi_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red, int K) {
  __shared__ unsigned long long sm[32 * NC];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const double *__restrict__ Bm = ctl->Bm;
  const double *__restrict__ X = ctl->Xm;
  unsigned long long m[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) m[j] = 0;
  for (int64_t i = warp; i < g.n; i += nwarps) {
    const int32_t rs = g.rp[i], re = g.rp[i + 1];
    double acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.0;
    int32_t s = rs;
    for (; s + 2 <= re; s += 2) {
      const double a0 = g.a64[s], a1 = g.a64[s + 1];
      const int64_t x0 = static_cast<int64_t>(g.col[s]) * K, x1 = static_cast<int64_t>(g.col[s + 1]) * K;
      double v0[NC], v1[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int c = lane + 32 * j;
        v0[j] = c < K ? X[x0 + c] : 0.0;
        v1[j] = c < K ? X[x1 + c] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] = fma(a1, v1[j], fma(a0, v0[j], acc[j]));
    }
    for (; s < re; ++s) {
      const double a = g.a64[s];
      const int64_t xc = static_cast<int64_t>(g.col[s]) * K;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int c = lane + 32 * j;
        if (c < K) acc[j] = fma(a, X[xc + c], acc[j]);
      }
    }
    const double dg = g.diag64[i];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = lane + 32 * j;
      if (c >= K) continue;
      const int64_t idx = i * K + c;
      const double r = Bm[idx] - (dg * X[idx] + acc[j]);
      B.rK[idx] = r;
      m[j] = umax(m[j], bits(fabs(r)));
    }
  }
  column_max_commit<NC>(m, ctl->cols.rmax, K, sm);
  last_block_control(ctl, red, CK_REFINEK);
}

// ---------------------------------------------------------------------------
// Section VII least-squares batches: right-hand side [0_K; y_s] of every
// augmented system, and extraction of x^_s (the first K_s unknowns).
// ---------------------------------------------------------------------------
__global__ void lsq_rhs_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                               const int64_t *__restrict__ aug_off, const int32_t *__restrict__ K,
                               const int64_t *__restrict__ y_off, const double *__restrict__ y,
                               double *__restrict__ rhs) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t sy = sys_of_row[i];
    const int64_t local = i - aug_off[sy];
    rhs[i] = local < K[sy] ? 0.0 : y[y_off[sy] + (local - K[sy])];
  }
}

__global__ void lsq_extract_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                                   const int64_t *__restrict__ aug_off,
                                   const int32_t *__restrict__ K, const int64_t *__restrict__ x_off,
                                   const double *__restrict__ x_aug, double *__restrict__ xhat) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t sy = sys_of_row[i];
    const int64_t local = i - aug_off[sy];
    if (local < K[sy]) xhat[x_off[sy] + local] = x_aug[i];
  }
}

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int flat_grid(int64_t n) {
  const int64_t need = (n + kBlock - 1) / kBlock;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, num_sms() * 8)));
}

// Blocks per SM of a tiled kernel with its two-stage shared memory; the
// dynamic shared-memory limit is raised once per kernel.
std::mutex g_occ_mu;
std::unordered_map<const void *, int> g_occ;

template <class K>
int resident_blocks(K kernel, size_t smem, int threads) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto it = g_occ.find(reinterpret_cast<const void *>(kernel));
  if (it != g_occ.end()) return it->second;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, threads, smem);
  bps = std::max(bps, 1);
  g_occ[reinterpret_cast<const void *>(kernel)] = bps;
  return bps;
}

// Persistent grid: one wave of resident CTAs (a multiple of the SM count),
// or fewer when there are fewer tiles.
template <class K>
int tile_grid(K kernel, size_t smem, int32_t ntiles, int threads) {
  const int64_t cap = static_cast<int64_t>(num_sms()) * resident_blocks(kernel, smem, threads);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ntiles, cap)));
}

template <class K, class... Args>
void launch_tiled(K kernel, size_t smem, int32_t ntiles, int threads, cudaStream_t st,
                  Args... args) {
  kernel<<<tile_grid(kernel, smem, ntiles, threads), threads, smem, st>>>(args...);
}

template <int G>
void launch64(const GraphView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  launch_tiled(sweep64_kernel<G>, 2 * Layout64::bytes, v.ntiles_small, kBlock, st, v, B, ctl, red);
}

// The FP32 sweeps and the residual come in two shared-memory sizes: tiles of
// at most 1024 slots, or at most 512 (half the staging, twice the resident
// CTAs).  The row tiles' slot limit picks the variant.
#define GABP_TS_DISPATCH(g, ...)                                     \
  do {                                                               \
    if ((g).tile_slots > 0 && (g).tile_slots <= 512) { constexpr int TSZ = 512; __VA_ARGS__; } \
    else { constexpr int TSZ = kTileSlotsBig; __VA_ARGS__; }         \
  } while (0)

int launch_residual(const Graph &g, cudaStream_t st, double *r_out, Ctl *ctl, DevScalars *red,
                    int kind) {
  GABP_TS_DISPATCH(g, launch_tiled(residual64_kernel<TSZ>, 2 * LayoutRes<TSZ>::bytes, g.ntiles_big,
                                   kTileBlock, st, g.view(), r_out, ctl, red, kind));
  return 1;
}

template <int G>
void prepare_group() {
  resident_blocks(sweep64_kernel<G>, 2 * Layout64::bytes, kBlock);
}

// In-place FP32 full sweep: one wave of resident blocks, rows grid-stride.
template <int G>
void launch_pull(const GraphView &v, bool bf16, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  if (bf16)
    launch_tiled(pull32_kernel<__nv_bfloat16, G>, 0, (v.n + kBlock / G - 1) / (kBlock / G), kBlock, st,
                 v, B, ctl, red);
  else
    launch_tiled(pull32_kernel<float, G>, 0, (v.n + kBlock / G - 1) / (kBlock / G), kBlock, st, v, B,
                 ctl, red);
}

template <int G>
void prepare_pull() {
  resident_blocks(pull32_kernel<float, G>, 0, kBlock);
  resident_blocks(pull32_kernel<__nv_bfloat16, G>, 0, kBlock);
}

}  // namespace

int launch_init(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  init_kernel<<<flat_grid(g.n), kBlock, 0, st>>>(g.n, B.r64, ctl, red, g.sys_of_row, g.sys_bmax);
  return 1;
}

int launch_sweep64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                   const GraphView *view) {
  const GraphView v = view ? *view : g.view();
  switch (g.group) {
    case 2: launch64<2>(v, st, B, ctl, red); break;
    case 4: launch64<4>(v, st, B, ctl, red); break;
    case 8: launch64<8>(v, st, B, ctl, red); break;
    case 16: launch64<16>(v, st, B, ctl, red); break;
    default: launch64<32>(v, st, B, ctl, red); break;
  }
  return 1;
}

int launch_sweep32(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                   bool bf16, const GraphView *view) {
  if (g.pull_lanes > 0 && !view) {
    const GraphView v = g.view();
    switch (g.pull_lanes) {
      case 2: launch_pull<2>(v, bf16, st, B, ctl, red); break;
      case 4: launch_pull<4>(v, bf16, st, B, ctl, red); break;
      case 8: launch_pull<8>(v, bf16, st, B, ctl, red); break;
      case 16: launch_pull<16>(v, bf16, st, B, ctl, red); break;
      default: launch_pull<32>(v, bf16, st, B, ctl, red); break;
    }
    return 1;
  }
  const GraphView v = view ? *view : g.view();
  GABP_TS_DISPATCH(g, {
    const size_t smem = 2 * Layout32<TSZ>::bytes;
    if (bf16)
      launch_tiled(sweep32_kernel<__nv_bfloat16, TSZ>, smem, v.ntiles_big, kTileBlock, st, v, B,
                   ctl, red);
    else
      launch_tiled(sweep32_kernel<float, TSZ>, smem, v.ntiles_big, kTileBlock, st, v, B, ctl, red);
  });
  return 1;
}

int launch_mean(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, bool bf16,
                const GraphView *view) {
  const GraphView v = view ? *view : g.view();
  GABP_TS_DISPATCH(g, {
    if (bf16)
      launch_tiled(mean_kernel<__nv_bfloat16, TSZ>, 2 * LayoutMean<__nv_bfloat16, TSZ>::bytes,
                   v.ntiles_big, kTileBlock, st, v, B, ctl, red);
    else
      launch_tiled(mean_kernel<float, TSZ>, 2 * LayoutMean<float, TSZ>::bytes, v.ntiles_big,
                   kTileBlock, st, v, B, ctl, red);
  });
  return 1;
}

// Colour schedule: b into the renumbered order, x back to the caller's.
// Element t of an n x width array: row t / width, column t % width.
__global__ void permute_gather_kernel(int64_t total, int32_t width, const int32_t *__restrict__ perm,
                                      const double *__restrict__ src, double *__restrict__ dst) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[t] = src[static_cast<int64_t>(perm[t / width]) * width + t % width];
}
__global__ void permute_scatter_kernel(int64_t total, int32_t width, const int32_t *__restrict__ perm,
                                       const double *__restrict__ src, double *__restrict__ dst) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[static_cast<int64_t>(perm[t / width]) * width + t % width] = src[t];
}

int launch_permute(int32_t n, int32_t width, cudaStream_t st, const int32_t *perm, const double *src,
                   double *dst, bool scatter) {
  const int64_t total = static_cast<int64_t>(n) * width;
  if (scatter) permute_scatter_kernel<<<flat_grid(total), kBlock, 0, st>>>(total, width, perm, src, dst);
  else permute_gather_kernel<<<flat_grid(total), kBlock, 0, st>>>(total, width, perm, src, dst);
  return 1;
}

int launch_check64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                   bool aitken) {
  (void)B;
  if (!aitken) return launch_residual(g, st, nullptr, ctl, red, CK_CHECK64);
  // extrapolated means into x, then the residual of x
  aitken_kernel<<<flat_grid(g.n), kBlock, 0, st>>>(g.n, ctl, nullptr);
  return 1 + launch_residual(g, st, nullptr, ctl, red, CK_CHECK64);
}

int launch_aitken(int32_t n, cudaStream_t st, Ctl *ctl, double *out) {
  aitken_kernel<<<flat_grid(n), kBlock, 0, st>>>(n, ctl, out);
  return 1;
}

int launch_ait_record(int32_t n, cudaStream_t st, Buffers B, const Ctl *ctl) {
  ait_record_kernel<<<flat_grid(n), kBlock, 0, st>>>(n, B, ctl);
  return 1;
}

int launch_refine_update(int32_t n, cudaStream_t st, Buffers B, Ctl *ctl) {
  refine_update_kernel<<<flat_grid(n), kBlock, 0, st>>>(n, B, ctl);
  return 1;
}

int launch_refine(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  refine_update_kernel<<<flat_grid(g.n), kBlock, 0, st>>>(g.n, B, ctl);
  return 1 + launch_residual(g, st, B.r64, ctl, red, CK_REFINE);
}

// Columns per lane of the multi right-hand-side kernels: ceil(K / 32) rounded
// up to 1, 2, 4 or 8 (K <= 256).
#define GABP_NC_DISPATCH(K, CALL)                  \
  do {                                             \
    const int nc_ = ((K) + 31) / 32;               \
    if (nc_ <= 1) { constexpr int NC = 1; CALL; }  \
    else if (nc_ <= 2) { constexpr int NC = 2; CALL; } \
    else if (nc_ <= 4) { constexpr int NC = 4; CALL; } \
    else { constexpr int NC = 8; CALL; }           \
  } while (0)

int launch_init_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K) {
  const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(g.n) * 32 + kBlock - 1) / kBlock,
                                                      static_cast<int64_t>(num_sms()) * 8));
  GABP_NC_DISPATCH(K, (init_multi_kernel<NC><<<std::max(grid, 1), kBlock, 0, st>>>(g.n, B, ctl, red, K)));
  return 1;
}

int launch_mean_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K,
                      const GraphView *view) {
  const GraphView v = view ? *view : g.view();
  const int64_t rows = v.row1 - v.row0;
  const int grid = static_cast<int>(std::min<int64_t>((rows * 32 + kBlock - 1) / kBlock,
                                                      static_cast<int64_t>(num_sms()) * 8));
  GABP_NC_DISPATCH(K, (mean_multi_kernel<NC><<<std::max(grid, 1), kBlock, 0, st>>>(v, B, ctl, red, K)));
  return 1;
}

int launch_refine_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K) {
  const int64_t total = static_cast<int64_t>(g.n) * K;
  refine_multi_update_kernel<<<flat_grid(total), kBlock, 0, st>>>(total, B, ctl, K);
  const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(g.n) * 32 + kBlock - 1) / kBlock,
                                                      static_cast<int64_t>(num_sms()) * 8));
  GABP_NC_DISPATCH(K, (residual_multi_kernel<NC><<<std::max(grid, 1), kBlock, 0, st>>>(g.view(), B, ctl, red, K)));
  return 2;
}

// Sets the shared-memory limits and caches the occupancy of every kernel the
// handle can launch (done at create time, before any graph is recorded).
void prepare_kernels(int group, bool bf16) {
  num_sms();
  prepare_pull<2>();
  prepare_pull<4>();
  prepare_pull<8>();
  prepare_pull<16>();
  prepare_pull<32>();
  switch (group) {
    case 2: prepare_group<2>(); break;
    case 4: prepare_group<4>(); break;
    case 8: prepare_group<8>(); break;
    case 16: prepare_group<16>(); break;
    default: prepare_group<32>(); break;
  }
  for (int ts : {512, kTileSlotsBig}) {
    Graph probe;
    probe.tile_slots = ts;
    GABP_TS_DISPATCH(probe, {
      resident_blocks(residual64_kernel<TSZ>, 2 * LayoutRes<TSZ>::bytes, kTileBlock);
      if (bf16) {
        resident_blocks(sweep32_kernel<__nv_bfloat16, TSZ>, 2 * Layout32<TSZ>::bytes, kTileBlock);
        resident_blocks(mean_kernel<__nv_bfloat16, TSZ>, 2 * LayoutMean<__nv_bfloat16, TSZ>::bytes,
                        kTileBlock);
      } else {
        resident_blocks(sweep32_kernel<float, TSZ>, 2 * Layout32<TSZ>::bytes, kTileBlock);
        resident_blocks(mean_kernel<float, TSZ>, 2 * LayoutMean<float, TSZ>::bytes, kTileBlock);
      }
    });
  }
}

void tile_sizes(int *big_slots, int *big_rows, int *small_slots, int *small_rows) {
  *big_slots = kTileSlotsBig;
  *big_rows = kTileRowsBig;
  *small_slots = kTileSlotsSmall;
  *small_rows = kTileRowsSmall;
}

int launch_lsq_rhs(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row,
                   const int64_t *aug_off, const int32_t *K, const int64_t *y_off, const double *y,
                   double *rhs) {
  lsq_rhs_kernel<<<flat_grid(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, y_off, y, rhs);
  return 1;
}

int launch_lsq_extract(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row,
                       const int64_t *aug_off, const int32_t *K, const int64_t *x_off,
                       const double *x_aug, double *xhat) {
  lsq_extract_kernel<<<flat_grid(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, x_off,
                                                          x_aug, xhat);
  return 1;
}

double bits_to_double(unsigned long long u) {
  double d;
  static_assert(sizeof(d) == sizeof(u), "size");
  std::memcpy(&d, &u, sizeof(d));
  return d;
}

}  // namespace gabp
