// gabp_dense.cu -- Section VII batches in dense bipartite form.
//
// The augmented system of Section VII,
//     [ I_K   S^T ] [x^]   [0]
//     [ S    -Psi ] [z ] = [y],        S of size N x K,
// has a complete bipartite graph: every unknown x^_r (r < K) is joined to
// every z_j (j < N) by the weight S_jr, and no two nodes of the same kind are
// joined.  Both directed messages of edge (z_j, x^_r) therefore live at the
// same position (j, r) of an N x K grid laid out like S:
//     Mz(j, r) = message x^_r -> z_j,      Mx(j, r) = message z_j -> x^_r.
// One synchronous round of Alg. 2 is then an elementwise map over the grid,
//     Mz'(j, r) from S_jr, the totals of x^_r and Mx(j, r)   (its reverse),
//     Mx'(j, r) from S_jr, the totals of z_j  and Mz(j, r),
// and the totals of the next round are the row sums (z_j) and column sums
// (x^_r) of the new grid.  There are no index arrays and no scatter: every
// access is a coalesced run and a sweep streams the grid once.
//
// Work mapping: persistent CTAs of 8 warps claim whole systems, largest
// first, from an atomic counter.  Inside a system, a warp takes whole grid
// rows (rows w, w + 8, ...), its lanes on the columns lane + 32 q (q < Q =
// ceil(K / 32) rounded up to 1, 2, 4 or 8).  A row's sum is the warp's sum
// and has one writer; each warp keeps the column sums of its lanes in
// registers, and the warps' column sums are added in warp order.  No sum
// depends on timing: the same input gives the same bits on every run.  The
// node work of a round (totals, tentative means, monitors) runs before the
// grid pass, from the sums the previous sweep left.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

namespace gabp {
namespace {

constexpr int kDenseBlock = 256;   // 8 warps
constexpr int kDenseWarps = kDenseBlock / 32;

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <class T> using T2 = typename V2<T>::t;

template <class T>
__device__ __forceinline__ T2<T> mk2(T a, T b) {
  T2<T> v;
  v.x = a;
  v.y = b;
  return v;
}

__device__ __forceinline__ float rcp(float d) { return rcp32(d); }
__device__ __forceinline__ double rcp(double d) { return recip64(d); }

__device__ __forceinline__ bool bad(float d) { return !(d != 0.0f) || !isfinite(d); }
__device__ __forceinline__ bool bad(double d) { return zero_or_nonfinite(d); }

// Both directed messages of one grid position.
template <class T>
struct Quad {
  T pz, ez, px, ex;
};

template <class T> struct FullIO;
template <> struct FullIO<float> {
  const float4 *__restrict__ in;
  float4 *__restrict__ out;
  __device__ Quad<float> ld(int64_t p) const {
    const float4 v = __ldcs(in + p);
    return Quad<float>{v.x, v.y, v.z, v.w};
  }
  __device__ void st(int64_t p, const Quad<float> &q) const {
    __stcs(out + p, make_float4(q.pz, q.ez, q.px, q.ex));
  }
};
template <> struct FullIO<double> {
  const double2 *__restrict__ inz, *__restrict__ inx;
  double2 *__restrict__ outz, *__restrict__ outx;
  __device__ Quad<double> ld(int64_t p) const {
    const double2 z = __ldcs(inz + p), x = __ldcs(inx + p);
    return Quad<double>{z.x, z.y, x.x, x.y};
  }
  __device__ void st(int64_t p, const Quad<double> &q) const {
    __stcs(outz + p, make_double2(q.pz, q.ez));
    __stcs(outx + p, make_double2(q.px, q.ex));
  }
};

__device__ __forceinline__ float2 ld_h(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_h(const __nv_bfloat162 *p) {
  return __bfloat1622float2(__ldcs(p));
}
__device__ __forceinline__ void st_h(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_h(__nv_bfloat162 *p, float2 v) {
  __stcs(p, __float22bfloat162_rn(v));
}

// A lane's running column sum.  With a warp per grid row it runs down only
// the rows of its warp, N / 8 <= 64 terms, and the eight warps' sums are
// added in warp order: the rounding floor stays near 1e-6 relative in FP32,
// below the precision rule's 1e-4 cycle threshold, so no compensation is
// carried (a compensated sum cost four adds a term).
template <class T>
struct ColSum {
  T s = T(0);
  __device__ __forceinline__ void add(T v) { s += v; }
  __device__ __forceinline__ T value() const { return s; }
};

// Claims the next system (thread 0) and hands its index to the whole CTA.
__device__ __forceinline__ int32_t claim(Ctl *ctl, int32_t *slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = static_cast<int32_t>(atomicAdd(&ctl->work_next, 1u));
  __syncthreads();
  return *slot;
}

// ---------------------------------------------------------------------------
// Per-round state of a full sweep, shared by the synchronous and the serial
// kernels: the buffers that hold the node sums of the last sweep and receive
// those of this one, the flags of the round, and the node work.  Node i of
// the round has the totals P~_i = A_ii + sumP_i and h~_i = rhs_i + sumEta_i
// (A_ii = 1 for x^, -psi for z; rhs_i = b_i in FP64, the scaled residual in
// the mixed modes).  FP32 rounds also keep the monitors of the tentative
// means d_i = h~_i / P~_i and, at the freeze, 1/P~_i.
// ---------------------------------------------------------------------------
template <class T>
struct FullRound {
  using V = T2<T>;
  static constexpr bool kF64 = sizeof(T) == 8;
  bool first, write_x = false, write_msgs = true, freeze = false;
  bool damp_all;                  // damping blends the x^ -> z messages too
  double inv_rn;
  const double *__restrict__ b;
  double *__restrict__ x;
  T gam;
  const V *__restrict__ sum_in;
  V *__restrict__ sum_out;
  float *__restrict__ sumE_out;   // freeze: sums of the first mean messages
  const float2 *__restrict__ mon_prev;
  float2 *__restrict__ mon_out;
  uint32_t mdd = 0, md = 0, mdP = 0, mP = 0;       // maxima over the CTA's systems
  uint32_t smdd = 0, smd = 0, smdP = 0, smP = 0;   // maxima over the current system

  __device__ FullRound(const DenseView &d, const Buffers &B, const Ctl *ctl) {
    const int par = ctl->par_m, pe = ctl->par_e, pmon = ctl->par_mon;
    first = ctl->first != 0;
    if (kF64) {
      if (ctl->mode == CTL_ROUNDS) {
        write_x = ctl->sweeps >= ctl->rounds_target;   // the infer-only pass
        write_msgs = !write_x;
      } else {
        write_x = ctl->write_x != 0;
      }
    } else {
      freeze = ctl->pending_freeze != 0;
    }
    inv_rn = ctl->inv_rn;
    b = ctl->b;
    x = ctl->x;
    gam = static_cast<T>(ctl->damping);
    damp_all = d.damp_scope == 0;
    if constexpr (kF64) {
      sum_in = par ? d.sum64[1] : d.sum64[0];
      sum_out = par ? d.sum64[0] : d.sum64[1];
    } else {
      sum_in = par ? d.sum32[1] : d.sum32[0];
      sum_out = par ? d.sum32[0] : d.sum32[1];
    }
    sumE_out = pe ? d.sumE[0] : d.sumE[1];
    mon_prev = pmon ? B.mon32[1] : B.mon32[0];
    mon_out = pmon ? B.mon32[0] : B.mon32[1];
  }

  // The current system's maxima into the CTA's.
  __device__ __forceinline__ void fold() {
    mdd = max(mdd, smdd);
    md = max(md, smd);
    mdP = max(mdP, smdP);
    mP = max(mP, smP);
    smdd = smd = smdP = smP = 0;
  }

  // Totals (P~_i, h~_i) of node i; *rhs receives rhs_i.
  __device__ __forceinline__ V node(int64_t i, T aii, const Buffers &B, T *rhs) {
    const V sm = first ? mk2<T>(T(0), T(0)) : sum_in[i];
    if constexpr (kF64) {
      const T bi = b[i];
      const T TP = aii + sm.x, Th = bi + sm.y;
      if (write_x) x[i] = Th / TP;
      *rhs = bi;
      return mk2<T>(TP, Th);
    } else {
      const float r = first ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
      const float TP = aii + sm.x, Th = r + sm.y;
      const float2 prev = first ? make_float2(0.f, 0.f) : mon_prev[i];
      const float di = Th / TP;
      mon_out[i] = make_float2(TP, di);
      smdd = fmax_bits(smdd, di - prev.y);
      smd = fmax_bits(smd, di);
      smdP = fmax_bits(smdP, TP - prev.x);
      smP = fmax_bits(smP, TP);
      if (freeze) B.invP32[i] = 1.0f / TP;
      if (first) B.rhs32[i] = r;
      *rhs = r;
      return mk2<T>(TP, Th);
    }
  }

  // Sums of node i over the messages this round sent to it.
  __device__ __forceinline__ void put_sum(int64_t i, V v) const {
    if (!kF64 && freeze) sumE_out[i] = static_cast<float>(v.y);
    else sum_out[i] = v;
  }

  __device__ void finish(Ctl *ctl, DevScalars *red, bool brk) {
    if (brk) atomicOr(&red->breakdown, 1);
    if constexpr (kF64) {
      last_block_control(ctl, red, CK_SWEEP64);
    } else {
      block_max4(widen(mdd), widen(md), widen(mdP), widen(mP), &red->max_dx, &red->max_x,
                 &red->max_dP, &red->max_P);
      last_block_control(ctl, red, CK_SWEEP32);
    }
  }
};

// Per-round state of a mean-only sweep (frozen precisions, FP32): node i has
// h~_i = rhs_i + sumEta_i and d_i = h~_i / P~_i with the frozen 1/P~_i.
struct MeanRound {
  bool first;
  bool damp_all;                  // damping blends the x^ -> z messages too
  double inv_rn;
  float gam;
  const float *__restrict__ sum_in;
  float *__restrict__ sum_out;
  const float2 *__restrict__ mon_prev;
  float2 *__restrict__ mon_out;
  uint32_t mdd = 0, md = 0;       // maxima over the CTA's systems
  uint32_t smdd = 0, smd = 0, smdP = 0, smP = 0;   // over the current system (no P~ here)

  __device__ MeanRound(const DenseView &d, const Buffers &B, const Ctl *ctl) {
    const int pe = ctl->par_e, pmon = ctl->par_mon;
    first = ctl->first != 0;
    inv_rn = ctl->inv_rn;
    gam = static_cast<float>(ctl->damping);
    damp_all = d.damp_scope == 0;
    sum_in = pe ? d.sumE[1] : d.sumE[0];
    sum_out = pe ? d.sumE[0] : d.sumE[1];
    mon_prev = pmon ? B.mon32[1] : B.mon32[0];
    mon_out = pmon ? B.mon32[0] : B.mon32[1];
  }

  __device__ __forceinline__ void fold() {
    mdd = max(mdd, smdd);
    md = max(md, smd);
    smdd = smd = 0;
  }

  // h~_i of node i; *rhs receives rhs_i.
  __device__ __forceinline__ float node(int64_t i, const Buffers &B, float *rhs) {
    const float r = first ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
    const float Th = r + (first ? 0.f : sum_in[i]);
    const float prev = first ? 0.f : mon_prev[i].y;
    const float di = Th * B.invP32[i];
    mon_out[i] = make_float2(0.f, di);
    smdd = fmax_bits(smdd, di - prev);
    smd = fmax_bits(smd, di);
    if (first) B.rhs32[i] = r;
    *rhs = r;
    return Th;
  }

  __device__ void finish(Ctl *ctl, DevScalars *red) {
    block_max4(widen(mdd), widen(md), 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
    last_block_control(ctl, red, CK_MEAN);
  }
};

// Columns each lane holds for a system of K columns: 1, 2, 4 or 8.
template <class F>
__device__ __forceinline__ void by_columns(int K, F &&f) {
  const int kq = (K + 31) >> 5;
  if (kq > 4) f(std::integral_constant<int, 8>{});
  else if (kq > 2) f(std::integral_constant<int, 4>{});
  else if (kq > 1) f(std::integral_constant<int, 2>{});
  else f(std::integral_constant<int, 1>{});
}

// ---------------------------------------------------------------------------
// Per-system control (Ctl::retire = 1).  The CTA that claims a system applies
// the controller's rules (gabp_device.cuh) to that system's own maxima: the
// precision freeze of Section V after its full sweeps, the end of its inner
// solve after the sweeps with frozen precisions.  When a system's inner
// solve ends, the same CTA takes its refinement step at once (sys_refine:
// x += rn_s d, its FP64 residual, its stop rule), and the first sweep of its
// next inner solve comes with the next launch.  Systems that are done or
// failed are passed over by every claim.  Every
// rule reads only the system's own numbers, so a system takes the same
// sweeps, and its solution the same bits, in a batch as when it is solved
// alone.
// ---------------------------------------------------------------------------
struct SysShared {
  SysCtl sc;                    // the claimed system's state (kept by thread 0)
  int32_t s;                    // claimed index (largest-first order)
  int32_t mode;                 // this sweep: 0 full, 1 freeze, 2 mean-only
  int32_t flag;                 // 1: its inner solve ends here, 2: and the grid pass is skipped
  union {                       // per-warp maxima (8-byte aligned for the 64-bit view)
    uint32_t red[4][kDenseWarps];
    unsigned long long red64[2][kDenseWarps];
  };
};
static_assert(offsetof(SysShared, red64) % 8 == 0, "64-bit maxima must be 8-byte aligned");

// Thread 0's counts over the systems its CTA handled, committed once per
// launch (held in shared memory: only thread 0 touches them).
struct Tally {
  uint32_t frozen, done, failed, checks, wide_seen;
  int32_t outer, fail_status;
  unsigned long long positions, rmax, rrelmax;
};

__device__ __forceinline__ void tally_commit(Ctl *ctl, const Tally &t) {
  if (threadIdx.x != 0) return;
  if (t.positions) atomicAdd(&ctl->positions, t.positions);
  if (t.frozen) atomicSub(&ctl->sys_unfrozen, static_cast<int>(t.frozen));
  if (t.done) atomicAdd(&ctl->sys_done, static_cast<int>(t.done));
  if (t.failed) atomicAdd(&ctl->sys_failed, static_cast<int>(t.failed));
  if (t.checks) atomicAdd(&ctl->checks, static_cast<int>(t.checks));
  if (t.outer) atomicMax(&ctl->outer, t.outer);
  if (t.fail_status) atomicMax(&ctl->sys_fail_status, t.fail_status);
  if (t.wide_seen) atomicOr(&ctl->wide_now, 1);
  if (t.rmax) atomicMax(&ctl->sys_rmax, t.rmax);
  if (t.rrelmax) atomicMax(&ctl->sys_rrelmax, t.rrelmax);
}

// Claims the next system and hands it to the whole CTA.  With per-system
// control, systems that are not iterating (state != 0) are passed over and
// thread 0 loads the claimed system's state into sh.sc; a system's first
// sweep of the solve takes ||b_s||_inf as the scale of its first inner solve.
__device__ __forceinline__ int32_t claim_sys(Ctl *ctl, const DenseView &d, bool on,
                                             SysShared &sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t s;
    for (;;) {
      s = static_cast<int32_t>(atomicAdd(&ctl->work_next, 1u));
      if (s >= d.nsys || !on) break;
      const int32_t o = d.sys[s].orig;
      if (d.sysctl[o].state == 0) {
        sh.sc = d.sysctl[o];
        if (sh.sc.sweeps == 0) {   // the first inner solve of the solve
          sh.sc.rn = dv(d.sys_bmax[o]);
          sh.sc.goal = ctl->inner_tol;
        }
        sh.mode = sh.sc.frozen;
        break;
      }
    }
    sh.s = s;
  }
  __syncthreads();
  return sh.s;
}

__device__ __forceinline__ double sys_inv_rn(const SysShared &sh) {
  const double rn = sh.sc.rn;
  return rn > 0.0 ? 1.0 / rn : 0.0;
}

// The controller's rules for one system after the node work of a sweep of
// the given mode, on the system's maxima (bit patterns of non-negative
// floats): relative change of d, dd = max |d_i - d_i'| / max |d_i|, and on
// full sweeps the same for P~.  Updates the history in sc and returns true
// when the system's inner solve ends with this sweep.
__device__ bool sys_rules(SysCtl &sc, const Ctl *ctl, int mode, uint32_t mdd, uint32_t md,
                          uint32_t mdP, uint32_t mP) {
  const int k = ++sc.k;
  const double dd = static_cast<double>(__uint_as_float(mdd)) /
                    fmax(static_cast<double>(__uint_as_float(md)), DBL_MIN);
  if (mode == 0) {   // precision convergence: the freeze comes with the next sweep
    const double dP = static_cast<double>(__uint_as_float(mdP)) /
                      fmax(static_cast<double>(__uint_as_float(mP)), DBL_MIN);
    const double rho = dP / (k == 1 ? INFINITY : sc.prev_dP);
    const double errP = dP == 0.0 ? 0.0 : (rho < 1.0 ? dP * rho / (1.0 - rho) : INFINITY);
    if (k >= 3 && (errP < 1e-6 || dP < 1e-7 || (rho >= 1.0 && dP < 1e-4))) sc.frozen = 1;
    sc.prev_dP = dP;
  }
  const double rho_d = dd / (k == 1 ? INFINITY : sc.prev_dd);
  const double err_d = dd == 0.0 ? 0.0 : (rho_d < 1.0 ? dd * rho_d / (1.0 - rho_d) : INFINITY);
  sc.stall = rho_d >= 1.0 ? sc.stall + 1 : 0;
  sc.prev_dd = dd;
  if (k == 1 || dd < 0.9 * sc.best_dd) {
    sc.best_dd = dd;
    sc.since_best = 0;
  } else {
    sc.since_best++;
  }
  // (a system whose ladder climbed takes the FP32 storage's rule)
  const double floor_dd = sc.wide ? ctl->floor_dd_wide : ctl->floor_dd;
  const int plateau_n = sc.wide ? 0 : ctl->plateau;
  const bool plateau = plateau_n > 0 && sc.since_best >= plateau_n && dd < floor_dd;
  return mode != 0 && k >= 3 &&
         (err_d < sc.goal || (sc.stall >= 2 && dd < floor_dd) || plateau);
}

// After the node work of a system (every thread calls it): the system's
// maxima over the CTA and the rules (thread 0).  Returns 0 when the system
// goes on, 1 when its inner solve ends after this sweep's grid pass (a
// freeze sweep still writes the frozen coefficients), 2 when it ends here
// and the grid pass is skipped (a mean-only sweep; its sweep is then
// counted).  The caller runs sys_refine in both cases.
template <class Round>
__device__ int sys_after_nodes(SysShared &sh, const Ctl *ctl, const DenseSys &sy, Round &R,
                               int mode) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t v[4] = {R.smdd, R.smd, R.smdP, R.smP};
  R.fold();
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = __reduce_max_sync(0xffffffffu, v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) sh.red[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t m = 0;
      for (int ww = 0; ww < kDenseWarps; ++ww) m = max(m, sh.red[k][ww]);
      v[k] = m;
    }
    const bool end = sys_rules(sh.sc, ctl, mode, v[0], v[1], v[2], v[3]);
    sh.flag = end ? (mode == 2 ? 2 : 1) : 0;
    if (sh.flag == 2) sh.sc.sweeps++;
  }
  __syncthreads();
  return sh.flag;
}

// The end of a system's sweep (thread 0): positions swept and, with
// per-system control, its sweep count, a completed freeze and the write-back.
__device__ __forceinline__ void sys_end(SysShared &sh, const DenseView &d, const DenseSys &sy,
                                        bool on, int mode, Tally &t) {
  if (threadIdx.x != 0) return;
  t.positions += static_cast<unsigned long long>(sy.K) * sy.N;
  if (!on) return;
  if (mode == 1) {
    sh.sc.frozen = 2;
    t.frozen++;
  }
  sh.sc.sweeps++;
  d.sysctl[sy.orig] = sh.sc;
}

// Doubles of shared memory sys_refine needs: x^ (K), z (N), S x (N) and the
// warps' partial sums of S^T z (kDenseWarps x K).
constexpr int kRefineBuf = kDenseMaxK + 2 * kDenseMaxN + kDenseWarps * kDenseMaxK;

// One pass over S (FP64) for R~ x: a warp per grid row j (rows w, w + 8,
// ...), lanes on the columns lane + 32 q; (S x)_j is the warp's sum, and each
// warp's partial column sums of S^T z go to its own slice of `part` (added
// in warp order by the caller).  x^ is read from shared memory, so only the
// column sums live in registers.
template <int Q>
__device__ __forceinline__ void refine_rows(const DenseSys &sy, const double *__restrict__ S,
                                            const double *vx, const double *vz, double *az,
                                            double *part) {
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double col[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) col[q] = 0.0;
  for (int j = w; j < N; j += kDenseWarps) {
    const double zj = vz[j];
    double row = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int r = lane + 32 * q;
      if (r < K) {
        const double a = __ldcs(S + static_cast<int64_t>(j) * K + r);
        row += a * vx[r];
        col[q] += a * zj;
      }
    }
    row = group_sum<32>(row);
    if (lane == 0) az[j] = row;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    if (r < K) part[w * kDenseMaxK + r] = col[q];
  }
}

// The refinement step of a system whose inner solve ended in this sweep
// (every thread of the CTA calls it; thread 0 holds the state in sh.sc).
// With d the tentative means the sweep's node work left in `mon` and rn_s
// the scale of the inner solve:
//     x <- x + rn_s d,   r = b - R~ x   (FP64),
// R~ x from S in FP64 in one pass (refine_rows; fixed order: the same bits
// every run).
// Then the system's stop rule: done when max |r| / ||b_s|| < tol (max |r| <
// tol for the absolute rule); failed when r is not finite or exceeds 1e30
// ||b_s||, or after eight refinement steps without a 10 % smaller stop
// measure (a BF16 handle's system first climbs the precision ladder at its
// first such step: its later inner solves store FP32 mean messages, with a
// fresh stall budget); otherwise r is kept as the right-hand side of its
// next inner solve, whose scale is rn_s = max |r| (history reset, k = 0) and
// whose goal is what the system's stop rule still needs.
__device__ void sys_refine(SysShared &sh, const Ctl *ctl, const DenseView &d, const DenseSys &sy,
                           const Buffers &B, const float2 *mon, double *buf, Tally &t) {
  const int K = sy.K, N = sy.N, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double *vx = buf, *vz = buf + K, *az = buf + K + N, *part = buf + K + 2 * N;
  double *__restrict__ x = ctl->x;
  const double *__restrict__ b = ctl->b;
  const double *__restrict__ S = d.S64 + sy.pair0;
  const double rn = sh.sc.rn;
  for (int k = tid; k < K + N; k += kDenseBlock) {
    const int64_t g = sy.node0 + k;
    const double v = x[g] + static_cast<double>(mon[g].y) * rn;
    x[g] = v;
    if (k < K) vx[k] = v;
    else vz[k - K] = v;
  }
  for (int k = tid; k < kDenseWarps * K; k += kDenseBlock)
    part[(k / K) * kDenseMaxK + k % K] = 0.0;   // warps without rows leave theirs at zero
  __syncthreads();
  by_columns(K, [&](auto q) { refine_rows<decltype(q)::value>(sy, S, vx, vz, az, part); });
  __syncthreads();
  const double bs = dv(d.sys_bmax[sy.orig]);
  unsigned long long smr = 0, smrel = 0;
  auto residual = [&](int64_t g, double Ax) {
    const double ri = b[g] - Ax;
    B.r64[g] = ri;
    smr = umax(smr, bits(fabs(ri)));
    smrel = umax(smrel, bits(bs > 0.0 ? fabs(ri) / bs : (ri == 0.0 ? 0.0 : INFINITY)));
  };
  for (int r = tid; r < K; r += kDenseBlock) {   // x^ rows: x_r + (S^T z)_r
    double c = 0.0;
#pragma unroll
    for (int ww = 0; ww < kDenseWarps; ++ww) c += part[ww * kDenseMaxK + r];
    residual(sy.node0 + r, vx[r] + c);
  }
  for (int j = tid; j < N; j += kDenseBlock)   // z rows: (S x)_j - psi z_j
    residual(sy.node0 + K + j, az[j] - sy.psi * vz[j]);
  smr = warp_max(smr);
  smrel = warp_max(smrel);
  unsigned long long(*red)[kDenseWarps] = sh.red64;
  if (lane == 0) {
    red[0][w] = smr;
    red[1][w] = smrel;
  }
  __syncthreads();
  if (tid == 0) {
    for (int ww = 1; ww < kDenseWarps; ++ww) {
      smr = umax(smr, red[0][ww]);
      smrel = umax(smrel, red[1][ww]);
    }
    SysCtl &sc = sh.sc;
    const double rs = dv(smr), prog = ctl->rel ? dv(smrel) : rs;
    sc.outer++;
    t.checks++;
    t.outer = max(t.outer, sc.outer);
    int fail = 0;
    const bool progressed = sc.outer == 1 || prog < 0.9 * sc.best_prog;
    if (prog < ctl->tol) {
      sc.state = 2;
      t.done++;
    } else if (!isfinite(rs) || rs > 1e30 * fmax(bs, DBL_MIN)) {
      fail = GABP_ERR_DIVERGED;
    } else if (progressed) {
      sc.best_prog = prog;
      sc.outer_stall = 0;
    } else if (ctl->ladder && !sc.wide) {   // BF16 storage: climb to FP32 at the first stall
      sc.wide = 1;
      sc.outer_stall = 0;
    } else if (++sc.outer_stall >= 8) {
      fail = GABP_ERR_NOT_CONVERGED;
    }
    if (fail) {
      sc.state = 3;
      t.failed++;
      t.fail_status = max(t.fail_status, fail);
    } else if (sc.state == 0) {   // its next inner solve
      sc.k = 0;
      sc.stall = 0;
      sc.since_best = 0;
      sc.rn = rs;
      // the next inner solve only has to shrink the residual by the factor
      // the stop rule still needs (0.3 margin; at most 1e-2, never tighter
      // than inner_tol); after a step that did not shrink the stop measure
      // by 10 % it takes inner_tol again
      sc.goal = progressed ? fmin(1e-2, fmax(ctl->inner_tol, 0.3 * ctl->tol / fmax(prog, DBL_MIN)))
                           : ctl->inner_tol;
    }
    if (sc.state != 0) {
      t.rmax = umax(t.rmax, smr);
      t.rrelmax = umax(t.rrelmax, smrel);
    }
    d.sysctl[sy.orig] = sc;
  }
}

// ---------------------------------------------------------------------------
// Full sweep, T = double (FP64 solves and gabp_run_rounds) or float (mixed
// modes, with the precision freeze), synchronous schedule (Alg. 2).  The
// messages of Alg. 2 at grid position (j, r), from the totals of the round:
//     P_ij = -S^2 / (P~_i - P_ji),   eta_ij = -S (h~_i - eta_ji) / (P~_i - P_ji).
// FP32 freeze: c = -S / (P~_i - P_ji) is stored and the first mean-only
// messages eta_ij = c (h~_i - eta_ji) are written (storage E) instead of full
// messages.
// ---------------------------------------------------------------------------

// Grid rows each warp loads ahead: U (the tuned figure) when U rows of Q
// columns a lane fit eight values, else 8 / Q.
template <int U, int Q>
constexpr int rows_ahead() {
  return U * Q <= 8 ? U : (8 / Q > 0 ? 8 / Q : 1);
}

// One warp per grid row j (rows w, w + 8, ...; the U rows it loads ahead are
// j, j + 8, ..., so the rows each warp sums, and the bits of every sum, do
// not depend on U), lanes on the columns lane + 32 q (q < Q), as in the
// serial kernels.  The row sums (totals of z_j) have
// one writer each and go straight to the round's sums; each warp keeps its
// column sums (totals of x^_r) in registers, and they are added in warp
// order through `part`, in two halves of four warps (so that the FP64 slices
// fit shared memory) -- no atomics, the same bits on every run.
template <class T, class E, int U, int Q>
__device__ __forceinline__ void full_sync_rows(const DenseSys &sy, const T *__restrict__ Sg,
                                               const FullIO<T> &io, float2 *__restrict__ C,
                                               E *__restrict__ h_out, const T2<T> *tx,
                                               const T2<T> *tz, T2<T> *part, T2<T> *ax,
                                               FullRound<T> &R, bool &brk) {
  using V = T2<T>;
  constexpr bool kF64 = sizeof(T) == 8;
  constexpr int UU = rows_ahead<U, Q>();
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool first = R.first, freeze = R.freeze;
  const T gam = R.gam;
  V xr[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    xr[q] = r < K ? tx[r] : mk2<T>(T(1), T(0));
  }
  ColSum<T> cP[Q], cE[Q];
  for (int j0 = w; j0 < N; j0 += kDenseWarps * UU) {
    T a[UU][Q];
    Quad<T> m[UU][Q];
#pragma unroll
    for (int u = 0; u < UU; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = j0 + kDenseWarps * u, r = lane + 32 * q;
        a[u][q] = T(0);
        m[u][q] = Quad<T>{T(0), T(0), T(0), T(0)};
        if (j < N && r < K) {
          const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
          a[u][q] = __ldcs(Sg + p);
          if (!first) m[u][q] = io.ld(p);
        }
      }
#pragma unroll
    for (int u = 0; u < UU; ++u) {
      const int j = j0 + kDenseWarps * u;
      if (j >= N) break;   // the same for every lane of the warp
      const V zj = tz[j];
      T rz = T(0), re = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        if (r >= K) continue;
        const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
        const T av = a[u][q];
        const Quad<T> &mm = m[u][q];
        Quad<T> o{T(0), T(0), T(0), T(0)};
        if (av != T(0)) {
          const T dz = xr[q].x - mm.px;   // P~_r - P_{z_j -> x_r}: towards z_j
          const T dx = zj.x - mm.pz;      // P~_j - P_{x_r -> z_j}: towards x_r
          brk |= bad(dz) || bad(dx);
          const T iz = rcp(dz), ix = rcp(dx);
          if (!kF64 && freeze) {
            const T cz = -av * iz, cx = -av * ix;
            C[p] = make_float2(static_cast<float>(cz), static_cast<float>(cx));
            o.ez = cz * (xr[q].y - mm.ex);
            o.ex = cx * (zj.y - mm.ez);
          } else {
            o.pz = -(av * av) * iz;
            o.px = -(av * av) * ix;
            o.ez = -av * (xr[q].y - mm.ex) * iz;
            o.ex = -av * (zj.y - mm.ez) * ix;
          }
          if (gam > T(0)) {   // blend the information with its previous value
            o.ez = gam * mm.ez + (T(1) - gam) * o.ez;
            o.ex = gam * mm.ex + (T(1) - gam) * o.ex;
          }
        } else if (!kF64 && freeze) {
          C[p] = make_float2(0.f, 0.f);
        }
        if (!kF64 && freeze) {
          st_h(h_out + p, make_float2(static_cast<float>(o.ez), static_cast<float>(o.ex)));
        } else {
          io.st(p, o);
        }
        rz += o.pz;
        re += o.ez;
        cP[q].add(o.px);
        cE[q].add(o.ex);
      }
      rz = group_sum<32>(rz);
      re = group_sum<32>(re);
      if (lane == 0) R.put_sum(sy.node0 + K + j, mk2<T>(rz, re));
    }
  }
  for (int half = 0; half < 2; ++half) {
    if ((w >> 2) == half) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        if (r < K) part[(w & 3) * kDenseMaxK + r] = mk2<T>(cP[q].value(), cE[q].value());
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += kDenseBlock) {
      V s = half ? ax[k] : part[k];
      for (int ww = half ? 0 : 1; ww < 4; ++ww) {
        s.x += part[ww * kDenseMaxK + k].x;
        s.y += part[ww * kDenseMaxK + k].y;
      }
      ax[k] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Mean-only sweep with frozen precisions (FP32 arithmetic; storage E = float2
// or __nv_bfloat162 per grid position), synchronous schedule:
//     eta_z' = c_z (h~_r - eta_x),   eta_x' = c_x (h~_j - eta_z).
// Mapping and sums as in the full sweep: a warp per grid row, row sums with
// one writer, column sums added in warp order.
// ---------------------------------------------------------------------------
template <class E, int U, int Q>
__device__ __forceinline__ void mean_sync_rows(const DenseSys &sy, const float2 *__restrict__ C,
                                               const E *__restrict__ h_in, E *__restrict__ h_out,
                                               const float *tx, const float *tz, float *part,
                                               MeanRound &R) {
  constexpr int UU = rows_ahead<U, Q>();
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool first = R.first;
  const float gam = R.gam;
  float hr[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    hr[q] = r < K ? tx[r] : 0.f;
  }
  ColSum<float> cE[Q];
  for (int j0 = w; j0 < N; j0 += kDenseWarps * UU) {
    float2 c[UU][Q], hv[UU][Q];
#pragma unroll
    for (int u = 0; u < UU; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = j0 + kDenseWarps * u, r = lane + 32 * q;
        c[u][q] = make_float2(0.f, 0.f);
        hv[u][q] = c[u][q];
        if (j < N && r < K) {
          const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
          c[u][q] = __ldcs(C + p);
          if (!first) hv[u][q] = ld_h(h_in + p);
        }
      }
#pragma unroll
    for (int u = 0; u < UU; ++u) {
      const int j = j0 + kDenseWarps * u;
      if (j >= N) break;   // the same for every lane of the warp
      const float tzj = tz[j];
      float re = 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        if (r >= K) continue;
        const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
        float ez = c[u][q].x * (hr[q] - hv[u][q].y), ex = c[u][q].y * (tzj - hv[u][q].x);
        if (gam > 0.f) {
          ez = gam * hv[u][q].x + (1.f - gam) * ez;
          ex = gam * hv[u][q].y + (1.f - gam) * ex;
        }
        st_h(h_out + p, make_float2(ez, ex));
        re += ez;
        cE[q].add(ex);
      }
      re = group_sum<32>(re);
      if (lane == 0) R.sum_out[sy.node0 + K + j] = re;
    }
  }
  // this warp's column sums to its own slice (added in warp order later)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    if (r < K) part[w * kDenseMaxK + r] = cE[q].value();
  }
}

// One system's mean-only round, synchronous schedule: node work (h~ of x^
// into tx, of z into tz), the per-system rules, the grid pass and the column
// sums.  Also the round of a system whose precisions are frozen inside a
// sweep of the full phase (per-system control).
template <class E, int U>
__device__ __forceinline__ void mean_sync_system(const DenseView &d, const DenseSys &sy,
                                                 const Buffers &B, Ctl *ctl, MeanRound &R,
                                                 const E *__restrict__ h_in, E *__restrict__ h_out,
                                                 float *tx, float *tz, float *part, double *rbuf,
                                                 bool on, SysShared &sh, Tally &t) {
  const int K = sy.K, N = sy.N, tid = threadIdx.x;
  for (int k = tid; k < K + N; k += kDenseBlock) {
    float rhs;
    const float Th = R.node(sy.node0 + k, B, &rhs);
    if (k < K) tx[k] = Th;
    else tz[k - K] = Th;
  }
  if (on) {
    if (sys_after_nodes(sh, ctl, sy, R, 2)) {   // its inner solve ends: no grid pass
      sys_refine(sh, ctl, d, sy, B, R.mon_out, rbuf, t);
      return;
    }
  } else {
    R.fold();
  }
  __syncthreads();
  by_columns(K, [&](auto q) {
    mean_sync_rows<E, U, decltype(q)::value>(sy, d.C32, h_in, h_out, tx, tz, part, R);
  });
  __syncthreads();
  for (int k = tid; k < K; k += kDenseBlock) {
    float sum = part[k];
    for (int ww = 1; ww < kDenseWarps; ++ww) sum += part[ww * kDenseMaxK + k];
    R.sum_out[sy.node0 + k] = sum;
  }
  sys_end(sh, d, sy, on, 2, t);
}

template <class E, int U>
__global__ void __launch_bounds__(kDenseBlock)
dense_mean_kernel(DenseView d, Buffers B, Ctl *ctl, DevScalars *red) {
  __shared__ float tx[kDenseMaxK], tz[kDenseMaxN];      // h~ of this round
  __shared__ float part[kDenseWarps * kDenseMaxK];      // per-warp column sums
  __shared__ double rbuf[kRefineBuf];                   // refinement steps (per-system control)
  __shared__ SysShared sh;
  MeanRound R(d, B, ctl);
  const bool on = ctl->retire != 0;
  const int pe = ctl->par_e;
  const E *__restrict__ h_in = static_cast<const E *>(pe ? d.H[1] : d.H[0]);
  E *__restrict__ h_out = static_cast<E *>(pe ? d.H[0] : d.H[1]);
  // (systems whose precision ladder climbed: FP32 mean messages)
  const float2 *__restrict__ w_in = static_cast<const float2 *>(pe ? d.H32[1] : d.H32[0]);
  float2 *__restrict__ w_out = static_cast<float2 *>(pe ? d.H32[0] : d.H32[1]);
  __shared__ Tally t;   // thread 0's counts (kept out of the registers)
  if (threadIdx.x == 0) t = Tally{};
  for (;;) {
    const int32_t s = claim_sys(ctl, d, on, sh);
    if (s >= d.nsys) break;
    if (on) {
      R.inv_rn = sys_inv_rn(sh);
      R.first = sh.sc.k == 0;   // the first sweep of the system's inner solve
      if constexpr (!std::is_same_v<E, float2>) {
        if (sh.sc.wide) {
          if (threadIdx.x == 0) t.wide_seen = 1;
          mean_sync_system<float2, U>(d, d.sys[s], B, ctl, R, w_in, w_out, tx, tz, part, rbuf, on,
                                      sh, t);
          continue;
        }
      }
    }
    mean_sync_system<E, U>(d, d.sys[s], B, ctl, R, h_in, h_out, tx, tz, part, rbuf, on, sh, t);
  }
  tally_commit(ctl, t);
  R.finish(ctl, red);
}

template <class T, class E, int U>
__global__ void __launch_bounds__(kDenseBlock)
dense_full_kernel(DenseView d, Buffers B, Ctl *ctl, DevScalars *red) {
  using V = T2<T>;
  constexpr bool kF64 = sizeof(T) == 8;
  __shared__ V tx[kDenseMaxK], tz[kDenseMaxN];   // (P~, h~) of this round
  __shared__ V part[4 * kDenseMaxK];             // four warps' column sums at a time
  __shared__ V ax[kDenseMaxK];                   // column sums of the new messages
  __shared__ double rbuf[kF64 ? 1 : kRefineBuf];  // refinement steps (per-system control)
  __shared__ SysShared sh;
  FullRound<T> R(d, B, ctl);
  const bool on = ctl->retire != 0;
  const int par = ctl->par_m, pe = ctl->par_e;
  const T *__restrict__ Sg = kF64 ? reinterpret_cast<const T *>(d.S64)
                                  : reinterpret_cast<const T *>(d.S32);
  FullIO<T> io;
  if constexpr (kF64) {
    io.inz = par ? d.Mz64[1] : d.Mz64[0];
    io.inx = par ? d.Mx64[1] : d.Mx64[0];
    io.outz = par ? d.Mz64[0] : d.Mz64[1];
    io.outx = par ? d.Mx64[0] : d.Mx64[1];
  } else {
    io.in = par ? d.M32[1] : d.M32[0];
    io.out = par ? d.M32[0] : d.M32[1];
  }
  // freeze outputs (and the mean-only rounds of frozen systems, per-system
  // control): mean messages go to the other mean buffer
  E *__restrict__ h_out = static_cast<E *>(pe ? d.H[0] : d.H[1]);
  const E *__restrict__ h_in = static_cast<const E *>(pe ? d.H[1] : d.H[0]);
  MeanRound Rm(d, B, ctl);
  bool brk = false;
  __shared__ Tally t;   // thread 0's counts (kept out of the registers)
  if (threadIdx.x == 0) t = Tally{};
  const int tid = threadIdx.x;

  for (;;) {
    const int32_t s = claim_sys(ctl, d, on, sh);
    if (s >= d.nsys) break;
    const DenseSys sy = d.sys[s];
    const int K = sy.K, N = sy.N;
    int mode = R.freeze ? 1 : 0;
    if constexpr (!kF64) {
      if (on) {
        mode = sh.mode;
        R.freeze = mode == 1;
        R.inv_rn = Rm.inv_rn = sys_inv_rn(sh);
        R.first = Rm.first = sh.sc.k == 0;   // the first sweep of the system's inner solve
        if (mode == 2) {   // precisions frozen already: a mean-only round
          float *ftx = reinterpret_cast<float *>(tx), *ftz = reinterpret_cast<float *>(tz);
          float *fpart = reinterpret_cast<float *>(part);
          if constexpr (!std::is_same_v<E, float2>) {
            if (sh.sc.wide) {   // its precision ladder climbed: FP32 mean messages
              if (threadIdx.x == 0) t.wide_seen = 1;
              mean_sync_system<float2, U>(
                  d, sy, B, ctl, Rm, static_cast<const float2 *>(pe ? d.H32[1] : d.H32[0]),
                  static_cast<float2 *>(pe ? d.H32[0] : d.H32[1]), ftx, ftz, fpart, rbuf, on, sh, t);
              continue;
            }
          }
          mean_sync_system<E, U>(d, sy, B, ctl, Rm, h_in, h_out, ftx, ftz, fpart, rbuf, on, sh, t);
          continue;
        }
      }
    }
    // ---- node work of the round ----
    for (int k = tid; k < K + N; k += kDenseBlock) {
      T rhs;
      const V tv = R.node(sy.node0 + k, k < K ? T(1) : static_cast<T>(-sy.psi), B, &rhs);
      if (k < K) tx[k] = tv;
      else tz[k - K] = tv;
    }
    // (a full or freeze sweep never skips its grid pass: the freeze writes
    // the frozen coefficients the next inner solve needs)
    int end = 0;
    if (!kF64 && on) end = sys_after_nodes(sh, ctl, sy, R, mode);
    else R.fold();
    __syncthreads();
    if (!R.write_msgs) continue;
    // ---- grid pass (row sums of z written inside, column sums into ax) ----
    by_columns(K, [&](auto q) {
      full_sync_rows<T, E, U, decltype(q)::value>(sy, Sg, io, d.C32, h_out, tx, tz, part, ax, R,
                                                  brk);
    });
    for (int k = tid; k < K; k += kDenseBlock) R.put_sum(sy.node0 + k, ax[k]);
    sys_end(sh, d, sy, on, mode, t);
    if (end) sys_refine(sh, ctl, d, sy, B, R.mon_out, rbuf, t);
  }
  tally_commit(ctl, t);
  R.mdd = max(R.mdd, Rm.mdd);
  R.md = max(R.md, Rm.md);
  R.finish(ctl, red, brk);
}

// ---------------------------------------------------------------------------
// Serial schedule (Section III-C) in the dense form, with the nodes visited
// class by class: every x^_r first, then every z_j (no two nodes of a class
// are joined, so the order inside a class does not matter).
//   x^ class:  Mz'(j, r) from the totals of x^_r -- the column sums the last
//              sweep left -- and Mx(j, r);
//   z class:   the totals of z_j are the row sums of Mz'(j, .), and
//              Mx'(j, r) follows from them and Mz'(j, r).
// One warp therefore takes a whole row j, lanes on columns lane + 32 q
// (q < Q): it forms Mz'(j, .) in registers, sums the row across the warp,
// and forms Mx'(j, .) -- the sweep still streams the grid once.  Mz is read
// again only for damping (its previous information), so it is stored only
// when damping blends it (damp_scope 0).  Messages are updated in place: every grid position is
// read and written by the same lane within a sweep.
// Planar layout, pair p = pair0 + j K + r:
//   FP64:   Mx64[0][p] = (Px, eta_x), Mz64[0][p] = (Pz, eta_z);
//   FP32:   float2 planes (Px, eta_x) at M32[0], (Pz, eta_z) after them;
//   mean:   eta_x plane at H[0], eta_z plane after it (storage E1).
// The node sums the sweep leaves are exactly the totals the serial round
// ends with: x^ from the new Mx', z from the new Mz'.
// ---------------------------------------------------------------------------
template <class E> struct Half;
template <> struct Half<float2> { using t = float; };
template <> struct Half<__nv_bfloat162> { using t = __nv_bfloat16; };

__device__ __forceinline__ float ld1(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(__ldcs(p)); }
__device__ __forceinline__ void st1(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st1(__nv_bfloat16 *p, float v) { __stcs(p, __float2bfloat16_rn(v)); }


template <class T, class E1, int Q, bool FZ, bool FI>
__device__ __forceinline__ void full_serial_rows(const DenseSys &sy, const T *__restrict__ Sg,
                                                 T2<T> *__restrict__ mx, T2<T> *__restrict__ mz,
                                                 float2 *__restrict__ C, E1 *__restrict__ hx,
                                                 E1 *__restrict__ hz, const T2<T> *tx,
                                                 const T *zr, T2<T> *part, FullRound<T> &R,
                                                 bool &brk) {
  using V = T2<T>;
  constexpr bool kF64 = sizeof(T) == 8;
  constexpr int U = 8 / Q;   // rows in flight per warp step: U Q loads per lane and array
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // damp_x: blend the z -> x^ messages; damp_z: the x^ -> z ones as well
  constexpr bool first = FI, freeze = !kF64 && FZ;
  const bool damp_x = R.gam > T(0), damp_z = damp_x && R.damp_all;
  const T gam = R.gam;
  const T aii = static_cast<T>(-sy.psi);
  ColSum<T> cP[Q], cE[Q];
  for (int j0 = w * U; j0 < N; j0 += kDenseWarps * U) {
    T a[U][Q];
    V m[U][Q];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = j0 + u, r = lane + 32 * q;
        a[u][q] = T(0);
        m[u][q] = mk2<T>(T(0), T(0));
        if (j < N && r < K) {
          const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
          a[u][q] = __ldcs(Sg + p);
          if (!first) m[u][q] = __ldcs(mx + p);
        }
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= N) break;   // the same for every lane of the warp
      // x^_r -> z_j for the columns of this lane, and the totals of z_j
      // (freeze: c_z goes to C.x at once, c_x follows into C.y)
      T pz[Q], ez[Q];
      T sP = T(0), sE = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        pz[q] = ez[q] = T(0);
        const int r = lane + 32 * q;
        const T av = a[u][q];
        const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
        if (av != T(0)) {
          const V xr = tx[r];
          const T dz = xr.x - m[u][q].x;   // P~_r - P_{z_j -> x_r}
          const T iz = rcp(dz);
          pz[q] = -(av * av) * iz;
          if (freeze) {
            const T cz = -av * iz;
            reinterpret_cast<float *>(C)[2 * p] = static_cast<float>(cz);
            ez[q] = cz * (xr.y - m[u][q].y);
          } else {
            ez[q] = -av * (xr.y - m[u][q].y) * iz;
          }
          if (damp_z) ez[q] = gam * (first ? T(0) : __ldcs(mz + p).y) + (T(1) - gam) * ez[q];
        } else if (freeze && r < K) {
          reinterpret_cast<float *>(C)[2 * p] = 0.f;
        }
        sP += pz[q];
        sE += ez[q];
      }
      sP = group_sum<32>(sP);
      sE = group_sum<32>(sE);
      // breakdown (a zero or non-finite P~_r - P_{z_j -> x_r} in the row) shows
      // as a non-finite row sum; the z_j -> x^_r messages' in the column sums
      brk |= !isfinite(sP) || !isfinite(sE);
      const T TPz = aii + sP, Thz = zr[j] + sE;
      // z_j -> x^_r
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        if (r >= K) continue;
        const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
        const T av = a[u][q];
        T px = T(0), ex = T(0), cx = T(0);
        if (av != T(0)) {
          const T dx = TPz - pz[q];   // P~_j - P_{x_r -> z_j}
          const T ix = rcp(dx);
          px = -(av * av) * ix;
          if (freeze) {
            cx = -av * ix;
            ex = cx * (Thz - ez[q]);
          } else {
            ex = -av * (Thz - ez[q]) * ix;
          }
          if (damp_x) ex = gam * m[u][q].y + (T(1) - gam) * ex;
        }
        if (freeze) {
          reinterpret_cast<float *>(C)[2 * p + 1] = static_cast<float>(cx);
          st1(hx + p, static_cast<float>(ex));
          if (damp_z) st1(hz + p, static_cast<float>(ez[q]));
        } else {
          __stcs(mx + p, mk2<T>(px, ex));
          if (damp_z) __stcs(mz + p, mk2<T>(pz[q], ez[q]));
        }
        cP[q].add(px);
        cE[q].add(ex);
      }
      if (lane == 0) R.put_sum(sy.node0 + sy.K + j, mk2<T>(sP, sE));
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) brk |= !isfinite(cP[q].value()) || !isfinite(cE[q].value());
  // this warp's column sums to its own slice (added in warp order later)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    if (r < K) part[w * kDenseMaxK + r] = mk2<T>(cP[q].value(), cE[q].value());
  }
}

template <class E1, int Q>
__device__ __forceinline__ void mean_serial_rows(const DenseSys &sy, const float2 *__restrict__ C,
                                                 E1 *__restrict__ hx, E1 *__restrict__ hz,
                                                 const float *tx, const float *zr, float *part,
                                                 MeanRound &R) {
  constexpr int U = 8 / Q;
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool first = R.first, damp_x = R.gam > 0.f, damp_z = damp_x && R.damp_all;
  const float gam = R.gam;
  float hr[Q];
  ColSum<float> cE[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    hr[q] = r < K ? tx[r] : 0.f;
  }
  for (int j0 = w * U; j0 < N; j0 += kDenseWarps * U) {
    float2 c[U][Q];
    float ho[U][Q], zo[U][Q];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = j0 + u, r = lane + 32 * q;
        c[u][q] = make_float2(0.f, 0.f);
        ho[u][q] = zo[u][q] = 0.f;
        if (j < N && r < K) {
          const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
          c[u][q] = __ldcs(C + p);
          if (!first) {
            ho[u][q] = ld1(hx + p);
            if (damp_z) zo[u][q] = ld1(hz + p);
          }
        }
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= N) break;   // the same for every lane of the warp
      float ez[Q];
      float sE = 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        ez[q] = c[u][q].x * (hr[q] - ho[u][q]);
        if (damp_z) ez[q] = gam * zo[u][q] + (1.f - gam) * ez[q];
        sE += ez[q];
      }
      sE = group_sum<32>(sE);
      const float Thz = zr[j] + sE;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        if (r >= K) continue;
        const int64_t p = sy.pair0 + static_cast<int64_t>(j) * K + r;
        float ex = c[u][q].y * (Thz - ez[q]);
        if (damp_x) ex = gam * ho[u][q] + (1.f - gam) * ex;
        st1(hx + p, ex);
        if (damp_z) st1(hz + p, ez[q]);
        cE[q].add(ex);
      }
      if (lane == 0) R.sum_out[sy.node0 + sy.K + j] = sE;
    }
  }
  // this warp's column sums to its own slice (added in warp order later)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    if (r < K) part[w * kDenseMaxK + r] = cE[q].value();
  }
}

// One system's mean-only round, serial schedule (node work: h~ of x^ into
// tx, rhs of z into zr), as mean_sync_system.
template <class E1>
__device__ __forceinline__ void mean_serial_system(const DenseView &d, const DenseSys &sy,
                                                   const Buffers &B, Ctl *ctl, MeanRound &R,
                                                   E1 *hx, E1 *hz, float *tx, float *zr,
                                                   float *part, double *rbuf, bool on,
                                                   SysShared &sh, Tally &t) {
  const int K = sy.K, N = sy.N, tid = threadIdx.x;
  for (int k = tid; k < K + N; k += kDenseBlock) {
    float rhs;
    const float Th = R.node(sy.node0 + k, B, &rhs);
    if (k < K) tx[k] = Th;
    else zr[k - K] = rhs;
  }
  if (on) {
    if (sys_after_nodes(sh, ctl, sy, R, 2)) {   // its inner solve ends: no grid pass
      sys_refine(sh, ctl, d, sy, B, R.mon_out, rbuf, t);
      return;
    }
  } else {
    R.fold();
  }
  __syncthreads();
  by_columns(K, [&](auto q) {
    mean_serial_rows<E1, decltype(q)::value>(sy, d.C32, hx, hz, tx, zr, part, R);
  });
  __syncthreads();
  for (int k = tid; k < K; k += kDenseBlock) {
    float sum = part[k];
    for (int ww = 1; ww < kDenseWarps; ++ww) sum += part[ww * kDenseMaxK + k];
    R.sum_out[sy.node0 + k] = sum;
  }
  sys_end(sh, d, sy, on, 2, t);
}

template <class E1>
__global__ void __launch_bounds__(kDenseBlock)
dense_mean_serial_kernel(DenseView d, Buffers B, Ctl *ctl, DevScalars *red) {
  __shared__ float tx[kDenseMaxK];                   // h~ of x^
  __shared__ float part[kDenseWarps * kDenseMaxK];   // per-warp sums of the new eta_x, by column
  __shared__ float zr[kDenseMaxN];                   // rhs of z
  __shared__ double rbuf[kRefineBuf];                // refinement steps (per-system control)
  __shared__ SysShared sh;
  MeanRound R(d, B, ctl);
  const bool on = ctl->retire != 0;
  E1 *hx = static_cast<E1 *>(d.H[0]);
  E1 *hz = hx + d.pairs;
  float *wx = static_cast<float *>(d.H32[0]);   // (systems whose ladder climbed: FP32 planes)
  float *wz = wx + d.pairs;
  __shared__ Tally t;   // thread 0's counts (kept out of the registers)
  if (threadIdx.x == 0) t = Tally{};
  for (;;) {
    const int32_t s = claim_sys(ctl, d, on, sh);
    if (s >= d.nsys) break;
    if (on) {
      R.inv_rn = sys_inv_rn(sh);
      R.first = sh.sc.k == 0;   // the first sweep of the system's inner solve
      if constexpr (!std::is_same_v<E1, float>) {
        if (sh.sc.wide) {
          if (threadIdx.x == 0) t.wide_seen = 1;
          mean_serial_system<float>(d, d.sys[s], B, ctl, R, wx, wz, tx, zr, part, rbuf, on, sh, t);
          continue;
        }
      }
    }
    mean_serial_system<E1>(d, d.sys[s], B, ctl, R, hx, hz, tx, zr, part, rbuf, on, sh, t);
  }
  tally_commit(ctl, t);
  R.finish(ctl, red);
}

// FP32: three CTAs of 256 threads per SM (at most 85 registers a thread).
template <class T, class E>
__global__ void __launch_bounds__(kDenseBlock, sizeof(T) == 4 ? 3 : 1)
dense_full_serial_kernel(DenseView d, Buffers B, Ctl *ctl, DevScalars *red) {
  using V = T2<T>;
  using E1 = typename Half<E>::t;
  constexpr bool kF64 = sizeof(T) == 8;
  __shared__ V tx[kDenseMaxK];                   // totals of x^
  __shared__ V part[kDenseWarps * kDenseMaxK];   // per-warp sums of the new Mx', by column
  __shared__ T zr[kDenseMaxN];                   // rhs of z
  __shared__ double rbuf[kF64 ? 1 : kRefineBuf];  // refinement steps (per-system control)
  __shared__ SysShared sh;
  FullRound<T> R(d, B, ctl);
  const bool on = ctl->retire != 0;
  const T *__restrict__ Sg = kF64 ? reinterpret_cast<const T *>(d.S64)
                                  : reinterpret_cast<const T *>(d.S32);
  V *mx, *mz;
  if constexpr (kF64) {
    mx = d.Mx64[0];
    mz = d.Mz64[0];
  } else {
    mx = reinterpret_cast<float2 *>(d.M32[0]);
    mz = mx + d.pairs;
  }
  E1 *hx = static_cast<E1 *>(d.H[0]);
  E1 *hz = hx + d.pairs;
  MeanRound Rm(d, B, ctl);
  bool brk = false;
  __shared__ Tally t;   // thread 0's counts (kept out of the registers)
  if (threadIdx.x == 0) t = Tally{};
  const int tid = threadIdx.x;

  for (;;) {
    const int32_t s = claim_sys(ctl, d, on, sh);
    if (s >= d.nsys) break;
    const DenseSys sy = d.sys[s];
    const int K = sy.K, N = sy.N;
    int mode = R.freeze ? 1 : 0;
    if constexpr (!kF64) {
      if (on) {
        mode = sh.mode;
        R.freeze = mode == 1;
        R.inv_rn = Rm.inv_rn = sys_inv_rn(sh);
        R.first = Rm.first = sh.sc.k == 0;   // the first sweep of the system's inner solve
        if (mode == 2) {   // precisions frozen already: a mean-only round
          float *ftx = reinterpret_cast<float *>(tx), *fzr = reinterpret_cast<float *>(zr);
          float *fpart = reinterpret_cast<float *>(part);
          if constexpr (!std::is_same_v<E1, float>) {
            if (sh.sc.wide) {   // its precision ladder climbed: FP32 mean messages
              if (threadIdx.x == 0) t.wide_seen = 1;
              float *wx = static_cast<float *>(d.H32[0]);
              mean_serial_system<float>(d, sy, B, ctl, Rm, wx, wx + d.pairs, ftx, fzr, fpart, rbuf,
                                        on, sh, t);
              continue;
            }
          }
          mean_serial_system<E1>(d, sy, B, ctl, Rm, hx, hz, ftx, fzr, fpart, rbuf, on, sh, t);
          continue;
        }
      }
    }
    for (int k = tid; k < K + N; k += kDenseBlock) {
      T rhs;
      const V tv = R.node(sy.node0 + k, k < K ? T(1) : static_cast<T>(-sy.psi), B, &rhs);
      if (k < K) tx[k] = tv;
      else zr[k - K] = rhs;
    }
    int end = 0;   // (a full or freeze sweep never skips its grid pass)
    if (!kF64 && on) end = sys_after_nodes(sh, ctl, sy, R, mode);
    else R.fold();
    __syncthreads();
    if (!R.write_msgs) continue;
    by_columns(K, [&](auto q) {
      // (the sweep's kind as template flags: the common full sweep carries
      // neither the freeze's stores nor the first round's zero messages)
      constexpr int QQ = decltype(q)::value;
      if (R.freeze && R.first)
        full_serial_rows<T, E1, QQ, true, true>(sy, Sg, mx, mz, d.C32, hx, hz, tx, zr, part, R, brk);
      else if (R.freeze)
        full_serial_rows<T, E1, QQ, true, false>(sy, Sg, mx, mz, d.C32, hx, hz, tx, zr, part, R, brk);
      else if (R.first)
        full_serial_rows<T, E1, QQ, false, true>(sy, Sg, mx, mz, d.C32, hx, hz, tx, zr, part, R, brk);
      else
        full_serial_rows<T, E1, QQ, false, false>(sy, Sg, mx, mz, d.C32, hx, hz, tx, zr, part, R, brk);
    });
    __syncthreads();
    for (int k = tid; k < K; k += kDenseBlock) {
      V sum = part[k];
      for (int ww = 1; ww < kDenseWarps; ++ww) {
        sum.x += part[ww * kDenseMaxK + k].x;
        sum.y += part[ww * kDenseMaxK + k].y;
      }
      R.put_sum(sy.node0 + k, sum);
    }
    sys_end(sh, d, sy, on, mode, t);
    if (end) sys_refine(sh, ctl, d, sy, B, R.mon_out, rbuf, t);
  }
  tally_commit(ctl, t);
  R.mdd = max(R.mdd, Rm.mdd);
  R.md = max(R.md, Rm.md);
  R.finish(ctl, red, brk);
}

// ---------------------------------------------------------------------------
// FP64 residual of the augmented systems, r = b - R~ x:
//     x^ rows:  r_r = b_r - (x_r + sum_j S_jr z_j),
//     z rows:   r_j = b_j - (sum_r S_jr x_r - psi z_j),
// with max |r| and, per system, max |r| / ||b_s||_inf.  One warp per grid
// row (lanes on columns lane + 32 q, as in the serial sweeps): the row sum
// has a single writer, and each warp's column sums go to its own slice of
// `part`, added in warp order -- no atomics, the same result every run.
// With per-system control (FP64 solves) the stop rule is applied to each
// system here, and a system that meets it is done: later sweeps pass it over
// and its x stays.
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void residual_rows(const DenseSys &sy, const double *__restrict__ S64,
                                              const double *vx, const double *vz, double *az,
                                              double *part) {
  constexpr int U = 8 / Q;
  const int K = sy.K, N = sy.N, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double xr[Q], col[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    xr[q] = r < K ? vx[r] : 0.0;
    col[q] = 0.0;
  }
  for (int j0 = w * U; j0 < N; j0 += kDenseWarps * U) {
    double a[U][Q];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = j0 + u, r = lane + 32 * q;
        a[u][q] = (j < N && r < K) ? __ldcs(S64 + sy.pair0 + static_cast<int64_t>(j) * K + r) : 0.0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= N) break;   // the same for every lane of the warp
      const double zj = vz[j];
      double row = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        row += a[u][q] * xr[q];
        col[q] += a[u][q] * zj;
      }
      row = group_sum<32>(row);
      if (lane == 0) az[j] = row;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
    if (r < K) part[w * kDenseMaxK + r] = col[q];
  }
}

__global__ void __launch_bounds__(kDenseBlock)
dense_residual_kernel(DenseView d, double *__restrict__ r_out, Ctl *ctl, DevScalars *red,
                      int kind) {
  __shared__ double vx[kDenseMaxK], vz[kDenseMaxN];   // x^ and z of the system
  __shared__ double az[kDenseMaxN];                   // sum_r S_jr x_r per row
  __shared__ double part[kDenseWarps * kDenseMaxK];   // per warp: sum_j S_jr z_j
  __shared__ unsigned long long sred[2][kDenseWarps];
  __shared__ int32_t cur;
  const double *__restrict__ b = ctl->b;
  const double *__restrict__ x = ctl->x;
  const bool on = ctl->retire != 0 && kind == CK_CHECK64;
  const bool rel = ctl->rel != 0;
  const double tol = ctl->tol;
  unsigned long long mr = 0, mrel = 0;
  __shared__ Tally t;   // thread 0's counts (kept out of the registers)
  if (threadIdx.x == 0) t = Tally{};
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (;;) {
    const int32_t s = claim(ctl, &cur);
    if (s >= d.nsys) break;
    const DenseSys sy = d.sys[s];
    const int K = sy.K, N = sy.N;
    for (int k = tid; k < K + N; k += kDenseBlock) {
      const double v = x[sy.node0 + k];
      if (k < K) vx[k] = v;
      else vz[k - K] = v;
    }
    for (int k = tid; k < kDenseWarps * K; k += kDenseBlock)
      part[(k / K) * kDenseMaxK + k % K] = 0.0;   // warps without rows leave theirs at zero
    __syncthreads();
    by_columns(K, [&](auto q) { residual_rows<decltype(q)::value>(sy, d.S64, vx, vz, az, part); });
    __syncthreads();
    const double bs = dv(d.sys_bmax[sy.orig]);
    unsigned long long smr = 0, smrel = 0;
    for (int k = tid; k < K + N; k += kDenseBlock) {
      const int64_t i = sy.node0 + k;
      double Ax;
      if (k < K) {
        double c = 0.0;
#pragma unroll
        for (int w = 0; w < kDenseWarps; ++w) c += part[w * kDenseMaxK + k];
        Ax = vx[k] + c;
      } else {
        Ax = az[k - K] - sy.psi * vz[k - K];
      }
      const double ri = b[i] - Ax;
      if (r_out) r_out[i] = ri;
      smr = umax(smr, bits(fabs(ri)));
      smrel = umax(smrel, bits(bs > 0.0 ? fabs(ri) / bs : (ri == 0.0 ? 0.0 : INFINITY)));
    }
    mr = umax(mr, smr);
    mrel = umax(mrel, smrel);
    if (on) {   // the system's own stop rule (thread 0)
      smr = warp_max(smr);
      smrel = warp_max(smrel);
      if (lane == 0) {
        sred[0][wid] = smr;
        sred[1][wid] = smrel;
      }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < kDenseWarps; ++w) {
          smr = umax(smr, sred[0][w]);
          smrel = umax(smrel, sred[1][w]);
        }
        SysCtl &sc = d.sysctl[sy.orig];
        if (sc.state != 2 && (rel ? dv(smrel) < tol : dv(smr) < tol)) {
          sc.state = 2;
          t.done++;
        }
      }
    }
  }
  tally_commit(ctl, t);
  block_max4(mr, mrel, 0, 0, &red->max_r, &red->max_rrel, nullptr, nullptr);
  last_block_control(ctl, red, kind);
}

int g_sms = 0;
std::mutex g_mu;
std::unordered_map<const void *, int> g_res;

int sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

// Persistent grid: every resident CTA slot, but no more CTAs than systems.
template <class Kern>
int dense_grid(Kern kernel, int32_t nsys) {
  int bps = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_res.find(reinterpret_cast<const void *>(kernel));
    if (it == g_res.end()) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kDenseBlock, 0);
      bps = std::max(bps, 1);
      g_res[reinterpret_cast<const void *>(kernel)] = bps;
    } else {
      bps = it->second;
    }
  }
  return static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>(nsys, static_cast<int64_t>(sms()) * bps)));
}

}  // namespace

// Rows each warp loads ahead: 1, 2 or 4 (the autotuner's choice).
#define GABP_ROWS_DISPATCH(U, ...)                        \
  do {                                                    \
    if ((U) >= 4) { constexpr int UR = 4; __VA_ARGS__; }   \
    else if ((U) == 1) { constexpr int UR = 1; __VA_ARGS__; } \
    else { constexpr int UR = 2; __VA_ARGS__; }            \
  } while (0)

int launch_dense_full64(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  auto k = d.serial ? dense_full_serial_kernel<double, float2> : dense_full_kernel<double, float2, 2>;
  k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
  return 1;
}

int launch_dense_full32(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                        bool bf16) {
  if (d.serial) {
    auto k = bf16 ? dense_full_serial_kernel<float, __nv_bfloat162>
                  : dense_full_serial_kernel<float, float2>;
    k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    return 1;
  }
  GABP_ROWS_DISPATCH(d.rows_full, {
    if (bf16) {
      auto k = dense_full_kernel<float, __nv_bfloat162, UR>;
      k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    } else {
      auto k = dense_full_kernel<float, float2, UR>;
      k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    }
  });
  return 1;
}

int launch_dense_mean(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                      bool bf16) {
  if (d.serial) {
    auto k = bf16 ? dense_mean_serial_kernel<__nv_bfloat16> : dense_mean_serial_kernel<float>;
    k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    return 1;
  }
  GABP_ROWS_DISPATCH(d.rows_mean, {
    if (bf16) {
      auto k = dense_mean_kernel<__nv_bfloat162, UR>;
      k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    } else {
      auto k = dense_mean_kernel<float2, UR>;
      k<<<dense_grid(k, d.nsys), kDenseBlock, 0, st>>>(d.v, B, ctl, red);
    }
  });
  return 1;
}

int launch_dense_residual(const Dense &d, cudaStream_t st, double *r_out, Ctl *ctl,
                          DevScalars *red, bool refine) {
  dense_residual_kernel<<<dense_grid(dense_residual_kernel, d.nsys), kDenseBlock, 0, st>>>(
      d.v, r_out, ctl, red, refine ? CK_REFINE : CK_CHECK64);
  return 1;
}

// Caches the occupancy of every dense kernel (done at create time, before
// any graph is recorded).
void prepare_dense_kernels(bool bf16) {
  // (a BF16 handle also runs the FP32-storage mean kernels once its
  // precision ladder climbs)
  dense_grid(dense_full_kernel<double, float2, 2>, 1);
  dense_grid(dense_full_serial_kernel<double, float2>, 1);
  dense_grid(dense_residual_kernel, 1);
  dense_grid(dense_mean_serial_kernel<float>, 1);
  if (bf16) {
    dense_grid(dense_full_serial_kernel<float, __nv_bfloat162>, 1);
    dense_grid(dense_mean_serial_kernel<__nv_bfloat16>, 1);
  } else {
    dense_grid(dense_full_serial_kernel<float, float2>, 1);
  }
  for (int u : {1, 2, 4}) {
    GABP_ROWS_DISPATCH(u, {
      dense_grid(dense_mean_kernel<float2, UR>, 1);
      if (bf16) {
        dense_grid(dense_full_kernel<float, __nv_bfloat162, UR>, 1);
        dense_grid(dense_mean_kernel<__nv_bfloat162, UR>, 1);
      } else {
        dense_grid(dense_full_kernel<float, float2, UR>, 1);
      }
    });
  }
}

}  // namespace gabp
