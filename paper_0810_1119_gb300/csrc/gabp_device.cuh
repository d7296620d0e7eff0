// gabp_device.cuh -- device code shared by the kernel translation units:
// reductions on IEEE bit patterns, the FP64 reciprocal, L2 cache policies,
// and the solve controller that the last block of every controlling launch
// runs.  Included inside an anonymous namespace, so every translation unit
// keeps its own copy (the library is built without relocatable device code).
#pragma once

#include <cfloat>

#include "gabp_internal.h"

namespace gabp {
namespace {

__device__ __forceinline__ unsigned long long bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}

__device__ __forceinline__ double dv(unsigned long long u) {
  return __longlong_as_double(static_cast<long long>(u));
}

__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Running maximum of |v| for FP32 values, kept as the bit pattern of the
// non-negative float (NaN compares above +inf); widened to the FP64 bit
// pattern once per thread for the block reduction.
__device__ __forceinline__ uint32_t fmax_bits(uint32_t m, float v) {
  const uint32_t u = __float_as_uint(fabsf(v));
  return u > m ? u : m;
}
__device__ __forceinline__ unsigned long long widen(uint32_t m) {
  return bits(static_cast<double>(__uint_as_float(m)));
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide maximum of up to four non-negative values (as bit patterns),
// committed with one atomicMax per value and block by thread 0.  Every thread
// of the block must call it.
__device__ void block_max4(unsigned long long v0, unsigned long long v1, unsigned long long v2,
                           unsigned long long v3, unsigned long long *d0, unsigned long long *d1,
                           unsigned long long *d2, unsigned long long *d3) {
  __shared__ unsigned long long sm[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v0 = warp_max(v0); v1 = warp_max(v1); v2 = warp_max(v2); v3 = warp_max(v3);
  if (lane == 0) { sm[0][w] = v0; sm[1][w] = v1; sm[2][w] = v2; sm[3][w] = v3; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    unsigned long long u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = warp_max(lane < nw ? sm[k][lane] : 0ull);
    if (lane == 0) {
      if (d0 && u[0]) atomicMax(d0, u[0]);
      if (d1 && u[1]) atomicMax(d1, u[1]);
      if (d2 && u[2]) atomicMax(d2, u[2]);
      if (d3 && u[3]) atomicMax(d3, u[3]);
    }
  }
}

template <int G, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads call it; every thread gets the result).
template <class T>
__device__ T block_sum(T v) {
  __shared__ T part[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) part[w] = v;
  __syncthreads();
  T tot = T(0);
  for (int k = 0; k < nw; ++k) tot += part[k];
  return tot;
}

// L2 eviction policies (createpolicy): the once-per-sweep streams (A, c, rev,
// row pointers) are loaded evict-first so that the message buffers, which are
// read back on the next sweep, stay resident in the 126 MB L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// FP32 1/d of a cavity precision (the dense Section VII full sweeps): the
// hardware approximation (rcp.approx, within about one unit in the last
// place; precisions are never subnormal).  FP32 messages only drive the inner
// solves of the FP64 refinement, which removes errors of that size; there the
// IEEE division sequence was a third of a full sweep's instructions.  The CSR
// and grid sweeps keep the IEEE division: on an indefinite tree the in-place
// CSR form needed 60 % more sweeps with the approximation.
__device__ __forceinline__ float rcp32(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// 1/d in FP64: an FP32 reciprocal seed (relative error e0 < 2^-22), then the
// cubic Newton-Raphson step y (1 + e + e^2) with e = 1 - d y, whose error is
// e0^3 < 2^-66 before rounding.  For |d| outside [2^-99, 2^99) (where the
// FP32 seed could under- or overflow), zero or non-finite d, the IEEE
// division is used.  The range test reads the exponent field with integer
// instructions: on GB300 every FP64 compare would occupy the slow FP64 pipe.
__device__ __forceinline__ double recip64(double d) {
  const unsigned ex = static_cast<unsigned>(__double_as_longlong(d) >> 52) & 0x7FFu;
  if (ex - 924u > 1121u - 924u) return 1.0 / d;
  const double y = static_cast<double>(__frcp_rn(static_cast<float>(d)));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// d == 0 or d not finite (the breakdown of Alg. 2's division), tested on the
// bit pattern with integer instructions.
__device__ __forceinline__ bool zero_or_nonfinite(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d)) &
                               0x7FFFFFFFFFFFFFFFull;
  return u == 0ull || u >= 0x7FF0000000000000ull;
}

// ---------------------------------------------------------------------------
// Controller (one thread of the last block of a controlling launch).
// ---------------------------------------------------------------------------
enum CtrlKind { CK_INIT = 1, CK_SWEEP64, CK_CHECK64, CK_SWEEP32, CK_MEAN, CK_REFINE, CK_INITK,
                CK_MEANK, CK_REFINEK };

__device__ void finish(Ctl &c, int status) {
  c.status = status;
  c.done = 1;
  c.phase = PH_DONE;
}

// FP64 sweeps: whether sweep `t` (1-based) writes the tentative means, and
// where (the Aitken ring, or x).
__device__ void plan_means(Ctl &c, int t) {
  const bool check = (t % c.check_every == 0) || t >= c.max_iter;
  c.write_x = check || (c.aitken > 0 && t % c.aitken == 0);
  c.xw = c.aitken > 0 ? c.ring[c.nw % 3] : c.x;
}

__device__ bool diverged(double rn, double bnorm) {
  return !isfinite(rn) || rn > 1e30 * fmax(bnorm, DBL_MIN);
}

// Phase of the next mean-only sweep, number c.k + 1 of the inner solve: FP32
// storage once the ladder climbed, and the Aitken records after sweeps 64,
// 128, ... where a kernel of their own takes them (CSR handles).
__device__ __forceinline__ int mean_phase(const Ctl &c) {
  const bool rec = c.ait_rec && ((c.k + 1) & ((1 << kAitMinLevel) - 1)) == 0;
  return c.wide ? (rec ? PH_MEANWR : PH_MEANW) : (rec ? PH_MEANR : PH_MEAN);
}

// Reductions are read through volatile loads (they were committed by other
// blocks' atomics) and zeroed once consumed.
__device__ void control(Ctl &c, DevScalars *red, int kind) {
  volatile DevScalars *r = red;
  c.steps++;
  if (r->timeout) {
    finish(c, GABP_ERR_TIMEOUT);
    kind = 0;
  }
  switch (kind) {
    case CK_INIT: {
      c.bnorm = dv(r->max_b);
      r->max_b = 0;
      c.thr = c.rel ? c.tol * c.bnorm : c.tol;
      c.residual = c.bnorm;
      if (!isfinite(c.bnorm)) { finish(c, GABP_ERR_INVALID_ARG); break; }
      if (c.mode == CTL_FP64) {
        c.phase = PH_FULL64;
        plan_means(c, 1);
      } else if (c.mode == CTL_PREC) {
        // precisions only: zero right-hand side, unit scale
        c.rn = 1.0;
        c.inv_rn = 1.0;
        c.outer = 1;
        c.phase = PH_FULL32;
      } else {
        c.rn = c.bnorm;
        c.best_rn = INFINITY;
        c.outer_stall = -1;   // the first refinement check sets the reference
        if (c.rn < c.thr || c.bnorm == 0.0) { finish(c, GABP_OK); break; }
        c.inv_rn = 1.0 / c.rn;
        c.outer = 1;
        c.phase = c.frozen ? PH_MEAN : PH_FULL32;
      }
      break;
    }
    case CK_SWEEP64: {
      if (c.mode == CTL_ROUNDS) {
        // the pass after `rounds_target` sweeps only infers and leaves the
        // state alone, so the last round's messages stay in m64[par_m]
        const bool infer_pass = c.sweeps >= c.rounds_target;
        if (!infer_pass) { c.sweeps++; c.par_m ^= 1; c.first = 0; }
        // Aitken: the means of rounds R - 2s, R - s and R go to the ring
        if ((c.write_x || infer_pass) && c.aitken > 0) c.nw++;
        const int R = c.rounds_target, s2 = 2 * c.aitken;
        const bool ait = c.aitken > 0 && R >= s2;
        c.write_x = ait && (c.sweeps == R - s2 || c.sweeps == R - c.aitken);
        c.xw = ait ? c.ring[c.nw % 3] : c.x;
        break;
      }
      c.sweeps++;
      c.sweeps_full++;
      c.par_m ^= 1;
      c.first = 0;
      if (r->breakdown) { finish(c, GABP_ERR_BREAKDOWN); break; }
      if (c.write_x && c.aitken > 0) c.nw++;
      c.check_now = (c.sweeps % c.check_every == 0) || c.sweeps >= c.max_iter;
      if (c.check_now) c.phase = PH_CHECK64;
      plan_means(c, c.sweeps + 1);
      break;
    }
    case CK_CHECK64:
    case CK_REFINE: {
      c.checks++;
      const double rn = dv(r->max_r), rrel = dv(r->max_rrel);
      r->max_r = 0;
      r->max_rrel = 0;
      c.residual = rn;
      if (r->breakdown) { finish(c, GABP_ERR_BREAKDOWN); break; }
      // batched handles: every system meets its own relative rule
      const bool met = c.batched ? (c.rel ? rrel < c.tol : rn < c.tol) : rn < c.thr;
      if (met) { finish(c, GABP_OK); break; }
      if (diverged(rn, c.bnorm)) { finish(c, GABP_ERR_DIVERGED); break; }
      if (c.sweeps >= c.max_iter) { finish(c, GABP_ERR_NOT_CONVERGED); break; }
      if (kind == CK_CHECK64) { c.phase = PH_FULL64; break; }
      // Refinement that stopped paying: eight outer steps without a 10 %
      // smaller residual (inner solves no more accurate than their storage
      // allows).  Slow but real progress -- a batch whose slowest system
      // gains a little per step -- keeps going.  BF16 storage climbs the
      // precision ladder at its first such step: from then on the inner
      // solves store FP32 mean messages (each starts from zero messages, so
      // nothing is converted), with a fresh stall budget.
      {
        // progress in the measure the stop rule uses (batches: worst relative)
        const double prog = (c.batched && c.rel) ? rrel : rn;
        if (c.outer_stall < 0 || prog < 0.9 * c.best_rn) {
          c.best_rn = prog;
          c.outer_stall = 0;
        } else if (c.ladder && !c.wide) {
          c.wide = 1;
          c.outer_stall = 0;
          c.floor_dd = c.floor_dd_wide;
          c.plateau = 0;
        } else if (++c.outer_stall >= 8) {
          finish(c, GABP_ERR_NOT_CONVERGED);
          break;
        }
      }
      // Aitken on the mixed inner solves: after an extrapolated step that
      // did not shrink the residual by 10 %, the next step goes without
      if (c.ait_mixed) {
        c.ait_ok = !c.ait_use || rn < 0.9 * c.rn;
        c.ait_use = 0;
      }
      // next refinement step: solve A d = r / ||r|| from zero mean messages.
      // One system: the inner solve only has to shrink the residual by the
      // factor the stop rule still needs (0.3 margin), never more than
      // inner_tol.  A batch keeps inner_tol: its inner accuracy is measured
      // against the largest system's residual, which says nothing about the
      // smallest system's own relative rule.
      c.outer++;
      c.rn = rn;
      c.inv_rn = 1.0 / rn;
      c.inner_goal = c.batched ? c.inner_tol : fmax(c.inner_tol, 0.3 * c.thr / fmax(rn, DBL_MIN));
      c.k = 0;
      c.ait_k0 = 0;
      c.stall = 0;
      c.prev_dd = INFINITY;
      c.best_dd = INFINITY;
      c.since_best = 0;
      c.prev_dP = INFINITY;
      c.first = 1;
      c.phase = c.frozen ? mean_phase(c) : PH_FULL32;
      break;
    }
    case CK_SWEEP32:
    case CK_MEAN: {
      if (kind == CK_SWEEP32 && c.retire) {
        // per-system control: the sweep moved the full messages of unfrozen
        // systems and the mean messages of frozen (and freezing) ones
        c.sweeps_full++;
        c.par_m ^= 1;
        c.par_e ^= 1;
      } else if (kind == CK_SWEEP32) {
        c.sweeps_full++;
        if (c.pending_freeze) {
          c.frozen = 1;
          c.pending_freeze = 0;
          c.par_e ^= 1;
          c.e_slots = 1;
          c.ait_k0 = c.k + 1;   // this full sweep's number: the records start after it
        }
        else c.par_m ^= 1;
      } else {
        c.sweeps_mean++;
        c.sweeps_wide += c.wide;
        c.par_e ^= 1;
        c.e_slots = 0;
      }
      if (c.retire) {   // per-system control: a sweep in which some system stored FP32
        volatile Ctl *vc = &c;
        if (vc->wide_now) {
          c.sweeps_wide++;
          c.wide_now = 0;
        }
      }
      if (c.mode == CTL_PREC && c.frozen) {
        c.sweeps++;
        if (r->breakdown) finish(c, GABP_ERR_BREAKDOWN);
        else finish(c, GABP_OK);
        break;
      }
      c.par_mon ^= 1;
      c.second = c.first;
      c.first = 0;
      c.sweeps++;
      c.k++;
      const double mx = dv(r->max_x), mdx = dv(r->max_dx);
      const double mP = dv(r->max_P), mdP = dv(r->max_dP);
      r->max_x = 0; r->max_dx = 0; r->max_P = 0; r->max_dP = 0;
      if (r->breakdown) { finish(c, GABP_ERR_BREAKDOWN); break; }
      const double dd = mdx / fmax(mx, DBL_MIN);
      if (!isfinite(dd)) { finish(c, GABP_ERR_DIVERGED); break; }
      if (c.retire) {
        // per-system control: the sweep applied every rule to each system and
        // ran the refinement steps; the solve ends when every system is done
        // or failed, or at max_iter sweeps
        volatile Ctl *vc = &c;
        const int finished = vc->sys_done + vc->sys_failed;
        if (finished >= c.nsys || c.sweeps >= c.max_iter) {
          c.residual = dv(vc->sys_rmax);
          if (finished < c.nsys) finish(c, GABP_ERR_NOT_CONVERGED);
          else finish(c, vc->sys_failed ? vc->sys_fail_status : GABP_OK);
          break;
        }
        c.frozen = vc->sys_unfrozen == 0;
        c.phase = c.frozen ? PH_MEAN : PH_FULL32;
        break;
      }
      if (kind == CK_SWEEP32 && !c.frozen && !c.pending_freeze) {
        // Precision convergence: relative change of the node precisions,
        // remaining error extrapolated with the observed contraction rate.
        const double dP = mdP / fmax(mP, DBL_MIN);
        const double rho = dP / c.prev_dP;
        const double errP = dP == 0.0 ? 0.0 : (rho < 1.0 ? dP * rho / (1.0 - rho) : INFINITY);
        // A change that stopped shrinking below 1e-4 is FP32 rounding of the
        // precision sums (long rows settle into a two-sweep cycle of that size).
        if (c.k >= 3 && (errP < 1e-6 || dP < 1e-7 || (rho >= 1.0 && dP < 1e-4))) c.pending_freeze = 1;
        c.prev_dP = dP;
      }
      const double rho_d = dd / c.prev_dd;
      const double err_d = dd == 0.0 ? 0.0 : (rho_d < 1.0 ? dd * rho_d / (1.0 - rho_d) : INFINITY);
      c.stall = rho_d >= 1.0 ? c.stall + 1 : 0;
      c.prev_dd = dd;
      // Plateau: the change has not shrunk by 10 % for `plateau` sweeps (the
      // storage rounding floor of BF16 messages; off for FP32 storage).
      if (dd < 0.9 * c.best_dd) { c.best_dd = dd; c.since_best = 0; }
      else c.since_best++;
      const bool plateau = c.plateau > 0 && c.since_best >= c.plateau && dd < c.floor_dd;
      const bool inner_done = c.frozen && c.k >= 3 &&
                              (err_d < c.inner_goal || (c.stall >= 2 && dd < c.floor_dd) || plateau);
      if (inner_done || c.sweeps >= c.max_iter) {
        c.phase = PH_REFINE;
        if (c.ait_mixed) {
          // Aitken on the inner solve's means: the widest record spacing s
          // with 6 s <= k whose three latest records were all taken by mean
          // sweeps (after the freeze sweep ait_k0 of the first inner solve)
          int sel = -1;
          for (int j = kAitLevels - 1; j >= 0; --j) {
            const int s = 1 << (kAitMinLevel + j);
            if (6 * s <= c.k && ((c.k >> (kAitMinLevel + j)) - 2) * s > c.ait_k0) { sel = j; break; }
          }
          c.ait_level = sel;
          c.ait_m = sel >= 0 ? c.k >> (kAitMinLevel + sel) : 0;
          c.ait_use = sel >= 0 && c.ait_ok;
          c.ait_steps += c.ait_use;
          c.ait_md = mx;
        }
      } else {
        c.phase = c.frozen ? mean_phase(c) : PH_FULL32;
      }
      break;
    }
    case CK_INITK: {
      // per-column ||b_k||, thresholds and scales
      double worst = 0.0;
      bool all_done = true, bad = false;
      for (int k = 0; k < c.K; ++k) {
        const double bn = dv(c.cols.bmax[k]);
        c.cols.bmax[k] = 0;
        c.cols.bnorm[k] = bn;
        c.cols.thr[k] = c.rel ? c.tol * bn : c.tol;
        c.cols.rn[k] = bn;
        c.cols.inv_rn[k] = bn > 0.0 ? 1.0 / bn : 0.0;
        bad |= !isfinite(bn);
        all_done &= bn < c.cols.thr[k] || bn == 0.0;
        worst = fmax(worst, bn);
      }
      c.bnorm = worst;
      c.residual = worst;
      c.best_rn = worst;
      if (bad) { finish(c, GABP_ERR_INVALID_ARG); break; }
      if (all_done) { finish(c, GABP_OK); break; }
      c.outer = 1;
      c.first = 1;
      c.phase = PH_MEANK;
      break;
    }
    case CK_MEANK: {
      c.sweeps_mean++;
      c.par_e ^= 1;
      c.first = 0;
      c.sweeps++;
      c.k++;
      const double mx = dv(r->max_x), mdx = dv(r->max_dx);
      r->max_x = 0; r->max_dx = 0;
      const double dd = mdx / fmax(mx, DBL_MIN);
      if (!isfinite(dd)) { finish(c, GABP_ERR_DIVERGED); break; }
      const double rho_d = dd / c.prev_dd;
      const double err_d = dd == 0.0 ? 0.0 : (rho_d < 1.0 ? dd * rho_d / (1.0 - rho_d) : INFINITY);
      c.stall = rho_d >= 1.0 ? c.stall + 1 : 0;
      c.prev_dd = dd;
      const bool inner_done = c.k >= 3 && (err_d < c.inner_goal || (c.stall >= 2 && dd < 1e-4));
      c.phase = (inner_done || c.sweeps >= c.max_iter) ? PH_REFINEK : PH_MEANK;
      break;
    }
    case CK_REFINEK: {
      c.checks++;
      double worst = 0.0;
      bool all_done = true, bad = false;
      for (int k = 0; k < c.K; ++k) {
        const double rn = dv(c.cols.rmax[k]);
        c.cols.rmax[k] = 0;
        c.cols.rn[k] = rn;
        c.cols.inv_rn[k] = rn > 0.0 ? 1.0 / rn : 0.0;
        all_done &= rn < c.cols.thr[k];
        bad |= diverged(rn, c.cols.bnorm[k]);
        worst = fmax(worst, rn);
      }
      c.residual = worst;
      if (all_done) { finish(c, GABP_OK); break; }
      if (bad) { finish(c, GABP_ERR_DIVERGED); break; }
      if (c.sweeps >= c.max_iter) { finish(c, GABP_ERR_NOT_CONVERGED); break; }
      if (worst < 0.9 * c.best_rn) { c.best_rn = worst; c.outer_stall = 0; }
      else if (++c.outer_stall >= 8) { finish(c, GABP_ERR_NOT_CONVERGED); break; }
      c.outer++;
      c.k = 0;
      c.stall = 0;
      c.prev_dd = INFINITY;
      c.first = 1;
      {
        double need = INFINITY;   // the column furthest from its threshold sets the goal
        for (int k = 0; k < c.K; ++k)
          if (c.cols.rn[k] > 0.0) need = fmin(need, c.cols.thr[k] / c.cols.rn[k]);
        c.inner_goal = fmax(c.inner_tol, 0.3 * need);
      }
      c.phase = PH_MEANK;
      break;
    }
  }
  // Hard bound on controller steps: the loop ends even if a rule misfires.
  if (!c.done && c.mode != CTL_ROUNDS && c.steps > 4 * c.max_iter + 64)
    finish(c, GABP_ERR_NOT_CONVERGED);
  if (c.in_graph) {
    cudaGraphSetConditional(c.h_phase, c.done ? 0u : static_cast<unsigned>(c.phase));
    cudaGraphSetConditional(c.h_while, c.done ? 0u : 1u);
  }
}

// Called by every thread at the end of a controlling launch.  No waiting:
// each block bumps a counter after its atomics; the block that brings it to
// gridDim.x runs the controller.
__device__ void last_block_control(Ctl *ctl, DevScalars *red, int kind) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->blocks_done, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    ctl->blocks_done = 0;
    ctl->work_next = 0;
    if (kind != 0) control(*ctl, red, kind);   // 0: a colour pass that is not a sweep's last
    __threadfence();
  }
}

// ---------------------------------------------------------------------------
// Shared-memory staging with cp.async.bulk on an mbarrier.  Every wait is
// bounded in time: once kWaitLimitNs (gabp_internal.h) of the GPU's global
// timer have passed since its first unsatisfied poll it gives up and returns
// false.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr uint32_t r128(uint64_t b) {
  return static_cast<uint32_t>((b + 127) & ~uint64_t{127});
}
// Bytes of a staged array of `count` elements of size `es` (plus slack for
// the 16-byte rounding of the copy's start and end).
__host__ __device__ constexpr uint32_t region(int count, int es) {
  return r128(static_cast<uint64_t>(count + 32) * es);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for phase `parity` of `bar` for at most `limit_ns` nanoseconds of
// global time after the first unsatisfied poll (the timer is read only once
// a poll has failed, so a wait whose copy has landed costs one poll).
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity,
                                              unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 >= limit_ns) return false;
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitLimitNs);
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One staged array: elements [first, first + count) of `base`, copied from
// the 16-byte boundary at or below `first` to the one at or above the end.
template <class E>
struct Seg {
  static constexpr int64_t kPer = 16 / static_cast<int64_t>(sizeof(E));
  __device__ static uint32_t bytes(int64_t first, int64_t count) {
    const int64_t a0 = first - first % kPer;
    const int64_t a1 = (first + count + kPer - 1) / kPer * kPer;
    return static_cast<uint32_t>((a1 - a0) * static_cast<int64_t>(sizeof(E)));
  }
  __device__ static void copy(uint32_t dst, const E *base, int64_t first, int64_t count,
                              uint32_t bar) {
    const uint32_t b = bytes(first, count);
    if (b) bulk_g2s(dst, base + (first - first % kPer), b, bar);
  }
  __device__ static void copy(uint32_t dst, const E *base, int64_t first, int64_t count,
                              uint32_t bar, uint64_t policy) {
    const uint32_t b = bytes(first, count);
    if (b) bulk_g2s_hint(dst, base + (first - first % kPer), b, bar, policy);
  }
  // Shared-memory pointer to element `first` of a staged run.
  __device__ static E *at(unsigned char *region_ptr, int64_t first) {
    return reinterpret_cast<E *>(region_ptr) + first % kPer;
  }
};

}  // namespace
}  // namespace gabp
