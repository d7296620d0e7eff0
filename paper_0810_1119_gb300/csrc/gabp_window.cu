// gabp_window.cu -- the mean-only sweep of Alg. 2 with frozen precisions
// (eta_ij = c_ij (h~_i - eta_ji), h~_i = rhs_i + sum_k eta_ki) in the window
// form: the message exchange between senders and receivers is a fixed
// two-level permutation through shared memory instead of a scatter.
//
// Why: in the slot layout a row reads its incoming messages contiguously but
// sends each message to the slot rev[s] of another row.  On a random graph
// that is one scattered 4-byte store per directed edge, each touching its
// own 32-byte L2 sector; those stores, not the bytes, set the time of the
// tile form (mean_kernel).
//
// The window form cuts the rows into windows of consecutive rows (about
// `target` slots each).  The messages live in a receive-ordered buffer: the
// range of window J (16-byte aligned) holds every message bound for J,
// grouped by source window and, within a group, by destination slot.  The
// messages that window I sends to J therefore form one contiguous run in
// J's range.  One CTA per SM walks its windows; for window J it
//   A. copies J's whole range into shared memory with one bulk copy
//      (cp.async.bulk, issued while the previous window was being processed)
//      and places every element at its slot (p2: range position -> window
//      slot), rebuilding J's incoming messages in slot order;
//   B. forms the node totals h~_i of its rows in slot order (a thread per
//      row sums in slot order, a warp per row of degree > 64 in a fixed
//      butterfly order: deterministic), records d_i = h~_i / P~_i, and
//      overwrites each incoming message e with h~_i - e;
//   C. walks its send order -- its slots sorted by destination slot -- and
//      stores the message of send position q, c_q (h~_i - eta_ji) =
//      cq[q] * smem[outmap[q]], into its run of the destination window's
//      range (a run table gives each run's first position).
// Loads are whole-window bulk copies or contiguous streams, stores are
// contiguous within runs of W^2 / E elements on a random graph (W the window
// size), and the bytes per directed edge are those of the tile form:
// message in 4 + p2 2 + outmap 2 + c 4 + message out 4.
//
// Layouts.  The receive-ordered buffers (bins) belong to the window form.
// The freeze sweep (sweep32 / pull32) writes c32 and the first mean messages
// in the slot layout; the controller marks that with Ctl::e_slots, and the
// next window sweep reads its input from the slot layout (window J's slots
// are one contiguous range) and copies c into send order (cq) once.
// Refinement steps start from zero messages.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace gabp {
namespace {

constexpr int kWinBlock = 1024;     // threads per window CTA
constexpr int kWinUnroll = 8;       // independent loads in flight per thread (sends)
constexpr int kWinHeavy = 64;       // rows of higher degree are summed by a warp
constexpr int kWinRowsPerThread = 4;                    // rows a thread prefetches
constexpr int kWinMaxRows = kWinRowsPerThread * kWinBlock;   // rows per window at most

__device__ __forceinline__ float ld_eta(const float *p) { return *p; }
__device__ __forceinline__ float ld_eta(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Streams read once per sweep: evict-first in L2, not kept in L1.  Plain
// (non-volatile) asm: the compiler may issue them as early as it likes.
__device__ __forceinline__ uint16_t ld_stream(const uint16_t *p, uint64_t pol) {
  unsigned short v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_stream16(const void *p, uint64_t pol) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}
// Messages are written once per sweep and read back by the next: evict-last.
// No "memory" clobber: nothing in the kernel reads what these stores write.
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol));
}
__device__ __forceinline__ void st_keep(__nv_bfloat16 *p, float v, uint64_t pol) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const unsigned short u = *reinterpret_cast<const unsigned short *>(&h);
  asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(u), "l"(pol));
}
__device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
// Eight consecutive elements of a receive stage in shared memory (16-byte aligned).
__device__ __forceinline__ void load8_smem(const float *p, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8_smem(const __nv_bfloat16 *p, float (&v)[8]) {
  const uint4 a = *reinterpret_cast<const uint4 *>(p);
  const uint32_t u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&u[j]);
    v[2 * j] = __low2float(h);
    v[2 * j + 1] = __high2float(h);
  }
}

// Window wi's range [R0[wi], R0[wi+1]) of `src` into shared memory at dst:
// one bulk copy completing on the mbarrier bar (thread 0 only).
template <class T>
__device__ __forceinline__ void issue_range(const int32_t *R0, const T *src, int32_t wi, uint32_t dst,
                                            uint32_t bar, uint64_t pol) {
  const int32_t r0 = R0[wi], r1 = R0[wi + 1];
  const uint32_t bytes = static_cast<uint32_t>(r1 - r0) * static_cast<uint32_t>(sizeof(T));
  mbar_expect_tx(bar, bytes);
  if (bytes) bulk_g2s_hint(dst, src + r0, bytes, bar, pol);
}

// Input of a window sweep: none (the first sweep of an inner solve), the
// slot layout (the sweep after a freeze), or the receive-ordered buffer.
constexpr int kInZero = 0, kInSlots = 1, kInStaged = 2;

// The sweep over this CTA's windows, specialised on its input, on whether it
// copies c into send order and on damping (all three are the same for the
// whole launch): the common case -- staged input, no copy, no damping --
// keeps no dead branches in its inner loops.
template <class T, int IN, bool REFRESH, bool DAMP>
__device__ __forceinline__ void win_sweep(const GraphView &g, const WinView &w, const Buffers &B,
                                          Ctl *ctl, DevScalars *red, unsigned char *smem,
                                          uint64_t *bars) {
  T *recv = reinterpret_cast<T *>(smem);                                        // receive range
  uint16_t *om = reinterpret_cast<uint16_t *>(smem + w.off_om);                 // outmap
  float *cqs = reinterpret_cast<float *>(smem + w.off_cq);                      // cq
  float *slot = reinterpret_cast<float *>(smem + w.off_slot);                   // the window's slots
  int32_t *rstart = reinterpret_cast<int32_t *>(smem + w.off_rows);             // row starts (+ end)
  float *rowv = reinterpret_cast<float *>(smem + w.off_rows + 4 * (w.rcap + 1)); // row sums, then h~
  int2 *srt = reinterpret_cast<int2 *>(smem + w.off_srt);                       // send runs + sentinel
  uint32_t *rbits = reinterpret_cast<uint32_t *>(smem + w.off_bits);            // run starts (bitmap)
  const int pe = ctl->par_e, pmon = ctl->par_mon;
  constexpr bool zin = IN == kInZero;        // incoming messages known to be zero
  constexpr bool slots_in = REFRESH;         // c into send order (first sweep after a freeze)
  constexpr bool staged = IN == kInStaged;   // input from the receive-ordered buffer
  const double inv_rn = ctl->inv_rn;
  // (the parity selects with ?: -- indexing a kernel parameter's array with a
  // runtime value would copy the parameter to local memory)
  const T *__restrict__ bin_in = static_cast<const T *>(pe ? w.bins[1] : w.bins[0]);
  T *__restrict__ bin_out = static_cast<T *>(pe ? w.bins[0] : w.bins[1]);
  const T *__restrict__ eslot = static_cast<const T *>(pe ? B.e[1] : B.e[0]);
  const float2 *__restrict__ mon_prev = pmon ? B.mon32[1] : B.mon32[0];
  float2 *__restrict__ mon_out = pmon ? B.mon32[0] : B.mon32[1];
  const float gam = static_cast<float>(ctl->damping);
  const int NT = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NT >> 5;
  const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
  uint32_t mdd = 0, md = 0;
  const uint32_t bar_r = smem_u32(&bars[0]), bar_s = smem_u32(&bars[1]);
  if (tid == 0) {
    mbar_init(bar_r, 1);
    mbar_init(bar_s, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // parity of the copy each barrier still waits for (-1: none); every thread
  // keeps the same bookkeeping, thread 0 issues
  int pend_r = -1, pend_s = -1;
  if (staged && static_cast<int32_t>(blockIdx.x) < w.nwin) {
    if (tid == 0) issue_range(w.R0, bin_in, blockIdx.x, smem_u32(recv), bar_r, pol_keep);
    pend_r = 0;
  }

  int j = 0;
  bool failed = false;
  for (int32_t wi = blockIdx.x; wi < w.nwin; wi += gridDim.x, ++j) {
    const int32_t nx = wi + gridDim.x;
    // send streams of this window (their buffers were last read before the
    // barrier that ended the previous window)
    if (tid == 0) {
      fence_proxy_async();
      const int32_t a = w.R0[wi], bnd = w.R0[wi + 1];
      const uint32_t nb = static_cast<uint32_t>(bnd - a);
      mbar_expect_tx(bar_s, nb * 6u);
      if (nb) {
        bulk_g2s_hint(smem_u32(om), w.outmap + a, nb * 2u, bar_s, pol_stream);
        bulk_g2s_hint(smem_u32(cqs), w.cq + a, nb * 4u, bar_s, pol_stream);
      }
    }
    pend_s = j & 1;
    const int2 lo = w.win[wi], hi = w.win[wi + 1];
    const int32_t r0 = lo.x, s0 = lo.y, ns = hi.y - lo.y, nr = hi.x - lo.x;
    // this thread's rows (at most kWinRowsPerThread): their data now, used
    // in B; the row starts go to shared memory after the scatter below, so
    // that these loads overlap it
    float p_rhs[kWinRowsPerThread], p_invP[kWinRowsPerThread], p_prev[kWinRowsPerThread];
    int32_t p_rp[kWinRowsPerThread];
#pragma unroll
    for (int u = 0; u < kWinRowsPerThread; ++u) {
      const int32_t k = tid + u * NT;
      p_rhs[u] = 0.f;
      p_invP[u] = 0.f;
      p_prev[u] = 0.f;
      p_rp[u] = 0;
      if (k < nr) {
        const int32_t i = r0 + k;
        p_rp[u] = g.rp[i];
        p_rhs[u] = zin ? static_cast<float>(B.r64[i] * inv_rn) : B.rhs32[i];
        p_invP[u] = B.invP32[i];
        p_prev[u] = zin ? 0.f : mon_prev[i].y;
      }
    }
    const int32_t nsr = w.srun_ptr[wi + 1] - w.srun_ptr[wi];
    {
      const int32_t sb = w.srun_ptr[wi];
      for (int32_t k = tid; k < nsr; k += NT) srt[k] = w.sruns[sb + k];
      if (tid == 0) srt[nsr] = make_int2(ns, 0);   // sentinel: runs end at ns
      for (int32_t k = tid; k < w.nbits; k += NT) rbits[k] = 0u;
    }

    // ---- A: incoming messages into shared memory, slot order ----
    if (IN == kInSlots) {
      for (int32_t k = tid; k < ns; k += NT) slot[k] = ld_eta(eslot + s0 + k);
    } else if (staged) {
      const bool got = mbar_wait(bar_r, j & 1);
      if (__syncthreads_or(!got)) { failed = true; break; }
      pend_r = -1;
      const int32_t rb = w.R0[wi];
      for (int32_t g8 = tid; 8 * g8 < ns; g8 += NT) {
        const uint4 pv = ld_stream16(w.p2 + rb + 8 * g8, pol_stream);
        const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w};
        float v[8];
        load8_smem(recv + 8 * g8, v);   // the stage is padded to whole groups of 8
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int32_t k = 8 * g8 + jj;
          if (k < ns) slot[(pw[jj >> 1] >> (16 * (jj & 1))) & 0xFFFFu] = v[jj];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kWinRowsPerThread; ++u) {
      const int32_t k = tid + u * NT;
      if (k < nr) rstart[k] = p_rp[u] - s0;
    }
    if (tid == 0) rstart[nr] = ns;
    __syncthreads();
    // the receive stage is free: the next window's range streams in during B and C
    if (staged && nx < w.nwin) {
      if (tid == 0) {
        fence_proxy_async();
        issue_range(w.R0, bin_in, nx, smem_u32(recv), bar_r, pol_keep);
      }
      pend_r = (j + 1) & 1;
    }

    // run starts of the send order as a bitmap (read in C, after B's barrier)
    for (int32_t k = tid; k < nsr; k += NT) atomicOr(&rbits[srt[k].x >> 5], 1u << (srt[k].x & 31));
    // ---- B: node totals, d_i, and h~_i - e for every incoming slot: a
    // thread per row (its data prefetched), the row's slots summed in slot
    // order; rows of degree > 64 first take their sum from a warp each ----
    if constexpr (!zin) {
      for (int32_t hh = w.heavy_ptr[wi] + warp; hh < w.heavy_ptr[wi + 1]; hh += nwarp) {
        const int32_t k = w.heavy_rows[hh] - r0;
        const int32_t rs = rstart[k], re = rstart[k + 1];
        float part = 0.f;
        for (int32_t s = rs + lane; s < re; s += 32) part += slot[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) rowv[k] = part;
      }
      if (w.heavy_ptr[wi + 1] > w.heavy_ptr[wi]) __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kWinRowsPerThread; ++u) {
      const int32_t k = tid + u * NT;
      if (k < nr) {
        const int32_t lr = k, i = r0 + k;
        const int32_t rs = rstart[lr], re = rstart[lr + 1];
        const bool heavy = re - rs > kWinHeavy;
        float sH = 0.f;
        if constexpr (!zin) {
          if (heavy) sH = rowv[lr];
          else
            for (int32_t s = rs; s < re; ++s) sH += slot[s];
        }
        const float Th = p_rhs[u] + sH;
        const float di = Th * p_invP[u];
        mon_out[i] = make_float2(0.f, di);
        mdd = fmax_bits(mdd, di - p_prev[u]);
        md = fmax_bits(md, di);
        if constexpr (zin) B.rhs32[i] = p_rhs[u];
        if (heavy) rowv[lr] = Th;
        else if constexpr (zin)
          for (int32_t s = rs; s < re; ++s) slot[s] = Th;
        else
          for (int32_t s = rs; s < re; ++s) slot[s] = Th - slot[s];
      }
    }
    __syncthreads();
    // the long rows' slots, a warp each
    for (int32_t hh = w.heavy_ptr[wi] + warp; hh < w.heavy_ptr[wi + 1]; hh += nwarp) {
      const int32_t k = w.heavy_rows[hh] - r0;
      const int32_t rs = rstart[k], re = rstart[k + 1];
      const float Th = rowv[k];
      for (int32_t s = rs + lane; s < re; s += 32) slot[s] = zin ? Th : Th - slot[s];
    }
    if (w.heavy_ptr[wi + 1] > w.heavy_ptr[wi]) __syncthreads();
    // ---- C: outgoing messages ----
    {
      const bool got = mbar_wait(bar_s, j & 1);
      if (__syncthreads_or(!got)) { failed = true; break; }
      pend_s = -1;
      // each warp a contiguous range of send positions; the lanes take
      // consecutive positions (so a store instruction writes a contiguous
      // piece of a run), four rounds of 32 at a time.  A position's
      // destination is its run's first receive position plus its offset in
      // the run.
      const int32_t a = w.R0[wi];
      const int32_t per = ((ns + nwarp - 1) / nwarp + 127) & ~127;
      const int32_t qa = warp * per, qb = min(ns, qa + per);
      // run holding the warp's first position; a lane's run is that one plus
      // the run starts between the first position of its 32 and its own
      int32_t rb = 0;
      if (qa < qb) {
        int32_t lo_r = 0, hi_r = nsr - 1;
        while (lo_r < hi_r) {
          const int32_t m = (lo_r + hi_r + 1) >> 1;
          if (srt[m].x <= qa) lo_r = m; else hi_r = m - 1;
        }
        rb = lo_r;
      }
      const uint32_t below = ((2u << lane) - 1u) & ~1u;   // positions 1 .. lane of a word
      for (int32_t q0 = qa; q0 < qb; q0 += 128) {
        int32_t dst[4], sl[4];
        float cc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int32_t qw = q0 + 32 * u, q = qw + lane;
          const uint32_t word = rbits[qw >> 5];
          const int32_t rl = rb + __popc(word & below);
          rb += __popc(word & ~1u) + static_cast<int32_t>(rbits[(qw >> 5) + 1] & 1u);
          dst[u] = 0;
          sl[u] = 0;
          cc[u] = 0.f;
          if (q < qb) {
            const int2 e = srt[rl];
            dst[u] = e.y + (q - e.x);
            sl[u] = om[q];
            cc[u] = cqs[q];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int32_t q = q0 + 32 * u + lane;
          if (q < qb) {
            float c = cc[u];
            if constexpr (slots_in) {   // first sweep after a freeze: c into send order
              c = B.c32[s0 + sl[u]];
              w.cq[a + q] = c;
            }
            float v = c * slot[sl[u]];
            if constexpr (DAMP) {
              float o = 0.f;
              if constexpr (IN == kInSlots) o = ld_eta(eslot + g.rev[s0 + sl[u]]);
              else if constexpr (IN == kInStaged) o = ld_eta(bin_in + dst[u]);
              v = gam * o + (1.f - gam) * v;
            }
            st_keep(bin_out + dst[u], v, pol_keep);
          }
        }
      }
    }
    __syncthreads();   // the next window reuses the shared memory
  }
  if (failed && tid == 0) {
    // a copy that never landed: report it and let the copies still in
    // flight finish (bounded) before the CTA ends
    atomicOr(&red->timeout, 1);
    if (pend_r >= 0) mbar_wait(bar_r, pend_r);
    if (pend_s >= 0) mbar_wait(bar_s, pend_s);
  }
  __syncthreads();
  block_max4(widen(mdd), widen(md), 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
  last_block_control(ctl, red, CK_MEAN);
}

template <class T>
__global__ void __launch_bounds__(kWinBlock, 1)
mean_win_kernel(GraphView g, WinView w, Buffers B, Ctl *ctl, DevScalars *red) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];   // [0]: receive stage, [1]: send streams
  const bool zin = ctl->first != 0, slots = ctl->e_slots != 0, damp = ctl->damping > 0.0;
  if (zin) {
    if (slots) {
      if (damp) win_sweep<T, kInZero, true, true>(g, w, B, ctl, red, smem, bars);
      else win_sweep<T, kInZero, true, false>(g, w, B, ctl, red, smem, bars);
    } else {
      if (damp) win_sweep<T, kInZero, false, true>(g, w, B, ctl, red, smem, bars);
      else win_sweep<T, kInZero, false, false>(g, w, B, ctl, red, smem, bars);
    }
  } else if (slots) {
    if (damp) win_sweep<T, kInSlots, true, true>(g, w, B, ctl, red, smem, bars);
    else win_sweep<T, kInSlots, true, false>(g, w, B, ctl, red, smem, bars);
  } else {
    if (damp) win_sweep<T, kInStaged, false, true>(g, w, B, ctl, red, smem, bars);
    else win_sweep<T, kInStaged, false, false>(g, w, B, ctl, red, smem, bars);
  }
}

constexpr int kWinMaxSmem = 225 * 1024;   // largest dynamic shared memory a handle may use

// CTAs of the kernel per SM with `smem` bytes of windows.  The kernel's
// dynamic shared-memory limit is raised to the largest size any handle may
// use (never lowered: handles of different window sizes share the kernel).
template <class T>
int win_blocks_per_sm(size_t smem) {
  cudaFuncSetAttribute(mean_win_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWinMaxSmem);
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mean_win_kernel<T>, kWinBlock, smem);
  return bps;
}

}  // namespace

WinView Win::view() const {
  WinView v{};
  v.win = win;
  v.R0 = R0;
  v.p2 = p2;
  v.outmap = outmap;
  v.srun_ptr = srun_ptr;
  v.sruns = sruns;
  v.heavy_ptr = heavy_ptr;
  v.heavy_rows = heavy_rows;
  v.cq = cq;
  v.bins[0] = bins[0];
  v.bins[1] = bins[1];
  v.nwin = nwin;
  v.rcap = rcap;
  v.off_om = off_om;
  v.off_cq = off_cq;
  v.off_slot = off_slot;
  v.off_rows = off_rows;
  v.off_srt = off_srt;
  v.off_bits = off_bits;
  v.nbits = nbits;
  return v;
}

void free_windows(Win &W) {
  for (void *p : {static_cast<void *>(W.win), static_cast<void *>(W.R0), static_cast<void *>(W.p2),
                  static_cast<void *>(W.outmap), static_cast<void *>(W.srun_ptr),
                  static_cast<void *>(W.sruns), static_cast<void *>(W.heavy_ptr),
                  static_cast<void *>(W.heavy_rows), static_cast<void *>(W.cq), W.bins[0],
                  W.bins[1]})
    if (p) cudaFree(p);
  W = Win{};
}

namespace {
template <class V>
cudaError_t upload(V **dst, const std::vector<V> &src, cudaStream_t st, size_t pad = 0) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), sizeof(V) * (src.size() + pad + 1));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(*dst, 0, sizeof(V) * (src.size() + pad + 1), st);
  if (e == cudaSuccess && !src.empty())
    e = cudaMemcpyAsync(*dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // src is a host temporary
  return e;
}
}  // namespace

// Windows of about `target` slots (a row longer than that is a window of its
// own); every window's send order (its slots sorted by destination slot
// rev[s]); its receive range (the messages bound for it, grouped by source
// window in window order, each group in destination-slot order) and the
// placement p2 of every element; and every window's send runs (one per
// destination window: first send position, first receive position).  All of
// it depends on the graph only.
gabp_status build_windows(const Graph &g, int32_t target, bool bf16, Win &W, cudaStream_t st,
                          std::string *msg) {
  free_windows(W);
  const int32_t n = g.n;
  const int64_t E = g.E;
  if (g.ncol > 0) { *msg = "window form: synchronous schedule only"; return GABP_ERR_INVALID_ARG; }
  if (E == 0 || target < 32) { *msg = "window form: nothing to exchange"; return GABP_ERR_INVALID_ARG; }
  const std::vector<int32_t> &rp = g.h_rp, &rev = g.h_rev;
  const size_t esz = bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
  // windows: consecutive rows, cut before a row that would take the window
  // past `target` slots
  std::vector<int2> wins;
  int32_t wcap = 0;
  {
    int32_t r = 0;
    while (r < n) {
      const int32_t r0 = r, s0 = rp[r];
      while (r < n && (r == r0 || (rp[r + 1] - s0 <= target && r - r0 < kWinMaxRows))) ++r;
      // rows without slots at the end of a window join it (up to the row cap)
      while (r < n && rp[r + 1] == rp[r] && r - r0 < kWinMaxRows) ++r;
      wins.push_back(make_int2(r0, s0));
      wcap = std::max(wcap, rp[r] - s0);
    }
    wins.push_back(make_int2(n, static_cast<int32_t>(E)));
  }
  const int32_t nwin = static_cast<int32_t>(wins.size()) - 1;
  if (wcap > 65536) { *msg = "window form: a row has more than 65536 slots"; return GABP_ERR_INVALID_ARG; }
  // receive ranges, each padded to a multiple of 8 elements (16-byte aligned copies)
  std::vector<int32_t> R0(nwin + 1, 0);
  for (int32_t k = 0; k < nwin; ++k) R0[k + 1] = R0[k] + ((wins[k + 1].y - wins[k].y + 7) & ~7);
  const int64_t R = R0[nwin];
  std::vector<int32_t> wos(E);   // window of every slot
  for (int32_t k = 0; k < nwin; ++k)
    std::fill(wos.begin() + wins[k].y, wos.begin() + wins[k + 1].y, k);
  // send order: for increasing destination d, the sender slot s = rev[d]
  // takes the next send position of its window (qpos: window-local);
  // outmap and cq are kept in the padded range space of R0, so that a
  // window's streams are whole 16-byte-aligned bulk copies
  std::vector<uint16_t> outmap(R, 0);
  std::vector<int32_t> qpos(E), cursor(nwin, 0);
  for (int64_t d = 0; d < E; ++d) {
    const int32_t s = rev[d], I = wos[s];
    const int32_t q = cursor[I]++;
    outmap[R0[I] + q] = static_cast<uint16_t>(s - wins[I].y);
    qpos[s] = q;
  }
  // receive ranges (counting sort of each window's destination slots by the
  // window of their sender; stable in d) and the send runs they define
  std::vector<uint16_t> p2(R, 0);
  std::vector<std::vector<int2>> send(nwin);   // per sender: (first send position, first receive position)
  std::vector<int32_t> cnt(nwin, 0), first(nwin, 0), pos(nwin, 0), touched;
  for (int32_t J = 0; J < nwin; ++J) {
    const int32_t a = wins[J].y, b = wins[J + 1].y;
    touched.clear();
    for (int32_t d = a; d < b; ++d) {
      const int32_t I = wos[rev[d]];
      if (cnt[I]++ == 0) { touched.push_back(I); first[I] = d; }
    }
    std::sort(touched.begin(), touched.end());
    int32_t cat = 0;
    for (int32_t I : touched) {
      send[I].push_back(make_int2(qpos[rev[first[I]]], R0[J] + cat));
      pos[I] = cat;
      cat += cnt[I];
    }
    for (int32_t d = a; d < b; ++d) {
      const int32_t I = wos[rev[d]];
      p2[R0[J] + pos[I]++] = static_cast<uint16_t>(d - a);
    }
    for (int32_t I : touched) cnt[I] = 0;
  }
  std::vector<int32_t> srun_ptr(nwin + 1, 0);
  std::vector<int2> sruns;
  int32_t runcap = 0;
  for (int32_t I = 0; I < nwin; ++I) {
    // destination windows were visited in increasing order, so the runs of
    // I are in send order already
    sruns.insert(sruns.end(), send[I].begin(), send[I].end());
    srun_ptr[I + 1] = static_cast<int32_t>(sruns.size());
    runcap = std::max(runcap, static_cast<int32_t>(send[I].size()));
  }
  // rows of degree > kWinHeavy: a warp each
  std::vector<int32_t> heavy_ptr(nwin + 1, 0), heavy_rows;
  for (int32_t J = 0; J < nwin; ++J) {
    for (int32_t i = wins[J].x; i < wins[J + 1].x; ++i)
      if (rp[i + 1] - rp[i] > kWinHeavy) heavy_rows.push_back(i);
    heavy_ptr[J + 1] = static_cast<int32_t>(heavy_rows.size());
  }
  int32_t ecap = 0, rowcap = 0;   // largest padded range, most rows of a window
  for (int32_t k = 0; k < nwin; ++k) {
    ecap = std::max(ecap, R0[k + 1] - R0[k]);
    rowcap = std::max(rowcap, wins[k + 1].x - wins[k].x);
  }
  auto r128 = [](size_t b) { return (b + 127) & ~size_t{127}; };
  const size_t off_om = r128(static_cast<size_t>(ecap) * esz);
  const size_t off_cq = off_om + r128(static_cast<size_t>(ecap) * 2);
  const size_t off_slot = off_cq + r128(static_cast<size_t>(ecap) * 4);
  const size_t off_rows = off_slot + r128(static_cast<size_t>(wcap) * 4);
  const size_t off_srt = off_rows + r128(static_cast<size_t>(2 * rowcap + 1) * 4);
  const size_t off_bits = off_srt + r128(sizeof(int2) * (static_cast<size_t>(runcap) + 1));
  const int32_t nbits = (ecap + 31) / 32 + 8;   // the send loop reads a word past its last position
  const size_t smem = off_bits + sizeof(uint32_t) * static_cast<size_t>(nbits);
  if (smem > static_cast<size_t>(kWinMaxSmem)) {
    *msg = "window form: a window does not fit shared memory";
    return GABP_ERR_INVALID_ARG;
  }
  const int bps = bf16 ? win_blocks_per_sm<__nv_bfloat16>(smem) : win_blocks_per_sm<float>(smem);
  if (bps < 1) { *msg = "window form: no CTA fits an SM"; return GABP_ERR_INVALID_ARG; }
  cudaError_t e = cudaSuccess;
  auto up = [&](auto **dst, const auto &src, size_t pad) {
    if (e == cudaSuccess) e = upload(dst, src, st, pad);
  };
  up(&W.win, wins, 0);
  up(&W.R0, R0, 0);
  up(&W.p2, p2, kPad);
  up(&W.outmap, outmap, kPad);
  up(&W.srun_ptr, srun_ptr, 0);
  up(&W.sruns, sruns, 0);
  up(&W.heavy_ptr, heavy_ptr, 0);
  up(&W.heavy_rows, heavy_rows, 0);
  if (e == cudaSuccess) e = cudaMalloc(&W.cq, sizeof(float) * (R + kPad));
  if (e == cudaSuccess) e = cudaMemsetAsync(W.cq, 0, sizeof(float) * (R + kPad), st);
  for (int k = 0; k < 2; ++k) {
    if (e == cudaSuccess) e = cudaMalloc(&W.bins[k], esz * (R + kPad));
    if (e == cudaSuccess) e = cudaMemsetAsync(W.bins[k], 0, esz * (R + kPad), st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_windows(W);
    *msg = std::string("window form: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA;
  }
  W.nwin = nwin;
  W.wcap = wcap;
  W.runcap = runcap;
  W.target = target;
  W.rcap = rowcap;
  W.off_om = static_cast<int32_t>(off_om);
  W.off_cq = static_cast<int32_t>(off_cq);
  W.off_slot = static_cast<int32_t>(off_slot);
  W.off_rows = static_cast<int32_t>(off_rows);
  W.off_srt = static_cast<int32_t>(off_srt);
  W.off_bits = static_cast<int32_t>(off_bits);
  W.nbits = nbits;
  W.smem = smem;
  W.blocks = bps;
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    W.grid = std::max(1, std::min(nwin, std::max(sms, 1) * bps));
  }
  W.nruns = static_cast<int64_t>(sruns.size());
  return GABP_OK;
}

int launch_mean_win(const Graph &g, const Win &W, cudaStream_t st, Buffers B, Ctl *ctl,
                    DevScalars *red, bool bf16) {
  if (bf16)
    mean_win_kernel<__nv_bfloat16><<<W.grid, kWinBlock, W.smem, st>>>(g.view(), W.view(), B, ctl, red);
  else
    mean_win_kernel<float><<<W.grid, kWinBlock, W.smem, st>>>(g.view(), W.view(), B, ctl, red);
  return 1;
}

}  // namespace gabp
