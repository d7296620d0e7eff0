// gabp_resident.cu -- whole FP64 solves of small systems in one launch.
//
// A system whose messages fit in the shared memory of one thread-block
// cluster (up to 16 CTAs on 16 SMs) is solved by a single kernel: the rows
// are split into C contiguous parts, CTA c keeps the incoming messages of its
// rows (both buffers of the synchronous schedule, Section III-C) in its own
// shared memory, and each sweep of Alg. 2 stores every new message straight
// into the shared memory of the CTA that owns its destination row
// (distributed shared memory).  A cluster barrier separates the sweeps.
// Every `check_every` sweeps the tentative means x_i = h~_i / P~_i are
// written, the FP64 residual ||b - A x||_inf is formed (neighbour x read from
// the owning CTA), the CTAs' maxima are gathered in CTA 0 and every CTA takes
// the same stop decision from them.  No host round trip and no launch per
// sweep: the cost of a sweep is its FP64 arithmetic plus one barrier.
//
// The arithmetic per message is that of the CSR FP64 sweep (same reciprocal,
// same damping rule), so a solve stops after the same number of sweeps.
//
// Colour schedule (v.ncol > 0): the rows are renumbered by colour class and
// a sweep is one pass per class, each followed by a cluster barrier.  A pass
// reads and writes the single message buffer in place: nodes of a class are
// not adjacent, so no slot is read and written by the same pass.  The
// buffer starts from zero, and the means of a class are taken at its pass.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace gabp {
namespace {

namespace cg = cooperative_groups;

constexpr int kResBlock = 256;

// Shared-memory layout of every CTA of the cluster (the same offsets in all,
// so a remote address is the local offset in another CTA's window).
struct ResLayout {
  uint32_t m0, m1, a, dst, colp, lrow, lrp, dg, bb, tp, r0, r1, r2, y0, y1, red, bytes;
};
__host__ __device__ inline ResLayout res_layout(int smax, int rmax) {
  ResLayout L;
  auto up = [](uint32_t v) { return (v + 15u) & ~15u; };
  L.m0 = 0;
  L.m1 = up(L.m0 + 16u * smax);
  L.a = up(L.m1 + 16u * smax);
  L.dst = up(L.a + 8u * smax);
  L.colp = up(L.dst + 4u * smax);
  L.lrow = up(L.colp + 4u * smax);
  L.lrp = up(L.lrow + 2u * smax);
  L.dg = up(L.lrp + 4u * (rmax + 1));
  L.bb = up(L.dg + 8u * rmax);
  L.tp = up(L.bb + 8u * rmax);
  L.r0 = up(L.tp + 16u * rmax);   // Aitken ring of tentative means
  L.r1 = up(L.r0 + 8u * rmax);
  L.r2 = up(L.r1 + 8u * rmax);
  L.y0 = up(L.r2 + 8u * rmax);     // checked means (extrapolated or not), by check parity
  L.y1 = up(L.y0 + 8u * rmax);
  L.red = up(L.y1 + 8u * rmax);
  L.bytes = up(L.red + 8u * 4 * kResidentMaxCluster);
  return L;
}

// One sweep = (rows) node totals, and x when this sweep is checked;
// (slots) one message per thread, stored into the owning CTA; one cluster
// barrier.  A check's residual is formed right after that barrier and its
// maximum parked in CTA 0; the stop decision is read after the next sweep's
// barrier (so a check adds no barrier of its own).  Reduction slots and x
// are double-buffered by check parity, so a decision always sees the x and
// the maxima of its own check.
__global__ void __launch_bounds__(kResBlock) resident64_kernel(ResidentView v) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char sm[];
  const ResLayout L = res_layout(v.smax, v.rmax);
  const int me = static_cast<int>(cl.block_rank());
  const int C = static_cast<int>(cl.num_blocks());
  const int r0 = v.row0[me], R = v.row0[me + 1] - r0;
  const int32_t s0 = v.rp[r0], S = v.rp[r0 + R] - s0;
  double2 *m[2] = {reinterpret_cast<double2 *>(sm + L.m0), reinterpret_cast<double2 *>(sm + L.m1)};
  double *a = reinterpret_cast<double *>(sm + L.a);
  int32_t *dst = reinterpret_cast<int32_t *>(sm + L.dst);
  int32_t *colp = reinterpret_cast<int32_t *>(sm + L.colp);
  uint16_t *lrow = reinterpret_cast<uint16_t *>(sm + L.lrow);
  int32_t *lrp = reinterpret_cast<int32_t *>(sm + L.lrp);
  double *dg = reinterpret_cast<double *>(sm + L.dg);
  double *bb = reinterpret_cast<double *>(sm + L.bb);
  double2 *tp = reinterpret_cast<double2 *>(sm + L.tp);   // (P~_i, h~_i) of this sweep
  double *ring[3] = {reinterpret_cast<double *>(sm + L.r0), reinterpret_cast<double *>(sm + L.r1),
                     reinterpret_cast<double *>(sm + L.r2)};
  double *xs[2] = {reinterpret_cast<double *>(sm + L.y0), reinterpret_cast<double *>(sm + L.y1)};
  double *red = reinterpret_cast<double *>(sm + L.red);   // CTA 0: [parity][max r | breakdown][C]
  const int tid = threadIdx.x;
  __shared__ unsigned long long part[2];

  // ---- load this CTA's rows and slots; max |b| over the cluster ----
  unsigned long long mb = 0;
  for (int k = tid; k < R; k += kResBlock) {
    const int32_t i = r0 + k;
    const int32_t rs = v.rp[i] - s0, re = v.rp[i + 1] - s0;
    lrp[k] = rs;
    for (int32_t s = rs; s < re; ++s) lrow[s] = static_cast<uint16_t>(k);
    dg[k] = v.diag64[i];
    bb[k] = v.b[i];
    mb = umax(mb, bits(fabs(bb[k])));
  }
  if (tid == 0) lrp[R] = S;
  const bool colour = v.ncol > 0;
  for (int32_t s = tid; s < S; s += kResBlock) {
    a[s] = v.a64[s0 + s];
    dst[s] = v.dst[s0 + s];
    colp[s] = v.colp[s0 + s];
    if (colour) m[0][s] = make_double2(0.0, 0.0);   // read before written by later classes
  }
  if (tid < 2) part[tid] = 0;
  __syncthreads();
  mb = warp_max(mb);
  if ((tid & 31) == 0 && mb) atomicMax(&part[0], mb);
  __syncthreads();
  double *red0 = cl.map_shared_rank(red, 0);
  if (tid == 0) red0[me] = dv(part[0]);
  cl.sync();
  double bnorm = 0.0;
  for (int c = 0; c < C; ++c) bnorm = fmax(bnorm, red0[c]);
  const double thr = v.rel ? v.tol * bnorm : v.tol;
  cl.sync();   // red0 is rewritten by the first check

  const double gam = v.damping;
  const int ait = v.aitken;   // Delta^2 stride (0 = off)
  int nw = 0;                 // tentative means written to the ring
  int status = GABP_ERR_NOT_CONVERGED, checks = 0, sweeps = 0, pending = -1, pending_sweeps = 0;
  double rn = bnorm;
  bool brk = false;
  // Reads the maxima of check `c` from CTA 0 and decides: 1 = stop.
  auto decide = [&](int c) {
    const double *rr = red0 + (c & 1) * 2 * kResidentMaxCluster;
    double worst = 0.0;
    bool any_brk = false;
    for (int k = 0; k < C; ++k) {
      worst = isfinite(rr[k]) ? fmax(worst, rr[k]) : INFINITY;
      any_brk |= rr[kResidentMaxCluster + k] != 0.0;
      if (!isfinite(worst)) break;
    }
    rn = worst;
    sweeps = pending_sweeps;
    if (any_brk) { status = GABP_ERR_BREAKDOWN; return true; }
    if (rn < thr) { status = GABP_OK; return true; }
    if (!isfinite(rn) || rn > 1e30 * fmax(bnorm, DBL_MIN)) { status = GABP_ERR_DIVERGED; return true; }
    return false;
  };
  const int passes = colour ? v.ncol : 1;
  for (int it = 0; it < v.max_iter; ++it) {
    const int cur = it & 1;
    // messages known to be zero: the first synchronous sweep (the colour
    // schedule reads its zeroed buffer instead)
    const bool zin = it == 0 && !colour;
    const bool write_x = ((it + 1) % v.check_every == 0) || it + 1 >= v.max_iter;   // a check
    const bool to_ring = ait > 0 && (write_x || (it + 1) % ait == 0);
    double *xw = xs[checks & 1];
    double *rw = ring[nw % 3];
    const double *rp1 = ring[(nw + 2) % 3], *rp2 = ring[(nw + 1) % 3];   // written 1 and 2 steps ago
    double2 *m_in = colour ? m[0] : m[cur];
    double2 *m_out = colour ? m[0] : m[cur ^ 1];
    for (int c = 0; c < passes; ++c) {
      // this pass's rows: all of them, or those of colour class c
      const int k0 = colour ? min(max(v.cb[c] - r0, 0), R) : 0;
      const int k1 = colour ? min(max(v.cb[c + 1] - r0, 0), R) : R;
      const double gam_c = (colour && v.damp_last && c + 1 < passes) ? 0.0 : gam;
      for (int k = k0 + tid; k < k1; k += kResBlock) {
        double sP = 0.0, sH = 0.0;
        if (!zin)
          for (int32_t s = lrp[k]; s < lrp[k + 1]; ++s) {
            sP += m_in[s].x;
            sH += m_in[s].y;
          }
        const double TP = dg[k] + sP, Th = bb[k] + sH;
        tp[k] = make_double2(TP, Th);
        if (to_ring || write_x) {
          const double xi = Th / TP;
          if (to_ring) rw[k] = xi;
          if (write_x) {
            double y = xi;
            if (ait > 0 && nw >= 2) {   // Delta^2 of the means of rounds t - 2s, t - s, t
              const double c0 = rp2[k], c1 = rp1[k];
              const double d1 = c1 - c0, den = (xi - c1) - d1;
              const double scale = fmax(fmax(fabs(c0), fabs(c1)), fabs(xi));
              if (fabs(den) > 64.0 * DBL_EPSILON * scale) y = c0 - d1 * d1 / den;
            }
            xw[k] = y;
          }
        }
      }
      __syncthreads();
      for (int32_t s = lrp[k0] + tid; s < lrp[k1]; s += kResBlock) {
        const double2 t = tp[lrow[s]];
        const double2 mi = zin ? make_double2(0.0, 0.0) : m_in[s];
        const double d = t.x - mi.x;   // P~_i - P_ji
        brk |= zero_or_nonfinite(d);
        const double as = a[s], inv = recip64(d);
        const int32_t to = dst[s];
        double eta = -as * (t.y - mi.y) * inv;
        if (gam_c > 0.0) {
          const double old = zin ? 0.0 : cl.map_shared_rank(m_in, to >> 24)[to & 0xFFFFFF].y;
          eta = gam_c * old + (1.0 - gam_c) * eta;
        }
        cl.map_shared_rank(m_out, to >> 24)[to & 0xFFFFFF] = make_double2(-(as * as) * inv, eta);
      }
      cl.sync();   // this pass's messages delivered everywhere (the last: round it + 1; x visible)
    }
    if (to_ring) ++nw;
    if (pending >= 0) {
      const bool stop = decide(pending);
      pending = -1;
      if (stop) break;
    }
    if (!write_x) continue;
    // ---- residual of x: neighbour x read from the owning CTA ----
    unsigned long long mr = 0;
    for (int k = tid; k < R; k += kResBlock) {
      double acc = 0.0;
      for (int32_t s = lrp[k]; s < lrp[k + 1]; ++s) {
        const int32_t cp = colp[s];
        acc += a[s] * cl.map_shared_rank(xw, cp >> 16)[cp & 0xFFFF];
      }
      const double ri = bb[k] - (dg[k] * xw[k] + acc);
      mr = umax(mr, bits(fabs(ri)));
    }
    mr = warp_max(mr);
    if (tid == 0) part[1] = 0;
    const bool brk_cta = __syncthreads_or(brk) != 0;
    if ((tid & 31) == 0 && mr) atomicMax(&part[1], mr);
    __syncthreads();
    if (tid == 0) {
      double *rr = red0 + (checks & 1) * 2 * kResidentMaxCluster;
      rr[me] = dv(part[1]);
      rr[kResidentMaxCluster + me] = brk_cta ? 1.0 : 0.0;
    }
    pending = checks++;
    pending_sweeps = it + 1;
  }
  if (pending >= 0) {   // the last check (at max_iter) is decided here
    cl.sync();
    decide(pending);
  }
  const double *xf = xs[(checks - 1) & 1];
  if (checks > 0)
    for (int k = tid; k < R; k += kResBlock) v.x[r0 + k] = xf[k];
  if (me == 0 && tid == 0) {
    v.out->status = status;
    v.out->sweeps = sweeps;
    v.out->checks = checks;
    v.out->residual = rn;
    v.out->bnorm = bnorm;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace

uint32_t resident_smem_bytes(int smax, int rmax) { return res_layout(smax, rmax).bytes; }

// Launches one cluster of `C` CTAs.  Returns cudaErrorInvalidConfiguration
// (with the error state cleared) when this device cannot place such a
// cluster with that shared memory.
cudaError_t launch_resident64(const ResidentView &v, int C, cudaStream_t st) {
  const uint32_t smem = resident_smem_bytes(v.smax, v.rmax);
  auto cannot = [] {
    cudaGetLastError();
    return cudaErrorInvalidConfiguration;
  };
  if (cudaFuncSetAttribute(resident64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return cannot();
  if (C > 8 && cudaFuncSetAttribute(resident64_kernel,
                                    cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return cannot();
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kResBlock, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, resident64_kernel, &cfg) != cudaSuccess ||
      clusters < 1)
    return cannot();
  return cudaLaunchKernelEx(&cfg, resident64_kernel, v);
}

}  // namespace gabp
