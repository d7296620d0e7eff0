// gabp_naive.cu -- FP64 sweeps by Algorithm 1, the naive form (option naive),
// as a cross-check of the broadcast kernels of gabp_kernels.cu.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <algorithm>

namespace gabp {
namespace {

// ---------------------------------------------------------------------------
// FP64 round of Algorithm 1, the naive form (option naive): for every
// directed edge i -> j the cavity sums
//     P_{i\j} = A_ii + sum_{k in N(i)\j} P_ki,   h_{i\j} = b_i + sum_{k in N(i)\j} eta_ki
// are added up over the other incoming messages directly, O(deg^2) per row,
// instead of node total minus reverse message (Algorithm 2).  It is the same
// round without that cancellation, so it cross-checks the broadcast kernels
// on the same data.  One warp per row, lanes over the row's slots, each sum
// in slot order; the tentative mean x_i = h~_i / P~_i uses every incoming
// message.  Synchronous schedule, undamped.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) naive64_kernel(GraphView g, Buffers B, Ctl *ctl, DevScalars *red) {
  const int par = ctl->par_m;
  const bool first = ctl->first != 0;   // incoming messages are zero
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
  double *__restrict__ x = ctl->xw;
  const double2 *__restrict__ min = (par ? B.m64[1] : B.m64[0]);
  double2 *__restrict__ mout = (par ? B.m64[0] : B.m64[1]);
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  bool brk = false;
  for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32; i < g.n;
       i += warps) {
    const int32_t rs = g.rp[i], re = g.rp[i + 1];
    const double dgi = g.diag64[i], bi = b[i];
    if (write_x && lane == 0) {
      double P = dgi, H = bi;
      if (!first)
        for (int32_t t = rs; t < re; ++t) {
          P += min[t].x;
          H += min[t].y;
        }
      x[i] = H / P;
    }
    if (!write_msgs) continue;
    for (int32_t s = rs + lane; s < re; s += 32) {
      double P = dgi, H = bi;   // P_ii = A_ii and P_ii mu_ii = b_i
      if (!first)
        for (int32_t t = rs; t < re; ++t)
          if (t != s) {
            P += min[t].x;
            H += min[t].y;
          }
      brk |= zero_or_nonfinite(P);
      const double a = g.a64[s];
      mout[g.rev[s]] = make_double2(-(a * a) / P, -a * H / P);
    }
  }
  if (brk) atomicOr(&red->breakdown, 1);
  last_block_control(ctl, red, CK_SWEEP64);
}

}  // namespace

int launch_naive64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  // one warp per row, at most eight 256-thread blocks per SM in flight
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);   // the handle's device is current while it launches
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (static_cast<int64_t>(g.n) * 32 + kBlock - 1) / kBlock;
  const int64_t cap = static_cast<int64_t>(std::max(sms, 1)) * 8;
  naive64_kernel<<<static_cast<int>(std::max<int64_t>(1, std::min(blocks, cap))), kBlock, 0, st>>>(
      g.view(), B, ctl, red);
  return 1;
}

}  // namespace gabp
