// gabp_selfcheck.cu -- a diagnostic with no counterpart in the paper: a
// bounded device wait that can never be satisfied ends, and surfaces as
// GABP_ERR_TIMEOUT through the controller path the sweeps use, with the
// context still usable afterwards.
//
// The sweeps stage their tiles with cp.async.bulk on an mbarrier and wait for
// it for at most kWaitLimitNs of global time; a wait that gives up sets the
// `timeout` reduction flag, and the controller ends the solve with
// GABP_ERR_TIMEOUT.  The kernel below makes that wait run out on purpose: one
// warp waits, with the sweeps' own bounded wait, on an mbarrier that nothing
// ever arrives on (no copy is issued, so nothing is in flight when the
// kernel returns), for a time the caller chooses up to that limit, then
// reports exactly as a sweep would.
#include "gabp_internal.h"
#include "gabp_device.cuh"

namespace gabp {
namespace {

__global__ void wait_limit_kernel(Ctl *ctl, DevScalars *red, unsigned long long limit_ns,
                                  unsigned long long *ns) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);   // one arrival expected; none ever comes
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned long long t0 = global_timer_ns();
  const bool got = mbar_wait_for(b, 0, limit_ns);
  const unsigned long long t1 = global_timer_ns();
  if (threadIdx.x == 0) {
    *ns = t1 - t0;
    if (!got) atomicOr(&red->timeout, 1);
  }
  last_block_control(ctl, red, CK_SWEEP64);
}

}  // namespace

int launch_wait_limit(cudaStream_t st, Ctl *ctl, DevScalars *red, unsigned long long limit_ns,
                      unsigned long long *ns) {
  wait_limit_kernel<<<1, 32, 0, st>>>(ctl, red, limit_ns, ns);
  return 1;
}

}  // namespace gabp
