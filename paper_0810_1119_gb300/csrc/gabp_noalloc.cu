// gabp_noalloc.cu -- gabp_run_rounds_noalloc: synchronous FP64 GaBP rounds
// without any device allocation.
//
// Who needs this: callers that must not allocate device memory at the
// moment they call us -- applications that reserve all of their device
// memory up front (a serving process whose memory pool owns the whole GPU,
// where a late cudaMalloc fails or must not happen), code that runs inside
// an allocator or memory-pool callback and cannot re-enter the allocator,
// and latency-critical loops where cudaMalloc/cudaFree would synchronise
// the device.  Such callers already own their inputs and outputs; what they
// cannot provide on demand is our working space.  This entry point
// therefore keeps its working space (the two message buffers of the
// parallel schedule) in one fixed, file-scope device array that exists from
// the moment the library's module is loaded on a GPU until the process
// exits (or the device is reset).
//
// The computation is the same as gabp_run_rounds: `rounds` synchronous
// rounds of the broadcast form from zero messages, then the tentative means.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/gabp.h"

namespace {

// Largest CSR (entries including the diagonal) the array can serve.
constexpr int64_t kNoAllocMaxEntries = int64_t{1} << 18;

// Working space shared by every call on a device: two message buffers of
// (P, P mu) pairs, laid out per CSR entry, plus one breakdown flag word.
// 2 * 2^18 * 16 B + 256 B = 8 MiB + 256 B per GPU that loads the library.
static __device__ __align__(256) double2 g_noalloc_scratch[2 * kNoAllocMaxEntries + 16];

// One round for row i (a thread per row).  Entry e = (i, j), j != i, holds
// the message travelling INTO i from j in `in`; the message i -> j is written
// to entry rev[e] = (j, i) of `out`.  first = 1: all incoming messages are
// zero (round 1) and `in` is not read.  infer = 1: only x_i is written.
__global__ void noalloc_round_kernel(int64_t n, const int64_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col,
                                     const double *__restrict__ val,
                                     const int64_t *__restrict__ rev,
                                     const double *__restrict__ b, const double2 *__restrict__ in,
                                     double2 *__restrict__ out, double *__restrict__ x,
                                     int *breakdown, int first, int infer) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
    double aii = 0.0, sP = 0.0, sH = 0.0;
    for (int64_t e = rs; e < re; ++e) {
      if (col[e] == i) { aii = val[e]; continue; }
      if (!first) { sP += in[e].x; sH += in[e].y; }
    }
    const double TP = aii + sP, Th = b[i] + sH;   // P~_i, h~_i = P~_i mu~_i
    if (infer) { x[i] = Th / TP; continue; }
    for (int64_t e = rs; e < re; ++e) {
      if (col[e] == i) continue;
      const double2 m = first ? make_double2(0.0, 0.0) : in[e];   // m_{j->i}
      const double d = TP - m.x;                                   // P~_i - P_ji
      if (!(d != 0.0) || !isfinite(d)) atomicOr(breakdown, 1);
      const double a = val[e];
      out[rev[e]] = make_double2(-(a * a) / d, -a * (Th - m.y) / d);
    }
  }
}

}  // namespace

namespace gabp {
void set_thread_error(const std::string &msg);   // gabp_solve.cu: read by gabp_last_error(NULL)
}

namespace {
gabp_status fail(gabp_status s, const std::string &msg) {
  gabp::set_thread_error(msg);
  return s;
}
}  // namespace

extern "C" gabp_status gabp_run_rounds_noalloc(int64_t n, int64_t nnz, const int64_t *row_ptr_dev,
                                               const int32_t *col_dev, const double *val_dev,
                                               const int64_t *rev_dev, const double *b_dev,
                                               int32_t rounds, double *x_dev, void *stream) {
  if (n < 1 || nnz < n || !row_ptr_dev || !col_dev || !val_dev || !rev_dev || !b_dev || !x_dev ||
      rounds < 0)
    return fail(GABP_ERR_INVALID_ARG, "gabp_run_rounds_noalloc: invalid argument");
  if (nnz > kNoAllocMaxEntries)
    return fail(GABP_ERR_INVALID_ARG,
                "gabp_run_rounds_noalloc: nnz = " + std::to_string(nnz) + " exceeds the fixed " +
                    "working space of " + std::to_string(kNoAllocMaxEntries) + " entries");
  // NULL would be the legacy default stream, which synchronises implicitly
  // with every blocking stream of the process (including one that another
  // component may be capturing); the calling thread's per-thread default
  // stream keeps the ordering with legacy-stream work without that.
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamPerThread;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) return fail(GABP_ERR_CUDA, cudaGetErrorString(ce));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(GABP_ERR_INVALID_ARG,
                "gabp_run_rounds_noalloc: the stream is being captured; the call reads a status "
                "word back to the host and synchronises its stream, so it cannot run there");
  // Device address of the array on the current device.  Looked up on every
  // call (no memory is allocated by the lookup): after a device reset the
  // module is loaded again and the array may sit at a new address, so a
  // cached pointer could go stale.  The first call on a device also loads
  // the library's module there if it is not loaded yet.
  void *p = nullptr;
  ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (ce != cudaSuccess)
    return fail(GABP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
  double2 *scratch = static_cast<double2 *>(p);
  double2 *buf[2] = {scratch, scratch + kNoAllocMaxEntries};
  int *breakdown = reinterpret_cast<int *>(scratch + 2 * kNoAllocMaxEntries);
  // The flag is the only state that must start at zero; the message buffers
  // need no clearing (round 1 does not read them).
  ce = cudaMemsetAsync(breakdown, 0, sizeof(int), st);
  if (ce != cudaSuccess) return fail(GABP_ERR_CUDA, cudaGetErrorString(ce));
  const int block = 256;
  const int grid = static_cast<int>(std::min<int64_t>((n + block - 1) / block, 4096));
  int cur = 0;
  for (int32_t t = 0; t <= rounds; ++t) {
    const int infer = t == rounds;
    noalloc_round_kernel<<<grid, block, 0, st>>>(n, row_ptr_dev, col_dev, val_dev, rev_dev, b_dev,
                                                 buf[cur], buf[cur ^ 1], x_dev, breakdown,
                                                 t == 0 ? 1 : 0, infer);
    if (!infer) cur ^= 1;
  }
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(GABP_ERR_CUDA, cudaGetErrorString(ce));
  int flag = 0;
  ce = cudaMemcpyAsync(&flag, breakdown, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(GABP_ERR_CUDA, cudaGetErrorString(ce));
  if (flag) return fail(GABP_ERR_BREAKDOWN, "gabp_run_rounds_noalloc: breakdown");
  return GABP_OK;
}
