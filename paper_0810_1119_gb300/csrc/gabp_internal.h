// gabp_internal.h -- internal declarations shared by the library's
// translation units (not part of the C ABI).
//
// Device layout of one system (Section II-B graph, Alg. 2 messages):
//   The off-diagonal part of A is kept as a CSR over "slots".  Slot s of row i
//   (neighbour j = col[s]) stores the message travelling INTO node i from j,
//   m_{j->i}.  A sweep therefore reads each row's incoming messages as one
//   contiguous run, forms the node totals P~_i and h~_i = P~_i mu~_i, and
//   sends m_{i->j} by writing slot rev[s] (the slot of entry (j, i) in row j).
//   Each message is the pair (P, eta) with eta = P * mu (information form:
//   no division by A_ij is needed and eta sums directly into h~).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gabp.h"

namespace gabp {

constexpr int kBlock = 256;          // threads per block of the row kernels
constexpr int kCacheSlots = 4;       // slots per lane kept in registers

// Device-side reduction slots, zeroed before use.  Maxima of non-negative
// doubles are accumulated with 64-bit atomicMax on their bit patterns
// (IEEE order and unsigned order agree for non-negative values; NaN compares
// above +inf and so surfaces as "not finite").
struct DevScalars {
  unsigned long long max_dx;      // max_i |x_i^t - x_i^{t-1}|   (or |d| change)
  unsigned long long max_x;       // max_i |x_i^t|
  unsigned long long max_dP;      // max_i |P~_i^t - P~_i^{t-1}|
  unsigned long long max_P;       // max_i |P~_i^t|
  unsigned long long max_r;       // max_i |r_i|
  unsigned long long max_b;       // max_i |b_i|
  int breakdown;                  // set when P~_i - P_ji is zero or not finite
  int pad[3];
};

// One row bin: the rows a launch covers and its lanes-per-row.
struct RowBin {
  int32_t *rows = nullptr;  // device list of row ids; nullptr = rows 0..nrows-1
  int32_t nrows = 0;
  int group = 8;            // lanes per row (power of two, 1..32)
};

struct Graph {
  int32_t n = 0;
  int64_t E = 0;                 // directed edges (off-diagonal entries)
  // host copies used by the builder and the message export
  std::vector<int32_t> h_rp, h_col, h_rev;
  std::vector<int64_t> h_user_pos;   // CSR entry of A for each slot
  // device arrays
  int32_t *rp = nullptr, *col = nullptr, *rev = nullptr;
  double *a64 = nullptr, *diag64 = nullptr;
  float *a32 = nullptr, *diag32 = nullptr;
  std::vector<RowBin> bins;      // a partition of the rows
  int max_degree = 0;
};

}  // namespace gabp

struct gabp_s {
  gabp::Graph g;
  gabp_options opt;
  cudaStream_t stream = nullptr;
  std::string last_error;
  gabp_stats stats{};
  int64_t user_nnz = 0;            // nnz of the CSR given to gabp_create

  // FP64 full sweep state
  double2 *m64[2] = {nullptr, nullptr};
  int m64_cur = 0;                 // buffer holding the latest messages
  double *x_prev = nullptr;        // [n] previous tentative means (monitor)
  // FP32 state
  float2 *m32[2] = {nullptr, nullptr};
  float *e32[2] = {nullptr, nullptr};
  float *c32 = nullptr;            // [E] frozen mean coefficients
  float *invP32 = nullptr;         // [n] frozen 1/P~_i
  float *rhs32 = nullptr;          // [n] scaled right-hand side of the inner solve
  float2 *mon32[2] = {nullptr, nullptr};  // [n] (P~_i, d_i) of the last two sweeps
  // FP64 refinement state
  double *xw = nullptr, *r64 = nullptr;
  gabp::DevScalars *red = nullptr;        // device
  gabp::DevScalars *red_host = nullptr;   // pinned host mirror
  double *bbuf = nullptr, *xbuf = nullptr;  // device staging for gabp_solve_host
  // profiling (gabp_options.profile): pairs of events around kernels
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
};

namespace gabp {

// ---- kernels (gabp_kernels.cu) ----
int launch_sweep64(const Graph &g, cudaStream_t st, const double2 *min, double2 *mout,
                    const double *b, double *x_out, const double *x_prev, DevScalars *red,
                    bool write_msgs);
int launch_sweep32(const Graph &g, cudaStream_t st, const float2 *min, float2 *mout,
                    const float *rhs, const float2 *mon_prev, float2 *mon_out,
                    float *c_out, float *invP_out, float *eta_out, DevScalars *red);
int launch_mean32(const Graph &g, cudaStream_t st, const float *ein, float *eout,
                   const float *c, const float *invP, const float *rhs, const float2 *mon_prev,
                   float2 *mon_out, DevScalars *red);
int launch_residual64(const Graph &g, cudaStream_t st, const double *b, const double *x,
                       double *r_out, DevScalars *red);
int launch_max_abs(cudaStream_t st, const double *v, int64_t n, unsigned long long *slot);
int launch_scale_to_f32(cudaStream_t st, const double *v, int64_t n, double scale, float *out);
int launch_refine_update(cudaStream_t st, int64_t n, double *x, const float2 *mon, double inv_scale);
void launch_fill_zero(cudaStream_t st, void *p, size_t bytes);
double bits_to_double(unsigned long long u);

// ---- graph builder (gabp_build.cu) ----
gabp_status build_graph(Graph &g, int64_t n, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col, const double *val, const int64_t *rev,
                        const gabp_options &opt, cudaStream_t st, std::string *msg);
void free_graph(Graph &g);

}  // namespace gabp
