// gabp_kernels.cu -- sm_103a kernels of the synchronous broadcast GaBP sweep.
//
// Every sweep kernel implements one round of Alg. 2 (broadcast GaBP) with the
// parallel schedule of Section III-C: it reads only the previous round's
// messages (buffer "in") and writes the new round (buffer "out").
//
// Work mapping: a group of G lanes (G a power of two, G <= 32) owns one row i.
// The lanes stride over the row's slots, which hold the incoming messages
// m_{j->i}; the row totals
//     P~_i = A_ii + sum_k P_ki,        h~_i = b_i + sum_k eta_ki
// are formed with a shuffle reduction inside the group, and each lane then
// sends the messages of its own slots (the reverse message m_{j->i} needed by
// P~_i - P_ji is the value the lane already holds):
//     P_ij   = -A_ij^2 / (P~_i - P_ji)
//     eta_ij = -A_ij (h~_i - eta_ji) / (P~_i - P_ji)     (eta = P mu)
// written to slot rev[s] of row j.  Reads are contiguous; only the message
// store is a scatter.  Up to kCacheSlots slots per lane stay in registers
// between the two passes; longer rows re-read the tail.
#include "gabp_internal.h"

#include <algorithm>
#include <cstring>

namespace gabp {
namespace {

__device__ __forceinline__ unsigned long long bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}

__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide maximum of up to four non-negative values (as bit patterns),
// committed with one atomicMax per value and block.  Every thread of the
// block must call it.
__device__ void block_max4(unsigned long long v0, unsigned long long v1, unsigned long long v2,
                           unsigned long long v3, unsigned long long *d0, unsigned long long *d1,
                           unsigned long long *d2, unsigned long long *d3) {
  __shared__ unsigned long long sm[4][kBlock / 32];
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


// Row owned by this lane's group in the current warp step.
struct RowSlot {
  bool valid;
  int32_t i, rs, re;
};

__device__ __forceinline__ RowSlot row_at(const int32_t *__restrict__ rp,
                                          const int32_t *__restrict__ rows, int32_t nrows,
                                          int64_t ri) {
  RowSlot r;
  r.valid = ri < nrows;
  r.i = r.valid ? (rows ? rows[ri] : static_cast<int32_t>(ri)) : 0;
  r.rs = r.valid ? rp[r.i] : 0;
  r.re = r.valid ? rp[r.i + 1] : 0;
  return r;
}

// ---------------------------------------------------------------------------
// FP64 full sweep: new (P, eta) for every directed edge, plus optionally the
// tentative means x_i = h~_i / P~_i of the messages read (Alg. 2 step 4).
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kBlock)
sweep64_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ rev,
               const int32_t *__restrict__ rows, int32_t nrows, const double *__restrict__ a,
               const double *__restrict__ diag, const double *__restrict__ b,
               const double2 *__restrict__ min, double2 *__restrict__ mout,
               double *__restrict__ x_out, const double *__restrict__ x_prev, DevScalars *red,
               int write_msgs) {
  constexpr int R = kCacheSlots;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  unsigned long long mdx = 0, mx = 0;
  bool brk = false;

  for (int64_t base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const RowSlot row = row_at(rp, rows, nrows, base + sub);
    double2 mc[R];
    double ac[R];
    int32_t rc[R];
    double sP = 0.0, sH = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) {
        mc[k] = min[s];
        sP += mc[k].x;
        sH += mc[k].y;
        if (write_msgs) { ac[k] = a[s]; rc[k] = rev[s]; }
      }
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) {
      const double2 m = min[s];
      sP += m.x;
      sH += m.y;
    }
    sP = group_sum<G>(sP);
    sH = group_sum<G>(sH);
    if (!row.valid) continue;
    const double TP = diag[row.i] + sP;   // P~_i
    const double Th = b[row.i] + sH;      // h~_i = P~_i mu~_i
    if (x_out && gl == 0) {
      const double xi = Th / TP;
      x_out[row.i] = xi;
      if (x_prev) {
        mdx = umax(mdx, bits(fabs(xi - x_prev[row.i])));
        mx = umax(mx, bits(fabs(xi)));
      }
    }
    if (!write_msgs) continue;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) {
        const double d = TP - mc[k].x;    // P_{i\j} = P~_i - P_ji
        brk |= !(d != 0.0) || !isfinite(d);
        const double inv = 1.0 / d;
        mout[rc[k]] = make_double2(-(ac[k] * ac[k]) * inv, -ac[k] * (Th - mc[k].y) * inv);
      }
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) {
      const double2 m = min[s];
      const double av = a[s];
      const double d = TP - m.x;
      brk |= !(d != 0.0) || !isfinite(d);
      const double inv = 1.0 / d;
      mout[rev[s]] = make_double2(-(av * av) * inv, -av * (Th - m.y) * inv);
    }
  }
  if (brk) atomicOr(&red->breakdown, 1);
  if (x_prev) block_max4(mdx, mx, 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// FP32 full sweep (mixed modes, precision phase).  Messages (P, eta) in FP32,
// totals in FP32.  Always records (P~_i, d_i = h~_i / P~_i) per node and the
// change against the previous sweep.  With c_out != nullptr it is the
// freezing sweep: instead of new (P, eta) it stores the frozen coefficient
// c_ij = -A_ij / (P~_i - P_ji) at slot s of row i, 1/P~_i, and the first
// mean-only messages eta_ij = c_ij (h~_i - eta_ji) into eta_out.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kBlock)
sweep32_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ rev,
               const int32_t *__restrict__ rows, int32_t nrows, const float *__restrict__ a,
               const float *__restrict__ diag, const float *__restrict__ rhs,
               const float2 *__restrict__ min, float2 *__restrict__ mout,
               const float2 *__restrict__ mon_prev, float2 *__restrict__ mon_out,
               float *__restrict__ c_out, float *__restrict__ invP_out,
               float *__restrict__ eta_out, DevScalars *red) {
  constexpr int R = kCacheSlots;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const bool freeze = c_out != nullptr;
  unsigned long long mdd = 0, md = 0, mdP = 0, mP = 0;
  bool brk = false;

  for (int64_t base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const RowSlot row = row_at(rp, rows, nrows, base + sub);
    float2 mc[R];
    float ac[R];
    int32_t rc[R];
    float sP = 0.f, sH = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) {
        mc[k] = min[s];
        ac[k] = a[s];
        rc[k] = rev[s];
        sP += mc[k].x;
        sH += mc[k].y;
      }
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) {
      const float2 m = min[s];
      sP += m.x;
      sH += m.y;
    }
    sP = group_sum<G>(sP);
    sH = group_sum<G>(sH);
    if (!row.valid) continue;
    const float TP = diag[row.i] + sP;
    const float Th = rhs[row.i] + sH;
    if (gl == 0) {
      const float di = Th / TP;
      const float2 prev = mon_prev[row.i];
      mon_out[row.i] = make_float2(TP, di);
      mdd = umax(mdd, bits(fabs(static_cast<double>(di) - prev.y)));
      md = umax(md, bits(fabs(static_cast<double>(di))));
      mdP = umax(mdP, bits(fabs(static_cast<double>(TP) - prev.x)));
      mP = umax(mP, bits(fabs(static_cast<double>(TP))));
      if (freeze) invP_out[row.i] = 1.0f / TP;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) {
        const float d = TP - mc[k].x;
        brk |= !(d != 0.0f) || !isfinite(d);
        const float inv = 1.0f / d;
        if (freeze) {
          const float c = -ac[k] * inv;
          c_out[s] = c;
          eta_out[rc[k]] = c * (Th - mc[k].y);
        } else {
          mout[rc[k]] = make_float2(-(ac[k] * ac[k]) * inv, -ac[k] * (Th - mc[k].y) * inv);
        }
      }
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) {
      const float2 m = min[s];
      const float av = a[s];
      const float d = TP - m.x;
      brk |= !(d != 0.0f) || !isfinite(d);
      const float inv = 1.0f / d;
      if (freeze) {
        const float c = -av * inv;
        c_out[s] = c;
        eta_out[rev[s]] = c * (Th - m.y);
      } else {
        mout[rev[s]] = make_float2(-(av * av) * inv, -av * (Th - m.y) * inv);
      }
    }
  }
  if (brk) atomicOr(&red->breakdown, 1);
  block_max4(mdd, md, mdP, mP, &red->max_dx, &red->max_x, &red->max_dP, &red->max_P);
}

// ---------------------------------------------------------------------------
// FP32 mean-only sweep with frozen precisions: eta_ij = c_ij (h~_i - eta_ji),
// h~_i = rhs_i + sum_k eta_ki, d_i = h~_i / P~_i.  Records d_i and its change.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kBlock)
mean32_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ rev,
              const int32_t *__restrict__ rows, int32_t nrows, const float *__restrict__ c,
              const float *__restrict__ invP, const float *__restrict__ rhs,
              const float *__restrict__ ein, float *__restrict__ eout,
              const float2 *__restrict__ mon_prev, float2 *__restrict__ mon_out,
              DevScalars *red) {
  constexpr int R = kCacheSlots;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  unsigned long long mdd = 0, md = 0;

  for (int64_t base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const RowSlot row = row_at(rp, rows, nrows, base + sub);
    float ec[R], cc[R];
    int32_t rc[R];
    float sH = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) {
        ec[k] = ein[s];
        cc[k] = c[s];
        rc[k] = rev[s];
        sH += ec[k];
      }
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) sH += ein[s];
    sH = group_sum<G>(sH);
    if (!row.valid) continue;
    const float Th = rhs[row.i] + sH;
    if (gl == 0) {
      const float di = Th * invP[row.i];
      const float2 prev = mon_prev[row.i];
      mon_out[row.i] = make_float2(0.f, di);
      mdd = umax(mdd, bits(fabs(static_cast<double>(di) - prev.y)));
      md = umax(md, bits(fabs(static_cast<double>(di))));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int32_t s = row.rs + gl + k * G;
      if (s < row.re) eout[rc[k]] = cc[k] * (Th - ec[k]);
    }
    for (int32_t s = row.rs + gl + R * G; s < row.re; s += G) eout[rev[s]] = c[s] * (Th - ein[s]);
  }
  block_max4(mdd, md, 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x with its infinity norm (a CSR SpMV over the same
// row groups).
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kBlock)
residual64_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                  const int32_t *__restrict__ rows, int32_t nrows, const double *__restrict__ a,
                  const double *__restrict__ diag, const double *__restrict__ b,
                  const double *__restrict__ x, double *__restrict__ r_out, DevScalars *red) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  unsigned long long mr = 0;
  for (int64_t base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const RowSlot row = row_at(rp, rows, nrows, base + sub);
    double acc = 0.0;
    for (int32_t s = row.rs + gl; s < row.re; s += G) acc += a[s] * x[col[s]];
    acc = group_sum<G>(acc);
    if (!row.valid || gl != 0) continue;
    const double ri = b[row.i] - (diag[row.i] * x[row.i] + acc);
    if (r_out) r_out[row.i] = ri;
    mr = umax(mr, bits(fabs(ri)));
  }
  block_max4(mr, 0, 0, 0, &red->max_r, nullptr, nullptr, nullptr);
}

__global__ void max_abs_kernel(const double *__restrict__ v, int64_t n, unsigned long long *slot) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = umax(m, bits(fabs(v[i])));
  block_max4(m, 0, 0, 0, slot, nullptr, nullptr, nullptr);
}

__global__ void scale_to_f32_kernel(const double *__restrict__ v, int64_t n, double scale,
                                    float *__restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = static_cast<float>(v[i] * scale);
}

__global__ void refine_update_kernel(int64_t n, double *__restrict__ x,
                                     const float2 *__restrict__ mon, double inv_scale) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] += static_cast<double>(mon[i].y) * inv_scale;
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

// Blocks for a row launch: enough to give every row its group, capped at a
// whole number of waves over the SMs (the kernels are grid-stride).
int row_grid(int32_t nrows, int group) {
  const int64_t need = (static_cast<int64_t>(nrows) * group + kBlock - 1) / kBlock;
  const int64_t cap = static_cast<int64_t>(num_sms()) * 8;
  return static_cast<int>(std::max<int64_t>(1, std::min(need, cap)));
}

int flat_grid(int64_t n) {
  const int64_t need = (n + kBlock - 1) / kBlock;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, num_sms() * 8)));
}

#define GABP_DISPATCH_G(group, KERNEL, ...)                               \
  switch (group) {                                                        \
    case 1: KERNEL<1><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;       \
    case 2: KERNEL<2><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;       \
    case 4: KERNEL<4><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;       \
    case 8: KERNEL<8><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;       \
    case 16: KERNEL<16><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;     \
    default: KERNEL<32><<<grid, kBlock, 0, st>>>(__VA_ARGS__); break;     \
  }

}  // namespace

int launch_sweep64(const Graph &g, cudaStream_t st, const double2 *min, double2 *mout,
                    const double *b, double *x_out, const double *x_prev, DevScalars *red,
                    bool write_msgs) {
  int launched = 0;
  for (const RowBin &bin : g.bins) {
    if (bin.nrows == 0) continue;
    ++launched;
    const int grid = row_grid(bin.nrows, bin.group);
    GABP_DISPATCH_G(bin.group, sweep64_kernel, g.rp, g.rev, bin.rows, bin.nrows, g.a64, g.diag64,
                    b, min, mout, x_out, x_prev, red, write_msgs ? 1 : 0);
  }
  return launched;
}

int launch_sweep32(const Graph &g, cudaStream_t st, const float2 *min, float2 *mout,
                    const float *rhs, const float2 *mon_prev, float2 *mon_out, float *c_out,
                    float *invP_out, float *eta_out, DevScalars *red) {
  int launched = 0;
  for (const RowBin &bin : g.bins) {
    if (bin.nrows == 0) continue;
    ++launched;
    const int grid = row_grid(bin.nrows, bin.group);
    GABP_DISPATCH_G(bin.group, sweep32_kernel, g.rp, g.rev, bin.rows, bin.nrows, g.a32, g.diag32,
                    rhs, min, mout, mon_prev, mon_out, c_out, invP_out, eta_out, red);
  }
  return launched;
}

int launch_mean32(const Graph &g, cudaStream_t st, const float *ein, float *eout, const float *c,
                   const float *invP, const float *rhs, const float2 *mon_prev, float2 *mon_out,
                   DevScalars *red) {
  int launched = 0;
  for (const RowBin &bin : g.bins) {
    if (bin.nrows == 0) continue;
    ++launched;
    const int grid = row_grid(bin.nrows, bin.group);
    GABP_DISPATCH_G(bin.group, mean32_kernel, g.rp, g.rev, bin.rows, bin.nrows, c, invP, rhs,
                    ein, eout, mon_prev, mon_out, red);
  }
  return launched;
}

int launch_residual64(const Graph &g, cudaStream_t st, const double *b, const double *x,
                       double *r_out, DevScalars *red) {
  int launched = 0;
  for (const RowBin &bin : g.bins) {
    if (bin.nrows == 0) continue;
    ++launched;
    const int grid = row_grid(bin.nrows, bin.group);
    GABP_DISPATCH_G(bin.group, residual64_kernel, g.rp, g.col, bin.rows, bin.nrows, g.a64,
                    g.diag64, b, x, r_out, red);
  }
  return launched;
}

int launch_max_abs(cudaStream_t st, const double *v, int64_t n, unsigned long long *slot) {
  max_abs_kernel<<<flat_grid(n), kBlock, 0, st>>>(v, n, slot);
  return 1;
}

int launch_scale_to_f32(cudaStream_t st, const double *v, int64_t n, double scale, float *out) {
  scale_to_f32_kernel<<<flat_grid(n), kBlock, 0, st>>>(v, n, scale, out);
  return 1;
}

int launch_refine_update(cudaStream_t st, int64_t n, double *x, const float2 *mon,
                         double inv_scale) {
  refine_update_kernel<<<flat_grid(n), kBlock, 0, st>>>(n, x, mon, inv_scale);
  return 1;
}

void launch_fill_zero(cudaStream_t st, void *p, size_t bytes) {
  if (bytes) cudaMemsetAsync(p, 0, bytes, st);
}

double bits_to_double(unsigned long long u) {
  double d;
  static_assert(sizeof(d) == sizeof(u), "size");
  memcpy(&d, &u, sizeof(d));
  return d;
}

}  // namespace gabp
