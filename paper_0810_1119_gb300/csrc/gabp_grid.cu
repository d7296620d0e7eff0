// gabp_grid.cu -- nearest-neighbour operators on a box in the grid form.
//
// A matrix whose off-diagonal entries couple only nearest neighbours of a
// 1-, 2- or 3-D box in natural order (the 3-, 5- and 7-point Laplacians of
// Section IX, with any coefficients) has a graph with no index arrays worth
// storing: the neighbour of node (x, y, z) in direction d is a fixed offset
// away.  The grid form stores the two colour classes of the box, c = (x + y
// + z) mod 2, each as a half grid, and per class and direction one plane of
// A values and one of messages (layout in gabp_internal.h).  The message from
// node (c, H) to its neighbour in direction d lands in plane (1 - c, d ^ 1) at
// H + off(d): a sweep reads and writes every plane as a contiguous run.
//
// Schedules (Section III-C):
//   synchronous:  one launch per round over both classes, two message
//                 buffers (Alg. 2);
//   serial:       one launch per class, in place; the classes are the two
//                 colours of the box, so this is the serial schedule with
//                 the nodes visited class 0 first (red-black).
// The node and message arithmetic is that of the CSR kernels (same
// reciprocals, monitors, freeze and damping rules), one thread per node.
#include "gabp_internal.h"
#include "gabp_device.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

namespace gabp {
namespace {

constexpr int kGridBlock = 256;
constexpr int kMaxDir = 6;

// A node of one launch: class c, half-grid index H, row parity s, and which
// of its directions have a neighbour inside the box.
struct GNode {
  int c;
  int64_t H, slot;
  int s;
  unsigned in_box;   // bit d: the neighbour in direction d exists
};

// n / d for n < 2^31 from the view's multiplier and shift.
__device__ __forceinline__ uint32_t div_by(uint32_t n, uint64_t m, int s) {
  return static_cast<uint32_t>((static_cast<uint64_t>(n) * m) >> s);
}

// The box holds fewer than 2^31 nodes, so the coordinates come from 32-bit
// arithmetic: the two divisions per node are multiplications by the
// precomputed reciprocals (the class is a comparison).
__device__ __forceinline__ bool node_of(const GridView &g, int64_t t, GNode &n) {
  const int64_t count = g.pass < 0 ? 2 * g.Nh : g.Nh;
  if (t >= count) return false;
  n.slot = g.pass < 0 ? t : g.pass * g.Nh + t;
  n.c = n.slot >= g.Nh ? 1 : 0;
  n.H = n.slot - n.c * g.Nh;
  const uint32_t H = static_cast<uint32_t>(n.H), h0 = static_cast<uint32_t>(g.h0);
  const uint32_t row = div_by(H, g.m_h0, g.s_h0), z32 = div_by(row, g.m_p1, g.s_p1);
  const int hx = static_cast<int>(H - row * h0);
  const int z = static_cast<int>(z32), y = static_cast<int>(row - z32 * static_cast<uint32_t>(g.p1));
  n.s = (n.c + y + z) & 1;
  const int x = 2 * hx + n.s, p0 = 2 * g.h0;
  unsigned m = 0;
  if (x + 1 < p0) m |= 1u;
  if (x >= 1) m |= 2u;
  if (g.ndim > 1) {
    if (y + 1 < g.p1) m |= 4u;
    if (y >= 1) m |= 8u;
  }
  if (g.ndim > 2) {
    if (z + 1 < g.p2) m |= 16u;
    if (z >= 1) m |= 32u;
  }
  n.in_box = m;
  return true;
}

// Plane index of the message into (c, H) from direction d, and of the one
// (c, H) sends in direction d (into its neighbour, from direction d ^ 1).
__device__ __forceinline__ int64_t plane_in(const GridView &g, int c, int d, int64_t H) {
  return (static_cast<int64_t>(c) * g.D + d) * g.Nh + H;
}
__device__ __forceinline__ int64_t plane_out(const GridView &g, const GNode &n, int d) {
  int64_t off;
  switch (d) {
    case 0: off = n.s; break;
    case 1: off = n.s - 1; break;
    case 2: off = g.h0; break;
    case 3: off = -static_cast<int64_t>(g.h0); break;
    case 4: off = static_cast<int64_t>(g.h0) * g.p1; break;
    default: off = -static_cast<int64_t>(g.h0) * g.p1; break;
  }
  return plane_in(g, 1 - n.c, d ^ 1, n.H + off);
}
// Slot of the neighbour in direction d (residual).
__device__ __forceinline__ int64_t slot_of(const GridView &g, const GNode &n, int d) {
  return plane_out(g, n, d) - (static_cast<int64_t>(1 - n.c) * g.D + (d ^ 1)) * g.Nh +
         (1 - n.c) * g.Nh;
}

int64_t grid_blocks(int64_t count) {
  return std::max<int64_t>(1, (count + kGridBlock - 1) / kGridBlock);
}

// CTAs of a kernel resident on the device, cached per kernel (primed at
// create time, before any graph is recorded): the grid-stride launches take
// at most this many.
std::mutex g_res_mu;
std::unordered_map<const void *, int64_t> g_res_blocks;

template <class Kern>
int64_t resident_grid_blocks(Kern kernel) {
  std::lock_guard<std::mutex> lk(g_res_mu);
  auto it = g_res_blocks.find(reinterpret_cast<const void *>(kernel));
  if (it != g_res_blocks.end()) return it->second;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGridBlock, 0);
  const int64_t r = static_cast<int64_t>(std::max(sms, 1)) * std::max(per_sm, 1);
  g_res_blocks[reinterpret_cast<const void *>(kernel)] = r;
  return r;
}
int64_t launch_count(const GridView &v) { return v.pass < 0 ? 2 * v.Nh : v.Nh; }

// ---------------------------------------------------------------------------
// FP64 full sweep (Alg. 2): totals, the tentative mean when asked, and the
// (P, eta) message to every neighbour.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGridBlock)
grid_sweep64_kernel(GridView g, Buffers B, Ctl *ctl, DevScalars *red) {
  const int par = ctl->par_m;
  const bool zin = ctl->first != 0 && !g.in_place;
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
  const double2 *min = par ? B.m64[1] : B.m64[0];
  double2 *mout = par ? B.m64[0] : B.m64[1];
  const double gam = g.no_damp ? 0.0 : ctl->damping;
  bool brk = false;
  GNode n;
  if (node_of(g, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x, n)) {
    double a[kMaxDir];
    double2 m[kMaxDir];
    double sP = 0.0, sH = 0.0;
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      a[d] = 0.0;
      m[d] = make_double2(0.0, 0.0);
      if (d >= g.D || !((n.in_box >> d) & 1u)) continue;
      const int64_t p = plane_in(g, n.c, d, n.H);
      a[d] = g.a64[p];
      if (!zin) m[d] = min[p];
      sP += m[d].x;
      sH += m[d].y;
    }
    const double TP = g.diag64[n.slot] + sP, Th = b[n.slot] + sH;
    if (write_x) x[n.slot] = Th / TP;
    if (write_msgs)
#pragma unroll
      for (int d = 0; d < kMaxDir; ++d) {
        if (a[d] == 0.0) continue;
        const double dd = TP - m[d].x;   // P~_i - P_ji
        brk |= zero_or_nonfinite(dd);
        const double inv = recip64(dd);
        const int64_t q = plane_out(g, n, d);
        double eta = -a[d] * (Th - m[d].y) * inv;
        if (gam > 0.0) eta = gam * (zin ? 0.0 : min[q].y) + (1.0 - gam) * eta;
        mout[q] = make_double2(-(a[d] * a[d]) * inv, eta);
      }
  }
  if (__syncthreads_or(brk) && threadIdx.x == 0) atomicOr(&red->breakdown, 1);
  last_block_control(ctl, red, g.no_control ? 0 : CK_SWEEP64);
}

// ---------------------------------------------------------------------------
// FP32 full sweep of the mixed modes, with the precision freeze (storage E
// for the first mean-only messages): the node and message rules of the CSR
// FP32 sweep.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_e(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_e(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float ld_e(const float *p) { return *p; }
__device__ __forceinline__ float ld_e(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <class E>
__global__ void __launch_bounds__(kGridBlock)
grid_sweep32_kernel(GridView g, Buffers B, Ctl *ctl, DevScalars *red) {
  const int pm = ctl->par_m, pe = ctl->par_e, pmon = ctl->par_mon;
  const bool first = ctl->first != 0;
  const bool zin = first && !g.in_place;
  const bool freeze = ctl->pending_freeze != 0;
  const double inv_rn = ctl->inv_rn;
  const float2 *min = pm ? B.m32[1] : B.m32[0];
  float2 *mout = pm ? B.m32[0] : B.m32[1];
  E *eout = static_cast<E *>(pe ? B.e[0] : B.e[1]);   // freeze: the first mean-only messages
  const float2 *__restrict__ mon_prev = pmon ? B.mon32[1] : B.mon32[0];
  float2 *__restrict__ mon_out = pmon ? B.mon32[0] : B.mon32[1];
  const float gam = g.no_damp ? 0.f : static_cast<float>(ctl->damping);
  uint32_t mdd = 0, md = 0, mdP = 0, mP = 0;
  bool brk = false;
  GNode n;
  if (node_of(g, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x, n)) {
    float a[kMaxDir];
    float2 m[kMaxDir];
    float sP = 0.f, sH = 0.f;
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      a[d] = 0.f;
      m[d] = make_float2(0.f, 0.f);
      if (d >= g.D || !((n.in_box >> d) & 1u)) continue;
      const int64_t p = plane_in(g, n.c, d, n.H);
      a[d] = g.a32[p];
      if (!zin) m[d] = min[p];
      sP += m[d].x;
      sH += m[d].y;
    }
    const float rhs = first ? static_cast<float>(B.r64[n.slot] * inv_rn) : B.rhs32[n.slot];
    const float TP = g.diag32[n.slot] + sP, Th = rhs + sH;
    const float2 prev = first ? make_float2(0.f, 0.f) : mon_prev[n.slot];
    const float di = Th / TP;
    mon_out[n.slot] = make_float2(TP, di);
    mdd = fmax_bits(mdd, di - prev.y);
    md = fmax_bits(md, di);
    mdP = fmax_bits(mdP, TP - prev.x);
    mP = fmax_bits(mP, TP);
    if (freeze) B.invP32[n.slot] = 1.0f / TP;
    if (first) B.rhs32[n.slot] = rhs;
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      if (d >= g.D || !((n.in_box >> d) & 1u)) continue;
      const int64_t p = plane_in(g, n.c, d, n.H);
      if (a[d] == 0.f) {
        if (freeze) B.c32[p] = 0.f;
        continue;
      }
      const float dd = TP - m[d].x;   // P~_i - P_ji
      brk |= !(dd != 0.0f) || !isfinite(dd);
      const float inv = 1.0f / dd;
      const int64_t q = plane_out(g, n, d);
      if (freeze) {
        const float cc = -a[d] * inv;
        B.c32[p] = cc;
        float eta = cc * (Th - m[d].y);
        if (gam > 0.f) eta = gam * (zin ? 0.f : min[q].y) + (1.f - gam) * eta;
        st_e(eout + q, eta);
      } else {
        float eta = -a[d] * (Th - m[d].y) * inv;
        if (gam > 0.f) eta = gam * (zin ? 0.f : min[q].y) + (1.f - gam) * eta;
        mout[q] = make_float2(-(a[d] * a[d]) * inv, eta);
      }
    }
  }
  if (__syncthreads_or(brk) && threadIdx.x == 0) atomicOr(&red->breakdown, 1);
  block_max4(widen(mdd), widen(md), widen(mdP), widen(mP), &red->max_dx, &red->max_x,
             &red->max_dP, &red->max_P);
  last_block_control(ctl, red, g.no_control ? 0 : CK_SWEEP32);
}

// ---------------------------------------------------------------------------
// Mean-only sweep with frozen precisions: eta_ij = c_ij (h~_i - eta_ji),
// h~_i = r_i / ||r|| + sum eta_ki, d_i = h~_i / P~_i (frozen 1/P~_i).
// ---------------------------------------------------------------------------
template <class E>
__global__ void __launch_bounds__(kGridBlock)
grid_mean_kernel(GridView g, Buffers B, Ctl *ctl, DevScalars *red) {
  const int pe = ctl->par_e, pmon = ctl->par_mon;
  const bool first = ctl->first != 0;
  const bool zin = first && !g.in_place;
  const double inv_rn = ctl->inv_rn;
  const E *ein = static_cast<const E *>(pe ? B.e[1] : B.e[0]);
  E *eout = static_cast<E *>(pe ? B.e[0] : B.e[1]);
  const float2 *__restrict__ mon_prev = pmon ? B.mon32[1] : B.mon32[0];
  float2 *__restrict__ mon_out = pmon ? B.mon32[0] : B.mon32[1];
  const float gam = g.no_damp ? 0.f : static_cast<float>(ctl->damping);
  // Aitken on the inner solves (mixed solves with aitken > 0): this sweep is
  // number kk of its inner solve; at multiples of 2^j it records d in slot
  // (kk >> j) mod 3 of level j
  const int kk = ctl->k + 1;
  const bool rec = ctl->ait_mixed != 0 && (kk & ((1 << kAitMinLevel) - 1)) == 0;
  uint32_t mdd = 0, md = 0;
  GNode n;
  // nodes grid-stride (the grid is at most the resident CTAs), so that every
  // block reduces its monitors once
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; node_of(g, t, n);
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // every load of the node first (incoming messages, coefficients, node data)
    float e[kMaxDir], cf[kMaxDir];
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      e[d] = cf[d] = 0.f;
      if (d >= g.D || !((n.in_box >> d) & 1u)) continue;
      const int64_t p = plane_in(g, n.c, d, n.H);
      cf[d] = B.c32[p];
      if (!zin) e[d] = ld_e(ein + p);
    }
    const float rhs = first ? static_cast<float>(B.r64[n.slot] * inv_rn) : B.rhs32[n.slot];
    const float ip = B.invP32[n.slot];
    float sH = 0.f;
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) sH += e[d];
    const float Th = rhs + sH;
    const float prev = first ? 0.f : mon_prev[n.slot].y;
    const float di = Th * ip;
    mon_out[n.slot] = make_float2(0.f, di);
    mdd = fmax_bits(mdd, di - prev);
    md = fmax_bits(md, di);
    if (first) B.rhs32[n.slot] = rhs;
    if (rec) {
      const int64_t slots = 2 * g.Nh;
#pragma unroll 1
      for (int j = 0; j < kAitLevels; ++j) {
        const int lvl = kAitMinLevel + j;
        if (kk & ((1 << lvl) - 1)) break;   // not a multiple of 2^lvl: nor of the wider ones
        B.ait32[(static_cast<int64_t>(j) * 3 + (kk >> lvl) % 3) * slots + n.slot] = di;
      }
    }
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      const float cc = cf[d];
      if (cc == 0.f) continue;   // out of the box, or no edge
      const int64_t q = plane_out(g, n, d);
      float eta = cc * (Th - e[d]);
      if (gam > 0.f) eta = gam * (zin ? 0.f : ld_e(ein + q)) + (1.f - gam) * eta;
      st_e(eout + q, eta);
    }
  }
  block_max4(widen(mdd), widen(md), 0, 0, &red->max_dx, &red->max_x, nullptr, nullptr);
  last_block_control(ctl, red, g.no_control ? 0 : CK_MEAN);
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x over all slots, with max |r|.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGridBlock)
grid_residual_kernel(GridView g, double *__restrict__ r_out, Ctl *ctl, DevScalars *red, int kind) {
  const double *__restrict__ b = ctl->b;
  const double *__restrict__ x = ctl->x;
  unsigned long long mr = 0;
  GNode n;
  if (node_of(g, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x, n)) {
    double acc = g.diag64[n.slot] * x[n.slot];
#pragma unroll
    for (int d = 0; d < kMaxDir; ++d) {
      if (d >= g.D || !((n.in_box >> d) & 1u)) continue;
      const double a = g.a64[plane_in(g, n.c, d, n.H)];
      if (a != 0.0) acc += a * x[slot_of(g, n, d)];
    }
    const double ri = b[n.slot] - acc;
    if (r_out) r_out[n.slot] = ri;
    mr = bits(fabs(ri));
  }
  block_max4(mr, 0, 0, 0, &red->max_r, nullptr, nullptr, nullptr);
  last_block_control(ctl, red, kind);
}

}  // namespace

int launch_grid_full64(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red) {
  grid_sweep64_kernel<<<grid_blocks(launch_count(v)), kGridBlock, 0, st>>>(v, B, ctl, red);
  return 1;
}

int launch_grid_full32(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                       bool bf16) {
  if (bf16) grid_sweep32_kernel<__nv_bfloat16><<<grid_blocks(launch_count(v)), kGridBlock, 0, st>>>(v, B, ctl, red);
  else grid_sweep32_kernel<float><<<grid_blocks(launch_count(v)), kGridBlock, 0, st>>>(v, B, ctl, red);
  return 1;
}

int launch_grid_mean(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                     bool bf16) {
  if (bf16) {
    auto k = grid_mean_kernel<__nv_bfloat16>;
    k<<<std::min<int64_t>(grid_blocks(launch_count(v)), resident_grid_blocks(k)), kGridBlock, 0, st>>>(v, B, ctl, red);
  } else {
    auto k = grid_mean_kernel<float>;
    k<<<std::min<int64_t>(grid_blocks(launch_count(v)), resident_grid_blocks(k)), kGridBlock, 0, st>>>(v, B, ctl, red);
  }
  return 1;
}

int launch_grid_residual(const GridView &v, cudaStream_t st, double *r_out, Ctl *ctl,
                         DevScalars *red, bool refine) {
  GridView all = v;
  all.pass = -1;
  grid_residual_kernel<<<grid_blocks(launch_count(all)), kGridBlock, 0, st>>>(
      all, r_out, ctl, red, refine ? CK_REFINE : CK_CHECK64);
  return 1;
}

// ---------------------------------------------------------------------------
// Host: the planes of a nearest-neighbour operator on the box `dims`.
// ---------------------------------------------------------------------------
gabp_status build_grid(Grid &G, int32_t ndim, const int32_t *dims, int64_t nnz,
                       const int64_t *row_ptr, const int32_t *col, const double *val,
                       cudaStream_t st, std::vector<int32_t> &perm, std::string *msg) {
  if (ndim < 1 || ndim > 3 || !dims) {
    *msg = "gabp_create_grid: ndim must be 1, 2 or 3";
    return GABP_ERR_INVALID_ARG;
  }
  int64_t p[3] = {1, 1, 1};
  for (int k = 0; k < ndim; ++k) p[k] = dims[k];
  if (p[0] < 2 || p[0] % 2 != 0 || p[1] < 1 || p[2] < 1 || p[0] * p[1] * p[2] >= (int64_t{1} << 31) - 64) {
    *msg = "gabp_create_grid: dims[0] must be even and >= 2, the other dims >= 1, and the box below 2^31 nodes";
    return GABP_ERR_INVALID_ARG;
  }
  const int64_t n = p[0] * p[1] * p[2];
  if (!row_ptr || !col || !val || row_ptr[0] != 0 || row_ptr[n] != nnz) {
    *msg = "gabp_create_grid: row_ptr must start at 0 and end at nnz (n = the box's nodes)";
    return GABP_ERR_INVALID_ARG;
  }
  const int D = 2 * ndim;
  const int64_t h0 = p[0] / 2, Nh = n / 2;
  const int64_t stride[3] = {1, p[0], p[0] * p[1]};
  std::vector<double> a64(static_cast<size_t>(2 * D * Nh), 0.0), dg(static_cast<size_t>(n), 0.0);
  perm.assign(static_cast<size_t>(n), 0);
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t x = i % p[0], y = (i / p[0]) % p[1], z = i / (p[0] * p[1]);
    const int c = static_cast<int>((x + y + z) & 1);
    const int64_t H = x / 2 + h0 * (y + p[1] * z);
    const int64_t slot = c * Nh + H;
    perm[static_cast<size_t>(slot)] = static_cast<int32_t>(i);
    const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
    if (re < rs || re > nnz) {
      *msg = "gabp_create_grid: row_ptr is not monotone";
      return GABP_ERR_INVALID_ARG;
    }
    bool diag_seen = false;
    const int64_t xyz[3] = {x, y, z};
    for (int64_t e = rs; e < re; ++e) {
      const int64_t j = col[e];
      if (e > rs && col[e] <= col[e - 1]) {
        *msg = "gabp_create_grid: column indices of a row must be strictly increasing";
        return GABP_ERR_INVALID_ARG;
      }
      const double v = val[e];
      if (!std::isfinite(v)) {
        *msg = "gabp_create_grid: non-finite entry";
        return GABP_ERR_INVALID_ARG;
      }
      amax = std::max(amax, std::fabs(v));
      if (j == i) {
        dg[static_cast<size_t>(slot)] = v;
        diag_seen = true;
        continue;
      }
      int dir = -1;
      for (int k = 0; k < ndim && dir < 0; ++k) {
        if (j == i + stride[k] && xyz[k] + 1 < p[k]) dir = 2 * k;
        else if (j == i - stride[k] && xyz[k] >= 1) dir = 2 * k + 1;
      }
      if (dir < 0) {
        *msg = "gabp_create_grid: row " + std::to_string(i) + " couples column " + std::to_string(j) +
               ", which is not a nearest neighbour in the box";
        return GABP_ERR_INVALID_ARG;
      }
      a64[static_cast<size_t>((c * D + dir) * Nh + H)] = v;
    }
    if (!diag_seen || dg[static_cast<size_t>(slot)] == 0.0) {
      *msg = "gabp_create_grid: zero or missing diagonal in row " + std::to_string(i);
      return GABP_ERR_ZERO_DIAG;
    }
  }
  // symmetry: the value towards a neighbour equals the neighbour's value back
  const double tol = 1e-14 * amax;
  for (int64_t slot = 0; slot < n; ++slot) {
    const int c = static_cast<int>(slot / Nh);
    const int64_t i = perm[static_cast<size_t>(slot)];
    const int64_t x = i % p[0], y = (i / p[0]) % p[1], z = i / (p[0] * p[1]);
    const int64_t xyz[3] = {x, y, z};
    for (int d = 0; d < D; ++d) {
      const int k = d / 2;
      const bool up = (d & 1) == 0;
      if (up ? xyz[k] + 1 >= p[k] : xyz[k] < 1) continue;
      const int64_t j = up ? i + stride[k] : i - stride[k];
      const int64_t jx = j % p[0], jy = (j / p[0]) % p[1], jz = j / (p[0] * p[1]);
      const int64_t Hj = jx / 2 + h0 * (jy + p[1] * jz);
      const double aij = a64[static_cast<size_t>((c * D + d) * Nh + (slot - c * Nh))];
      const double aji = a64[static_cast<size_t>(((1 - c) * D + (d ^ 1)) * Nh + Hj)];
      if (std::fabs(aij - aji) > tol) {
        *msg = "gabp_create_grid: the matrix is not symmetric (rows " + std::to_string(i) + " and " +
               std::to_string(j) + ")";
        return GABP_ERR_NOT_SYMMETRIC;
      }
    }
  }
  std::vector<float> a32(a64.size()), dg32(dg.size());
  for (size_t k = 0; k < a64.size(); ++k) a32[k] = static_cast<float>(a64[k]);
  for (size_t k = 0; k < dg.size(); ++k) dg32[k] = static_cast<float>(dg[k]);
  cudaError_t ce = cudaSuccess;
  auto up = [&](auto **dst, const auto &src) {
    using T = std::remove_reference_t<decltype(src[0])>;
    if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void **>(dst), sizeof(T) * src.size());
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st);
  };
  up(&G.a64, a64);
  up(&G.diag64, dg);
  up(&G.a32, a32);
  up(&G.diag32, dg32);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    *msg = std::string("gabp_create_grid: ") + cudaGetErrorString(ce);
    return ce == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA;
  }
  for (int k = 0; k < 3; ++k) G.dims[k] = static_cast<int32_t>(p[k]);
  GridView &v = G.v;
  v.ndim = ndim;
  v.D = D;
  v.h0 = static_cast<int32_t>(h0);
  v.p1 = static_cast<int32_t>(p[1]);
  v.p2 = static_cast<int32_t>(p[2]);
  // multiplier and shift for n / d, 0 <= n < 2^31: with l = ceil(log2 d) and
  // m = ceil(2^(31 + l) / d), m d - 2^(31 + l) < d <= 2^l, which makes
  // floor(n m / 2^(31 + l)) = floor(n / d) (Granlund and Montgomery, Thm 4.2)
  auto magic = [](uint64_t d, uint64_t *m, int32_t *s) {
    int l = 0;
    while ((uint64_t{1} << l) < d) ++l;
    *s = 31 + l;
    *m = ((uint64_t{1} << (31 + l)) + d - 1) / d;
  };
  magic(static_cast<uint64_t>(h0), &v.m_h0, &v.s_h0);
  magic(static_cast<uint64_t>(p[1]), &v.m_p1, &v.s_p1);
  resident_grid_blocks(grid_mean_kernel<float>);
  resident_grid_blocks(grid_mean_kernel<__nv_bfloat16>);
  v.Nh = Nh;
  v.a64 = G.a64;
  v.diag64 = G.diag64;
  v.a32 = G.a32;
  v.diag32 = G.diag32;
  v.pass = -1;
  return GABP_OK;
}

void free_grid(Grid &G) {
  cudaFree(G.a64);
  cudaFree(G.diag64);
  cudaFree(G.a32);
  cudaFree(G.diag32);
  G.a64 = G.diag64 = nullptr;
  G.a32 = G.diag32 = nullptr;
}

}  // namespace gabp
