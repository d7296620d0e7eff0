// gabp_pinv.cu -- Section VII with Psi = 0: the Moore-Penrose solution
// x^ = S^+ y for the systems a gabp_create_lsq_batched handle was given with
// psi_s = 0.
//
// Section VII states that the augmented system [[I, S^T], [S, -Psi]] yields
// the pseudoinverse solution when Psi = 0.  GaBP cannot run on that matrix:
// every z node then has a zero diagonal, and the first round divides by it.
// The handle is therefore built with a positive Psi_0 for those systems, and
// the solve iterates
//     x^ <- x^ + (S^T S + Psi_0)^{-1} S^T (y - S x^)
// (iterated Tikhonov regularisation).  A fixed point satisfies the normal
// equations S^T (y - S x^) = 0, which for S of full column rank is
// x^ = S^+ y; each step multiplies the error along a right singular vector
// of S (singular value sigma) by psi_0 / (sigma^2 + psi_0).
//
// Every step is one augmented solve.  The first, with right-hand side
// [0; y], is the Section VII closed form.  The later ones take [g; 0] with
// g = S^T (y - S x^): eliminating z from [[I, S^T], [S, -Psi_0]] [a; b] =
// [g; 0] gives a = psi_0 (S^T S + Psi_0)^{-1} g, so x^ += a / psi_0.  That
// right-hand side is the normal-equation residual itself and shrinks as the
// iteration converges, so the relative accuracy of each augmented solve
// carries over to the step.  ([0; y - S x^] would give the same step, but
// y - S x^ tends to the least-squares residual, not to zero, and the inner
// solves' error would stall the iteration at that residual times their
// tolerance.)
//
// The kernels below are the pieces of that loop around the existing solve:
// the off-diagonal product of the augmented matrix (it maps [x^; 0] to
// [0; S x^] and [0; r] to [S^T r; 0]), the right-hand side, the update and a
// per-system maximum for the stop rule.  All FP64.
#include "gabp_internal.h"
#include "gabp_device.cuh"

namespace gabp {
namespace {

// u_i = sum over the off-diagonal entries of row i of A_ij v_j (CSR form):
// one warp per row.
__global__ void __launch_bounds__(kBlock) csr_offdiag_kernel(int32_t n, const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ col,
                                                             const double *__restrict__ a,
                                                             const double *__restrict__ v,
                                                             double *__restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  for (int64_t row = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32; row < n;
       row += warps) {
    double acc = 0.0;
    for (int32_t s = rp[row] + lane; s < rp[row + 1]; s += 32) acc += a[s] * v[col[s]];
    acc = group_sum<32>(acc);
    if (lane == 0) u[row] = acc;
  }
}

// The same product on the dense form, one block per system: the x^ rows sum
// a column of S against v_z (a thread per column, rows in order, so a warp
// reads consecutive entries), the z rows take a row of S against v_x (a warp
// per row).
__global__ void __launch_bounds__(kBlock) dense_offdiag_kernel(const DenseSys *__restrict__ sys,
                                                               int32_t nsys,
                                                               const double *__restrict__ S,
                                                               const double *__restrict__ v,
                                                               double *__restrict__ u) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t q = blockIdx.x; q < nsys; q += gridDim.x) {
    const DenseSys sy = sys[q];
    const int K = sy.K, N = sy.N;
    const double *Sg = S + sy.pair0;
    const double *vx = v + sy.node0, *vz = vx + K;
    double *ux = u + sy.node0, *uz = ux + K;
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) acc += Sg[static_cast<int64_t>(j) * K + r] * vz[j];
      ux[r] = acc;
    }
    for (int j = w; j < N; j += nw) {
      double acc = 0.0;
      for (int r = lane; r < K; r += 32) acc += Sg[static_cast<int64_t>(j) * K + r] * vx[r];
      acc = group_sum<32>(acc);
      if (lane == 0) uz[j] = acc;
    }
  }
}

// Position of augmented row i inside its system: < K_s for x^, else z.
struct AugRow {
  int32_t sy;
  int64_t local;
  int32_t K;
};
__device__ __forceinline__ AugRow aug_row(int64_t i, const int32_t *sys_of_row, const int64_t *aug_off,
                                          const int32_t *K) {
  const int32_t sy = sys_of_row[i];
  return AugRow{sy, i - aug_off[sy], K[sy]};
}

// v = [x^; 0]
__global__ void pinv_embed_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                                  const int64_t *__restrict__ aug_off, const int32_t *__restrict__ K,
                                  const int64_t *__restrict__ x_off, const double *__restrict__ xhat,
                                  double *__restrict__ v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AugRow a = aug_row(i, sys_of_row, aug_off, K);
    v[i] = a.local < a.K ? xhat[x_off[a.sy] + a.local] : 0.0;
  }
}

// rhs = [0; y - u_z] for the flagged systems, [0; 0] for the others (u_z = S x^)
__global__ void pinv_rhs_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                                const int64_t *__restrict__ aug_off, const int32_t *__restrict__ K,
                                const int64_t *__restrict__ y_off, const double *__restrict__ y,
                                const double *__restrict__ u, const uint8_t *__restrict__ flag,
                                double *__restrict__ rhs) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AugRow a = aug_row(i, sys_of_row, aug_off, K);
    rhs[i] = (a.local < a.K || !flag[a.sy]) ? 0.0 : y[y_off[a.sy] + (a.local - a.K)] - u[i];
  }
}

// x^ += the x^ part of the augmented solution, times scale[s] (null: 1)
__global__ void pinv_update_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                                   const int64_t *__restrict__ aug_off, const int32_t *__restrict__ K,
                                   const int64_t *__restrict__ x_off, const double *__restrict__ scale,
                                   const double *__restrict__ x_aug, double *__restrict__ xhat) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AugRow a = aug_row(i, sys_of_row, aug_off, K);
    if (a.local < a.K) xhat[x_off[a.sy] + a.local] += scale ? x_aug[i] * scale[a.sy] : x_aug[i];
  }
}

// smax[s] = max |u_i| over the x^ rows of system s (bit patterns of
// non-negative doubles order like the values)
__global__ void pinv_sysmax_kernel(int64_t n_aug, const int32_t *__restrict__ sys_of_row,
                                   const int64_t *__restrict__ aug_off, const int32_t *__restrict__ K,
                                   const double *__restrict__ u, unsigned long long *__restrict__ smax) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_aug;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AugRow a = aug_row(i, sys_of_row, aug_off, K);
    if (a.local < a.K) atomicMax(&smax[a.sy], bits(fabs(u[i])));
  }
}

int grid_for(int64_t n) {
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, 65535)));
}

}  // namespace

int launch_csr_offdiag(const Graph &g, cudaStream_t st, const double *v, double *u) {
  csr_offdiag_kernel<<<grid_for(static_cast<int64_t>(g.n) * 32), kBlock, 0, st>>>(g.n, g.rp, g.col, g.a64,
                                                                                  v, u);
  return 1;
}

int launch_dense_offdiag(const Dense &d, cudaStream_t st, const double *v, double *u) {
  dense_offdiag_kernel<<<std::max(1, std::min(d.nsys, 65535)), kBlock, 0, st>>>(d.sys, d.nsys, d.v.S64, v,
                                                                                 u);
  return 1;
}

int launch_pinv_embed(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                      const int32_t *K, const int64_t *x_off, const double *xhat, double *v) {
  pinv_embed_kernel<<<grid_for(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, x_off, xhat, v);
  return 1;
}

int launch_pinv_rhs(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                    const int32_t *K, const int64_t *y_off, const double *y, const double *u,
                    const uint8_t *flag, double *rhs) {
  pinv_rhs_kernel<<<grid_for(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, y_off, y, u, flag,
                                                      rhs);
  return 1;
}

int launch_pinv_update(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                       const int32_t *K, const int64_t *x_off, const double *scale, const double *x_aug,
                       double *xhat) {
  pinv_update_kernel<<<grid_for(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, x_off, scale, x_aug,
                                                         xhat);
  return 1;
}

int launch_pinv_sysmax(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                       const int32_t *K, const double *u, unsigned long long *smax) {
  pinv_sysmax_kernel<<<grid_for(n_aug), kBlock, 0, st>>>(n_aug, sys_of_row, aug_off, K, u, smax);
  return 1;
}

}  // namespace gabp
