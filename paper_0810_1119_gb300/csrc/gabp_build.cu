// gabp_build.cu -- graph builder: validates the CSR of A, splits off the
// diagonal, drops explicit zeros, derives the reverse-edge index in slot
// numbering, cuts the rows into tiles for the staged sweep kernels, picks the
// lanes-per-row from the mean degree and uploads the device arrays.
//
// Graph of Section II-B: node i per row, an edge per off-diagonal non-zero;
// P_ii = A_ii must be non-zero (Alg. 2 step 1 divides by it).
#include "gabp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

namespace gabp {

namespace {

// Device copy with kPad elements of zeroed slack past the end (the staged
// kernels round their bulk copies up to 16 bytes).
template <class T>
cudaError_t upload(T **dst, const T *src, size_t count, cudaStream_t st) {
  const size_t bytes = (count + kPad) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(*dst, 0, bytes, st);
  if (e == cudaSuccess && count)
    e = cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
  return e;
}

// Greedy row tiles: consecutive rows while the tile keeps <= max_slots slots
// and <= max_rows rows; a row with more than max_slots slots is alone.
// With colour classes (bounds = class row offsets), no tile spans two
// classes, and *first_tile[c] is the first tile of class c.
std::vector<int2> make_tiles(const std::vector<int32_t> &rp, int64_t n, int max_slots,
                             int max_rows, const std::vector<int32_t> *bounds = nullptr,
                             std::vector<int32_t> *first_tile = nullptr) {
  std::vector<int2> t;
  std::vector<int32_t> cuts = bounds ? *bounds : std::vector<int32_t>{0, static_cast<int32_t>(n)};
  if (first_tile) first_tile->clear();
  for (size_t c = 0; c + 1 < cuts.size(); ++c) {
    if (first_tile) first_tile->push_back(static_cast<int32_t>(t.size()));
    int64_t r = cuts[c];
    const int64_t hi = cuts[c + 1];
    while (r < hi) {
      const int32_t s0 = rp[r];
      int64_t end = r + 1;
      if (rp[r + 1] - s0 <= max_slots)
        while (end < hi && end - r < max_rows && rp[end + 1] - s0 <= max_slots) ++end;
      t.push_back(make_int2(static_cast<int>(r), s0));
      r = end;
    }
  }
  if (first_tile) first_tile->push_back(static_cast<int32_t>(t.size()));
  t.push_back(make_int2(static_cast<int>(n), rp[n]));
  return t;
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

// Returns GABP_OK or an error with *msg set.
// Row tiles of the FP32 sweeps and the residual: at most `slots` slots and
// `rows` rows per tile (a longer row is a tile of its own), the tile-local
// row id of every slot, and the heavy flag of every tile that holds a row of
// degree above `heavy_degree`.  Replaces the previous tiles.
cudaError_t set_row_tiles(Graph &g, int slots, int rows, int heavy_degree, cudaStream_t st) {
  const int64_t n = g.n;
  const std::vector<int2> tb =
      make_tiles(g.h_rp, n, slots, rows, g.ncol > 0 ? &g.col_rows : nullptr, &g.col_tiles_big);
  std::vector<uint16_t> lrow(g.E);
  for (size_t t = 0; t + 1 < tb.size(); ++t)
    for (int32_t r = tb[t].x; r < tb[t + 1].x; ++r)
      for (int32_t sl = g.h_rp[r]; sl < g.h_rp[r + 1]; ++sl)
        lrow[sl] = static_cast<uint16_t>(r - tb[t].x);
  std::vector<uint8_t> heavy(tb.size() - 1, 0);
  for (size_t t = 0; t + 1 < tb.size(); ++t)
    for (int32_t r = tb[t].x; r < tb[t + 1].x; ++r)
      if (g.h_rp[r + 1] - g.h_rp[r] > heavy_degree) heavy[t] = 1;
  // Row order inside every tile, longest rows first (stable): the warps of a
  // thread-per-row pass then take rows of similar length.
  std::vector<uint8_t> rord(n + kPad, 0);
  std::vector<int32_t> idx;
  for (size_t t = 0; t + 1 < tb.size(); ++t) {
    const int32_t r0 = tb[t].x, nr = tb[t + 1].x - r0;
    idx.resize(nr);
    for (int32_t k = 0; k < nr; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
      return g.h_rp[r0 + a + 1] - g.h_rp[r0 + a] > g.h_rp[r0 + b + 1] - g.h_rp[r0 + b];
    });
    for (int32_t k = 0; k < nr; ++k) rord[r0 + k] = static_cast<uint8_t>(idx[k]);
  }
  cudaFree(g.tiles_big); cudaFree(g.lrow_big); cudaFree(g.heavy_big); cudaFree(g.rord);
  g.tiles_big = nullptr;
  g.lrow_big = nullptr;
  g.heavy_big = nullptr;
  g.rord = nullptr;
  g.ntiles_big = static_cast<int32_t>(tb.size() - 1);
  g.tile_slots = slots;
  g.tile_rows = rows;
  g.heavy_degree = heavy_degree;
  cudaError_t ce = upload(&g.tiles_big, tb.data(), tb.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.lrow_big, lrow.data(), lrow.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.heavy_big, heavy.data(), heavy.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.rord, rord.data(), rord.size(), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  return ce;
}

gabp_status build_graph(Graph &g, int64_t n, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col, const double *val, const int64_t *rev,
                        const gabp_options &opt, cudaStream_t st, std::string *msg) {
  if (n < 1 || n > (int64_t{1} << 31) - 2) { *msg = "n out of range"; return GABP_ERR_INVALID_ARG; }
  if (!row_ptr || !col || !val) { *msg = "null CSR pointer"; return GABP_ERR_INVALID_ARG; }
  if (row_ptr[0] != 0 || row_ptr[n] != nnz || nnz < n) {
    *msg = "row_ptr must start at 0, end at nnz, and nnz >= n";
    return GABP_ERR_INVALID_ARG;
  }
  double amax = 0.0;
  std::vector<int64_t> diag_pos(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) { *msg = "row_ptr not monotone"; return GABP_ERR_INVALID_ARG; }
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (col[e] < 0 || col[e] >= n) { *msg = "column index out of range"; return GABP_ERR_INVALID_ARG; }
      if (e > row_ptr[i] && col[e] <= col[e - 1]) {
        *msg = "columns of a row must be strictly increasing";
        return GABP_ERR_INVALID_ARG;
      }
      if (!std::isfinite(val[e])) { *msg = "non-finite matrix value"; return GABP_ERR_INVALID_ARG; }
      amax = std::max(amax, std::fabs(val[e]));
      if (col[e] == i) diag_pos[i] = e;
    }
    if (diag_pos[i] < 0 || val[diag_pos[i]] == 0.0) {
      *msg = "missing or zero diagonal entry at row " + std::to_string(i);
      return GABP_ERR_ZERO_DIAG;
    }
  }
  // Twin (entry (j, i)) of every off-diagonal entry, from rev or by search.
  std::vector<int64_t> twin(nnz);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t j = col[e];
      if (j == i) { twin[e] = e; continue; }
      int64_t t;
      if (rev) {
        t = rev[e];
        if (t < row_ptr[j] || t >= row_ptr[j + 1] || col[t] != i) {
          *msg = "rev is not the reverse-edge permutation of the CSR";
          return GABP_ERR_NOT_SYMMETRIC;
        }
      } else {
        const int32_t *b = col + row_ptr[j], *en = col + row_ptr[j + 1];
        const int32_t *p = std::lower_bound(b, en, static_cast<int32_t>(i));
        if (p == en || *p != i) { *msg = "pattern of A is not symmetric"; return GABP_ERR_NOT_SYMMETRIC; }
        t = row_ptr[j] + (p - b);
      }
      if (std::fabs(val[t] - val[e]) > 1e-14 * amax) {
        *msg = "values of A are not symmetric";
        return GABP_ERR_NOT_SYMMETRIC;
      }
      twin[e] = t;
    }
  }
  // Slots: off-diagonal entries in CSR order.  A pair (i,j)/(j,i) whose
  // values are both zero is not an edge and gets no slot; otherwise both
  // directions get one (so every slot has a reverse slot).
  std::vector<int64_t> slot_of(nnz, -1);
  int64_t E = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] != i && (val[e] != 0.0 || val[twin[e]] != 0.0)) slot_of[e] = E++;
  if (E > (int64_t{1} << 31) - 64) { *msg = "too many off-diagonal entries"; return GABP_ERR_INVALID_ARG; }

  g.n = static_cast<int32_t>(n);
  g.E = E;
  g.h_rp.assign(n + 1, 0);
  g.h_col.resize(E);
  g.h_rev.resize(E);
  g.h_user_pos.resize(E);
  std::vector<double> a64(E), d64(n);
  std::vector<float> a32(E), d32(n);
  int max_deg = 0;
  for (int64_t i = 0; i < n; ++i) {
    d64[i] = val[diag_pos[i]];
    d32[i] = static_cast<float>(d64[i]);
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int64_t s = slot_of[e];
      if (s < 0) continue;
      g.h_col[s] = col[e];
      g.h_rev[s] = static_cast<int32_t>(slot_of[twin[e]]);
      g.h_user_pos[s] = e;
      a64[s] = val[e];
      // the same FP32 value in both slots of a pair (the in-place FP32 sweep
      // recomputes a message from the other slot's copy of A_ij)
      a32[s] = static_cast<float>(0.5 * (val[e] + val[twin[e]]));
    }
  }
  // row pointers over slots
  {
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
      g.h_rp[i] = static_cast<int32_t>(s);
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (slot_of[e] >= 0) ++s;
      max_deg = std::max<int>(max_deg, static_cast<int>(s - g.h_rp[i]));
    }
    g.h_rp[n] = static_cast<int32_t>(s);
  }
  g.max_degree = max_deg;

  // Lanes per row: the next power of two at or above the mean degree.
  int G = opt.group_lanes;
  if (G <= 0) {
    const double avg = static_cast<double>(E) / static_cast<double>(n);
    G = next_pow2(static_cast<int>(std::ceil(avg)));
  }
  g.group = std::min(32, std::max(2, next_pow2(G)));
  int big_s, big_r, small_s, small_r;
  tile_sizes(&big_s, &big_r, &small_s, &small_r);
  const std::vector<int2> ts = make_tiles(g.h_rp, n, small_s, small_r,
                                          g.ncol > 0 ? &g.col_rows : nullptr, &g.col_tiles_small);
  g.ntiles_small = static_cast<int32_t>(ts.size() - 1);
  if (opt.tile_slots > 0) big_s = opt.tile_slots;
  if (opt.tile_rows > 0) big_r = opt.tile_rows;
  cudaError_t ce = set_row_tiles(g, big_s, big_r, opt.heavy_degree > 0 ? opt.heavy_degree : kHeavyDegree, st);
  if (ce == cudaSuccess) ce = upload(&g.tiles_small, ts.data(), ts.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.rp, g.h_rp.data(), g.h_rp.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.col, g.h_col.data(), g.h_col.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.rev, g.h_rev.data(), g.h_rev.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.a64, a64.data(), a64.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.a32, a32.data(), a32.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.diag64, d64.data(), d64.size(), st);
  if (ce == cudaSuccess) ce = upload(&g.diag32, d32.data(), d32.size(), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) {
    prepare_kernels(g.group, opt.precision == GABP_PREC_MIXED_BF16);
    ce = cudaGetLastError();
  }
  if (ce != cudaSuccess) {
    *msg = std::string("device upload failed: ") + cudaGetErrorString(ce);
    return ce == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA;
  }
  return GABP_OK;
}

gabp_status build_systems(Graph &g, int32_t nsys, const int64_t *sys_row_off,
                          const int64_t *row_ptr, const int32_t *col, cudaStream_t st,
                          std::string *msg) {
  if (nsys < 1 || !sys_row_off || sys_row_off[0] != 0 || sys_row_off[nsys] != g.n) {
    *msg = "system offsets must start at 0 and end at n";
    return GABP_ERR_INVALID_ARG;
  }
  std::vector<int32_t> sys(g.n);
  for (int32_t s = 0; s < nsys; ++s) {
    const int64_t r0 = sys_row_off[s], r1 = sys_row_off[s + 1];
    if (r1 <= r0) { *msg = "every system needs at least one row"; return GABP_ERR_INVALID_ARG; }
    for (int64_t i = r0; i < r1; ++i) {
      sys[i] = s;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (col[e] < r0 || col[e] >= r1) {
          *msg = "an entry couples two systems (row " + std::to_string(i) + ")";
          return GABP_ERR_INVALID_ARG;
        }
    }
  }
  g.nsys = nsys;
  g.h_sys_row_off.assign(sys_row_off, sys_row_off + nsys + 1);
  cudaError_t ce = upload(&g.sys_of_row, sys.data(), sys.size(), st);
  if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void **>(&g.sys_bmax), sizeof(unsigned long long) * nsys);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(g.sys_bmax, 0, sizeof(unsigned long long) * nsys, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    *msg = std::string("device upload failed: ") + cudaGetErrorString(ce);
    return ce == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA;
  }
  return GABP_OK;
}

void free_graph(Graph &g) {
  cudaFree(g.sys_of_row); cudaFree(g.sys_bmax);
  g.sys_of_row = nullptr;
  g.sys_bmax = nullptr;
  cudaFree(g.tiles_big); cudaFree(g.tiles_small); cudaFree(g.lrow_big); cudaFree(g.heavy_big);
  cudaFree(g.rord);
  g.rord = nullptr;
  g.tiles_big = g.tiles_small = nullptr;
  g.lrow_big = nullptr;
  g.heavy_big = nullptr;
  cudaFree(g.rp); cudaFree(g.col); cudaFree(g.rev);
  cudaFree(g.a64); cudaFree(g.a32); cudaFree(g.diag64); cudaFree(g.diag32);
  g.rp = g.col = g.rev = nullptr;
  g.a64 = g.diag64 = nullptr;
  g.a32 = g.diag32 = nullptr;
}

}  // namespace gabp
