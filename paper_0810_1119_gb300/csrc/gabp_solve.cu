// gabp_solve.cu -- solve drivers and the extern "C" entry points of gabp.h.
//
// FP64 mode: plain synchronous sweeps of Alg. 2 (every sweep updates the
// precision and mean messages), with the FP64 residual ||b - A x||_inf as the
// stop rule, evaluated every check_every sweeps.
//
// Mixed modes: FP32 messages inside FP64 iterative refinement.
//   outer step:  r = b - A x (FP64);  solve A d = r / ||r|| by FP32 GaBP;
//                x += ||r|| d (FP64);  stop when the FP64 residual meets tol.
//   The precision messages do not depend on the right-hand side (Alg. 2:
//   P_ij involves only A and other precisions), so the first inner solve runs
//   full FP32 sweeps until the node precisions P~_i settle, then freezes them
//   into c_ij = -A_ij / (P~_i - P_ji) and 1/P~_i; every later sweep is the
//   linear mean-only map eta_ij = c_ij (h~_i - eta_ji).
#include "gabp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>

using namespace gabp;

namespace {

struct CudaFail {
  cudaError_t err;
  const char *what;
};

#define CK(expr)                                                     \
  do {                                                               \
    cudaError_t _e = (expr);                                         \
    if (_e != cudaSuccess) throw CudaFail{_e, #expr};                \
  } while (0)

thread_local std::string g_create_error;

template <class T>
void ensure(T **p, size_t count) {
  if (!*p) CK(cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T)));
}

gabp_status fail(gabp_handle h, gabp_status s, const std::string &msg) {
  if (h) h->last_error = msg;
  return s;
}

template <class F>
gabp_status guarded(gabp_handle h, F &&f) {
  try {
    return f();
  } catch (const CudaFail &c) {
    const std::string m = std::string(c.what) + ": " + cudaGetErrorString(c.err);
    return fail(h, c.err == cudaErrorMemoryAllocation ? GABP_ERR_OOM : GABP_ERR_CUDA, m);
  } catch (const std::bad_alloc &) {
    return fail(h, GABP_ERR_OOM, "host allocation failed");
  }
}

constexpr double kTiny = std::numeric_limits<double>::min();

double dval(unsigned long long u) { return bits_to_double(u); }

void ensure_common(gabp_handle h) {
  ensure(&h->red, 1);
  if (!h->red_host) CK(cudaMallocHost(reinterpret_cast<void **>(&h->red_host), sizeof(DevScalars)));
}

void ensure64(gabp_handle h) {
  ensure_common(h);
  ensure(&h->m64[0], h->g.E);
  ensure(&h->m64[1], h->g.E);
}

void ensure32(gabp_handle h) {
  ensure_common(h);
  const size_t n = h->g.n, E = h->g.E;
  ensure(&h->m32[0], E); ensure(&h->m32[1], E);
  ensure(&h->e32[0], E); ensure(&h->e32[1], E);
  ensure(&h->c32, E);
  ensure(&h->invP32, n); ensure(&h->rhs32, n);
  ensure(&h->mon32[0], n); ensure(&h->mon32[1], n);
  ensure(&h->r64, n);
}

enum { K_FULL = 0, K_MEAN = 1, K_RES = 2, K_OTHER = 3 };
constexpr int kEventPairs = 64;

// Adds the device time of the recorded kernels to the stats (the stream has
// been synchronised by the caller).
void prof_flush(gabp_handle h) {
  for (int p = 0; p < h->ev_used; ++p) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[2 * p], h->ev[2 * p + 1]));
    gabp_stats &S = h->stats;
    double *slot = h->ev_kind[p] == K_FULL ? &S.ms_full
                 : h->ev_kind[p] == K_MEAN ? &S.ms_mean
                 : h->ev_kind[p] == K_RES  ? &S.ms_residual : &S.ms_other;
    *slot += ms;
  }
  h->ev_used = 0;
}

// Launches the kernels issued by f, counting them and, with profiling on,
// bracketing them with a pair of events on the handle's stream.
template <class F>
void run(gabp_handle h, int kind, F &&f) {
  int pair = -1;
  if (h->opt.profile) {
    if (h->ev.empty()) {
      h->ev.resize(2 * kEventPairs);
      h->ev_kind.resize(kEventPairs);
      for (cudaEvent_t &e : h->ev) CK(cudaEventCreate(&e));
    }
    if (h->ev_used == kEventPairs) {
      CK(cudaStreamSynchronize(h->stream));
      prof_flush(h);
    }
    pair = h->ev_used++;
    h->ev_kind[pair] = kind;
    CK(cudaEventRecord(h->ev[2 * pair], h->stream));
  }
  h->stats.kernel_launches += f();
  if (pair >= 0) CK(cudaEventRecord(h->ev[2 * pair + 1], h->stream));
}

void zero_scalars(gabp_handle h) { CK(cudaMemsetAsync(h->red, 0, sizeof(DevScalars), h->stream)); }

void read_scalars(gabp_handle h) {
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->red_host, h->red, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  prof_flush(h);
}

// ||b||_inf on the device.
double rhs_norm(gabp_handle h, const double *b) {
  zero_scalars(h);
  run(h, K_OTHER, [&] { return launch_max_abs(h->stream, b, h->g.n, &h->red->max_b); });
  read_scalars(h);
  return dval(h->red_host->max_b);
}

bool diverged(double rn, double bnorm) {
  return !std::isfinite(rn) || rn > 1e30 * std::max(bnorm, kTiny);
}

gabp_status solve_fp64(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                       int32_t *iters) {
  Graph &g = h->g;
  cudaStream_t st = h->stream;
  ensure64(h);
  gabp_stats &S = h->stats;
  S = gabp_stats{};
  S.n = g.n;
  S.edges = g.E;
  const double bnorm = rhs_norm(h, b);
  S.rhs_norm = bnorm;
  if (!std::isfinite(bnorm)) return fail(h, GABP_ERR_INVALID_ARG, "b has non-finite entries");
  const double thr = h->opt.residual_kind == GABP_RESIDUAL_REL ? tol * bnorm : tol;
  const int check = h->opt.check_every > 0 ? h->opt.check_every : 4;
  CK(cudaMemsetAsync(h->m64[0], 0, sizeof(double2) * std::max<int64_t>(g.E, 1), st));
  int cur = 0, t = 0;
  gabp_status status = GABP_ERR_NOT_CONVERGED;
  double rn = std::numeric_limits<double>::infinity();
  zero_scalars(h);
  if (max_iter <= 0) {
    // Round 0: all messages zero, x_i = b_i / A_ii.
    run(h, K_FULL, [&] { return launch_sweep64(g, st, h->m64[cur], h->m64[cur ^ 1], b, x, nullptr, h->red, false); });
    run(h, K_RES, [&] { return launch_residual64(g, st, b, x, nullptr, h->red); });
    read_scalars(h);
    S.residual_checks = 1;
    rn = dval(h->red_host->max_r);
    status = rn < thr ? GABP_OK : GABP_ERR_NOT_CONVERGED;
  }
  while (t < max_iter) {
    ++t;
    const bool chk = (t % check == 0) || t == max_iter;
    // Sweep t reads round t-1, writes round t and (on check sweeps) the
    // tentative means of round t-1.
    run(h, K_FULL, [&] { return launch_sweep64(g, st, h->m64[cur], h->m64[cur ^ 1], b, chk ? x : nullptr, nullptr, h->red, true); });
    cur ^= 1;
    if (!chk) continue;
    CK(cudaMemsetAsync(&h->red->max_r, 0, sizeof(unsigned long long), st));
    run(h, K_RES, [&] { return launch_residual64(g, st, b, x, nullptr, h->red); });
    read_scalars(h);
    ++S.residual_checks;
    if (h->red_host->breakdown) { status = GABP_ERR_BREAKDOWN; break; }
    rn = dval(h->red_host->max_r);
    if (rn < thr) { status = GABP_OK; break; }
    if (diverged(rn, bnorm)) { status = GABP_ERR_DIVERGED; break; }
  }
  h->m64_cur = cur;
  S.sweeps_total = S.sweeps_full = t;
  S.outer_steps = 1;
  S.residual = rn;
  S.status = status;
  if (iters) *iters = t;
  if (status != GABP_OK)
    return fail(h, status, std::string("FP64 solve: ") + gabp_status_string(status) +
                               ", residual " + std::to_string(rn));
  return GABP_OK;
}

gabp_status solve_mixed(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                        int32_t *iters) {
  Graph &g = h->g;
  cudaStream_t st = h->stream;
  ensure32(h);
  const int64_t n = g.n, E = std::max<int64_t>(g.E, 1);
  gabp_stats &S = h->stats;
  S = gabp_stats{};
  S.n = g.n;
  S.edges = g.E;
  const double bnorm = rhs_norm(h, b);
  S.rhs_norm = bnorm;
  if (!std::isfinite(bnorm)) return fail(h, GABP_ERR_INVALID_ARG, "b has non-finite entries");
  const double thr = h->opt.residual_kind == GABP_RESIDUAL_REL ? tol * bnorm : tol;
  const double inner_tol = h->opt.inner_tol > 0 ? h->opt.inner_tol : 1e-6;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  CK(cudaMemcpyAsync(h->r64, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double rn = bnorm;
  gabp_status status = GABP_ERR_NOT_CONVERGED;
  int sweeps = 0;
  if (rn < thr) status = GABP_OK;
  bool frozen = false;
  int mc = 0, ec = 0, pc = 0;
  while (status == GABP_ERR_NOT_CONVERGED) {
    ++S.outer_steps;
    run(h, K_OTHER, [&] { return launch_scale_to_f32(st, h->r64, n, 1.0 / rn, h->rhs32); });
    if (!frozen) {
      mc = 0;
      CK(cudaMemsetAsync(h->m32[mc], 0, sizeof(float2) * E, st));
    } else {
      CK(cudaMemsetAsync(h->e32[ec], 0, sizeof(float) * E, st));
    }
    CK(cudaMemsetAsync(h->mon32[pc], 0, sizeof(float2) * n, st));
    bool pending_freeze = false, inner_done = false;
    double prev_dd = std::numeric_limits<double>::infinity();
    double prev_dP = prev_dd;
    int k = 0, stall = 0;
    while (!inner_done && sweeps < max_iter) {
      zero_scalars(h);
      const int po = pc ^ 1;
      if (!frozen) {
        if (pending_freeze) {
          run(h, K_FULL, [&] { return launch_sweep32(g, st, h->m32[mc], nullptr, h->rhs32, h->mon32[pc], h->mon32[po], h->c32,
                         h->invP32, h->e32[ec], h->red); });
          frozen = true;
        } else {
          run(h, K_FULL, [&] { return launch_sweep32(g, st, h->m32[mc], h->m32[mc ^ 1], h->rhs32, h->mon32[pc], h->mon32[po],
                         nullptr, nullptr, nullptr, h->red); });
          mc ^= 1;
        }
        ++S.sweeps_full;
      } else {
        run(h, K_MEAN, [&] { return launch_mean32(g, st, h->e32[ec], h->e32[ec ^ 1], h->c32, h->invP32, h->rhs32, h->mon32[pc],
                      h->mon32[po], h->red); });
        ec ^= 1;
        ++S.sweeps_mean;
      }
      pc = po;
      ++sweeps;
      ++k;
      read_scalars(h);
      const DevScalars &R = *h->red_host;
      if (R.breakdown) { status = GABP_ERR_BREAKDOWN; break; }
      const double dd = dval(R.max_dx) / std::max(dval(R.max_x), kTiny);
      if (!std::isfinite(dd)) { status = GABP_ERR_DIVERGED; break; }
      if (!frozen && !pending_freeze) {
        // Precision convergence: relative change of the node precisions,
        // with the remaining error estimated from the contraction rate.
        const double dP = dval(R.max_dP) / std::max(dval(R.max_P), kTiny);
        const double rho = dP / prev_dP;
        const double errP = rho < 1.0 ? dP * rho / (1.0 - rho) : std::numeric_limits<double>::infinity();
        if (k >= 3 && (errP < 1e-6 || dP < 1e-7 || (rho >= 1.0 && dP < 1e-5))) pending_freeze = true;
        prev_dP = dP;
      }
      const double rho_d = dd / prev_dd;
      const double err_d = rho_d < 1.0 ? dd * rho_d / (1.0 - rho_d) : std::numeric_limits<double>::infinity();
      stall = rho_d >= 1.0 ? stall + 1 : 0;
      prev_dd = dd;
      if (frozen && k >= 3 && (err_d < inner_tol || (stall >= 2 && dd < 1e-4))) inner_done = true;
    }
    if (status != GABP_ERR_NOT_CONVERGED) break;
    // x += ||r|| d, then the FP64 residual.
    run(h, K_OTHER, [&] { return launch_refine_update(st, n, x, h->mon32[pc], rn); });
    CK(cudaMemsetAsync(&h->red->max_r, 0, sizeof(unsigned long long), st));
    run(h, K_RES, [&] { return launch_residual64(g, st, b, x, h->r64, h->red); });
    read_scalars(h);
    ++S.residual_checks;
    rn = dval(h->red_host->max_r);
    if (rn < thr) { status = GABP_OK; break; }
    if (diverged(rn, bnorm)) { status = GABP_ERR_DIVERGED; break; }
    if (sweeps >= max_iter) break;
  }
  S.sweeps_total = sweeps;
  S.residual = rn;
  S.status = status;
  if (iters) *iters = sweeps;
  if (status != GABP_OK)
    return fail(h, status, std::string("mixed solve: ") + gabp_status_string(status) +
                               ", residual " + std::to_string(rn));
  return GABP_OK;
}

gabp_status solve_dispatch(gabp_handle h, const double *b, double *x, double tol,
                           int32_t max_iter, int32_t *iters) {
  if (h->opt.precision == GABP_PREC_FP64) return solve_fp64(h, b, x, tol, max_iter, iters);
  return solve_mixed(h, b, x, tol, max_iter, iters);
}

void release(gabp_handle h) {
  free_graph(h->g);
  cudaFree(h->m64[0]); cudaFree(h->m64[1]); cudaFree(h->x_prev);
  cudaFree(h->m32[0]); cudaFree(h->m32[1]); cudaFree(h->e32[0]); cudaFree(h->e32[1]);
  cudaFree(h->c32); cudaFree(h->invP32); cudaFree(h->rhs32);
  cudaFree(h->mon32[0]); cudaFree(h->mon32[1]);
  cudaFree(h->xw); cudaFree(h->r64); cudaFree(h->red);
  cudaFree(h->bbuf); cudaFree(h->xbuf);
  if (h->red_host) cudaFreeHost(h->red_host);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
}

}  // namespace

extern "C" {

void gabp_default_options(gabp_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = GABP_PREC_FP64;
  opt->residual_kind = GABP_RESIDUAL_REL;
  opt->check_every = 0;
  opt->group_lanes = 0;
  opt->autotune = 0;
  opt->inner_tol = 1e-6;
  opt->stream = nullptr;
}

gabp_status gabp_create(gabp_handle *out, int64_t n, int64_t nnz, const int64_t *row_ptr_host,
                        const int32_t *col_host, const double *val_host, const int64_t *rev_host,
                        const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID_ARG;
  *out = nullptr;
  g_create_error.clear();
  gabp_handle h = new (std::nothrow) gabp_s;
  if (!h) return GABP_ERR_OOM;
  if (opt) h->opt = *opt; else gabp_default_options(&h->opt);
  if (h->opt.precision < GABP_PREC_FP64 || h->opt.precision > GABP_PREC_MIXED_BF16) {
    delete h;
    g_create_error = "unknown precision mode";
    return GABP_ERR_INVALID_ARG;
  }
  h->stream = static_cast<cudaStream_t>(h->opt.stream);
  h->user_nnz = nnz;
  gabp_status s = guarded(h, [&] {
    std::string msg;
    gabp_status r = build_graph(h->g, n, nnz, row_ptr_host, col_host, val_host, rev_host, h->opt,
                                h->stream, &msg);
    if (r != GABP_OK) h->last_error = msg;
    return r;
  });
  if (s != GABP_OK) {
    g_create_error = h->last_error;
    release(h);
    delete h;
    return s;
  }
  *out = h;
  return GABP_OK;
}

gabp_status gabp_destroy(gabp_handle h) {
  if (!h) return GABP_OK;
  cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
  return GABP_OK;
}

gabp_status gabp_set_stream(gabp_handle h, void *stream) {
  if (!h) return GABP_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  h->opt.stream = stream;
  return GABP_OK;
}

gabp_status gabp_solve(gabp_handle h, const double *b_dev, double *x_dev, double tol,
                       int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!b_dev || !x_dev || !(tol >= 0.0) || !std::isfinite(tol))
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve: null pointer or invalid tol");
  return guarded(h, [&] { return solve_dispatch(h, b_dev, x_dev, tol, max_iter, iters); });
}

gabp_status gabp_solve_host(gabp_handle h, const double *b_host, double *x_host, double tol,
                            int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!b_host || !x_host || !(tol >= 0.0) || !std::isfinite(tol))
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_host: null pointer or invalid tol");
  return guarded(h, [&] {
    const size_t bytes = sizeof(double) * h->g.n;
    ensure(&h->bbuf, h->g.n);
    ensure(&h->xbuf, h->g.n);
    CK(cudaMemcpyAsync(h->bbuf, b_host, bytes, cudaMemcpyHostToDevice, h->stream));
    const gabp_status s = solve_dispatch(h, h->bbuf, h->xbuf, tol, max_iter, iters);
    CK(cudaMemcpyAsync(x_host, h->xbuf, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return s;
  });
}

gabp_status gabp_solve_multi(gabp_handle h, const double *B_dev, double *X_dev, int32_t nrhs,
                             double tol, int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!B_dev || !X_dev || nrhs < 1 || !(tol >= 0.0) || !std::isfinite(tol))
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_multi: invalid argument");
  return guarded(h, [&] {
    const int64_t n = h->g.n;
    ensure(&h->bbuf, n);
    ensure(&h->xbuf, n);
    int32_t total = 0;
    gabp_status worst = GABP_OK;
    for (int32_t k = 0; k < nrhs; ++k) {
      CK(cudaMemcpy2DAsync(h->bbuf, sizeof(double), B_dev + k, sizeof(double) * nrhs,
                           sizeof(double), n, cudaMemcpyDeviceToDevice, h->stream));
      int32_t it = 0;
      const gabp_status s = solve_dispatch(h, h->bbuf, h->xbuf, tol, max_iter, &it);
      total += it;
      CK(cudaMemcpy2DAsync(X_dev + k, sizeof(double) * nrhs, h->xbuf, sizeof(double),
                           sizeof(double), n, cudaMemcpyDeviceToDevice, h->stream));
      if (s != GABP_OK && worst == GABP_OK) worst = s;
    }
    CK(cudaStreamSynchronize(h->stream));
    if (iters) *iters = total;
    return worst;
  });
}

gabp_status gabp_get_stats(gabp_handle h, gabp_stats *stats) {
  if (!h || !stats) return GABP_ERR_INVALID_ARG;
  *stats = h->stats;
  return GABP_OK;
}

gabp_status gabp_run_rounds(gabp_handle h, const double *b_dev, int32_t rounds, double *x_dev) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!b_dev || !x_dev || rounds < 0)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_run_rounds: invalid argument");
  return guarded(h, [&] {
    Graph &g = h->g;
    cudaStream_t st = h->stream;
    ensure64(h);
    zero_scalars(h);
    CK(cudaMemsetAsync(h->m64[0], 0, sizeof(double2) * std::max<int64_t>(g.E, 1), st));
    int cur = 0;
    for (int32_t t = 0; t < rounds; ++t) {
      run(h, K_FULL, [&] { return launch_sweep64(g, st, h->m64[cur], h->m64[cur ^ 1], b_dev, nullptr, nullptr, h->red, true); });
      cur ^= 1;
    }
    // Tentative means of the last round's messages (no messages written).
    run(h, K_FULL, [&] { return launch_sweep64(g, st, h->m64[cur], h->m64[cur ^ 1], b_dev, x_dev, nullptr, h->red, false); });
    h->m64_cur = cur;
    read_scalars(h);
    if (h->red_host->breakdown) return fail(h, GABP_ERR_BREAKDOWN, "breakdown during rounds");
    return GABP_OK;
  });
}

gabp_status gabp_get_messages(gabp_handle h, double *P_host, double *mu_host) {
  if (!h || !P_host || !mu_host) return GABP_ERR_INVALID_ARG;
  return guarded(h, [&] {
    const Graph &g = h->g;
    std::memset(P_host, 0, sizeof(double) * h->user_nnz);
    std::memset(mu_host, 0, sizeof(double) * h->user_nnz);
    if (g.E == 0 || !h->m64[h->m64_cur]) return GABP_OK;
    std::vector<double2> m(g.E);
    CK(cudaMemcpyAsync(m.data(), h->m64[h->m64_cur], sizeof(double2) * g.E,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // Slot s of row i holds m_{j->i}; it belongs at the CSR entry (j, i),
    // which is the entry of the reverse slot.
    for (int64_t s = 0; s < g.E; ++s) {
      const int64_t pos = g.h_user_pos[g.h_rev[s]];
      P_host[pos] = m[s].x;
      mu_host[pos] = m[s].x != 0.0 ? m[s].y / m[s].x : 0.0;
    }
    return GABP_OK;
  });
}

const char *gabp_last_error(gabp_handle h) {
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

const char *gabp_status_string(gabp_status s) {
  switch (s) {
    case GABP_OK: return "GABP_OK";
    case GABP_ERR_INVALID_ARG: return "GABP_ERR_INVALID_ARG";
    case GABP_ERR_NOT_SYMMETRIC: return "GABP_ERR_NOT_SYMMETRIC";
    case GABP_ERR_ZERO_DIAG: return "GABP_ERR_ZERO_DIAG";
    case GABP_ERR_BREAKDOWN: return "GABP_ERR_BREAKDOWN";
    case GABP_ERR_DIVERGED: return "GABP_ERR_DIVERGED";
    case GABP_ERR_NOT_CONVERGED: return "GABP_ERR_NOT_CONVERGED";
    case GABP_ERR_CUDA: return "GABP_ERR_CUDA";
    case GABP_ERR_OOM: return "GABP_ERR_OOM";
    case GABP_ERR_TIMEOUT: return "GABP_ERR_TIMEOUT";
  }
  return "GABP_UNKNOWN_STATUS";
}

const char *gabp_version(void) { return "gabp-gb300 0.1 (sm_103a)"; }

}  // extern "C"
