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
//
// All decisions are taken on the device (the controller in gabp_kernels.cu).
// Two drivers run the same kernels:
//   * graph driver (default): one CUDA graph per handle and mode -- an init
//     kernel, then a WHILE node around a SWITCH on the phase; the controller
//     sets both conditions.  One launch and one synchronisation per solve.
//   * host driver (gabp_options.profile = 1): the host reads the control
//     block after every phase and launches the next one, bracketing each
//     kernel with CUDA events to report per-kind device times.
#include "gabp_internal.h"

#include <algorithm>
#include <cfloat>
#include <chrono>
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

}  // namespace

namespace gabp {
// Message for gabp_last_error(NULL) from entry points that have no handle.
void set_thread_error(const std::string &msg) { g_create_error = msg; }
}  // namespace gabp

namespace {

// Device buffer with kPad elements of slack (the staged kernels round their
// bulk copies up to 16 bytes).
template <class T>
void ensure(T **p, size_t count) {
  if (!*p) {
    CK(cudaMalloc(reinterpret_cast<void **>(p), (count + kPad) * sizeof(T)));
    CK(cudaMemset(*p, 0, (count + kPad) * sizeof(T)));
  }
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

bool is_bf16(gabp_handle h) { return h->opt.precision == GABP_PREC_MIXED_BF16; }

void free_resident(Resident &r);
void zero_messages(gabp_handle h, cudaStream_t st, bool full);
void zero_multi_messages(gabp_handle h, cudaStream_t st);
gabp_status resident_solve(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                           int32_t *iters, bool *ran);

void ensure_common(gabp_handle h) {
  ensure(&h->red, 1);
  ensure(&h->ctl, 1);
  if (!h->ctl_host) CK(cudaMallocHost(reinterpret_cast<void **>(&h->ctl_host), sizeof(Ctl)));
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
}

// Dense Section VII batches: grid-sized message buffers and node sums.
void ensure_dense64(gabp_handle h) {
  Dense &d = *h->dense;
  if (d.have64) return;
  DenseView &v = d.v;
  for (int k = 0; k < 2; ++k) {
    if (k == 0 || !d.serial) {   // the serial schedule updates messages in place
      ensure(&v.Mz64[k], d.pairs);
      ensure(&v.Mx64[k], d.pairs);
    }
    ensure(&v.sum64[k], d.nodes);
  }
  d.have64 = true;
}

void ensure_dense32(gabp_handle h) {
  Dense &d = *h->dense;
  if (d.have32) return;
  DenseView &v = d.v;
  Buffers &B = h->buf;
  const size_t hb = (d.pairs + kPad) * (is_bf16(h) ? sizeof(__nv_bfloat162) : sizeof(float2));
  for (int k = 0; k < 2; ++k) {
    ensure(&v.sum32[k], d.nodes);
    ensure(&v.sumE[k], d.nodes);
    if (k == 1 && d.serial) continue;   // the serial schedule updates messages in place
    ensure(&v.M32[k], d.pairs);
    CK(cudaMalloc(&v.H[k], hb));
    CK(cudaMemset(v.H[k], 0, hb));
    if (is_bf16(h)) {   // FP32 mean messages for the precision ladder
      const size_t wb = (d.pairs + kPad) * sizeof(float2);
      CK(cudaMalloc(&v.H32[k], wb));
      CK(cudaMemset(v.H32[k], 0, wb));
    }
  }
  ensure(&v.C32, d.pairs);
  const size_t n = h->g.n;
  ensure(&B.invP32, n);
  ensure(&B.mon32[0], n); ensure(&B.mon32[1], n);
  ensure(&B.r64, n);
  ensure(&B.rhs32, n);
  d.have32 = true;
}

// Grid form: message planes (2 D Nh entries) and node slots (2 Nh).
void ensure_grid64(gabp_handle h) {
  Grid &G = *h->grid;
  if (G.have64) return;
  ensure(&h->buf.m64[0], G.planes());
  ensure(&h->buf.m64[1], G.planes());
  G.have64 = true;
}

void ensure_grid32(gabp_handle h) {
  Grid &G = *h->grid;
  if (G.have32) return;
  Buffers &B = h->buf;
  const size_t M = G.planes(), n = G.slots();
  ensure(&B.m32[0], M); ensure(&B.m32[1], M);
  const size_t eb = (M + kPad) * (is_bf16(h) ? sizeof(__nv_bfloat16) : sizeof(float));
  for (int k = 0; k < 2; ++k) {
    CK(cudaMalloc(&B.e[k], eb));
    CK(cudaMemset(B.e[k], 0, eb));
    if (is_bf16(h)) {   // FP32 mean messages for the precision ladder
      CK(cudaMalloc(&B.e32[k], (M + kPad) * sizeof(float)));
      CK(cudaMemset(B.e32[k], 0, (M + kPad) * sizeof(float)));
    }
  }
  ensure(&B.c32, M);
  if (h->opt.aitken > 0) ensure(&B.ait32, static_cast<size_t>(kAitLevels) * 3 * n);
  ensure(&B.invP32, n);
  ensure(&B.mon32[0], n); ensure(&B.mon32[1], n);
  ensure(&B.r64, n);
  ensure(&B.rhs32, n);
  G.have32 = true;
}

// Message entries of the handle's buffers (CSR slots, or grid planes).
size_t message_entries(gabp_handle h) { return h->grid ? h->grid->planes() : h->g.E; }

void ensure64(gabp_handle h) {
  ensure_common(h);
  if (h->dense) { ensure_dense64(h); return; }
  if (h->grid) { ensure_grid64(h); return; }
  if (h->have64) return;
  ensure(&h->buf.m64[0], h->g.E);
  ensure(&h->buf.m64[1], h->g.E);
  h->have64 = true;
}

void ensure32(gabp_handle h) {
  ensure_common(h);
  if (h->dense) { ensure_dense32(h); return; }
  if (h->grid) { ensure_grid32(h); return; }
  if (h->have32) return;
  const size_t n = h->g.n, E = h->g.E;
  Buffers &B = h->buf;
  ensure(&B.m32[0], E); ensure(&B.m32[1], E);
  const size_t eb = (E + kPad) * (is_bf16(h) ? sizeof(__nv_bfloat16) : sizeof(float));
  CK(cudaMalloc(&B.e[0], eb));
  CK(cudaMalloc(&B.e[1], eb));
  CK(cudaMemset(B.e[0], 0, eb));
  CK(cudaMemset(B.e[1], 0, eb));
  if (is_bf16(h)) {   // FP32 mean messages for the precision ladder
    for (int k = 0; k < 2; ++k) {
      CK(cudaMalloc(&B.e32[k], (E + kPad) * sizeof(float)));
      CK(cudaMemset(B.e32[k], 0, (E + kPad) * sizeof(float)));
    }
  }
  ensure(&B.c32, E);
  if (h->opt.aitken > 0) ensure(&B.ait32, static_cast<size_t>(kAitLevels) * 3 * n);
  ensure(&B.invP32, n);
  ensure(&B.mon32[0], n); ensure(&B.mon32[1], n);
  ensure(&B.tot32[0], n); ensure(&B.tot32[1], n);
  ensure(&B.r64, n);
  ensure(&B.rhs32, n);
  h->have32 = true;
}

// ---- profiling (host driver) ----
enum { K_FULL = 0, K_MEAN = 1, K_RES = 2, K_OTHER = 3 };
constexpr int kEventPairs = 64;

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

// Kernels of one phase on stream st (used by both drivers).
int launch_phase(gabp_handle h, cudaStream_t st, int phase) {
  const Graph &g = h->g;
  if (h->dense) {
    const Dense &d = *h->dense;
    switch (phase) {
      case PH_FULL64: return launch_dense_full64(d, st, h->buf, h->ctl, h->red);
      case PH_CHECK64: return launch_dense_residual(d, st, nullptr, h->ctl, h->red, false);
      case PH_FULL32: return launch_dense_full32(d, st, h->buf, h->ctl, h->red, is_bf16(h));
      case PH_MEAN: return launch_dense_mean(d, st, h->buf, h->ctl, h->red, is_bf16(h));
      case PH_MEANW: {   // FP32 mean messages after the ladder climbed (one controller)
        Dense w = d;
        w.v.H[0] = d.v.H32[0];
        w.v.H[1] = d.v.H32[1];
        return launch_dense_mean(w, st, h->buf, h->ctl, h->red, false);
      }
      case PH_REFINE:
        return launch_refine_update(g.n, st, h->buf, h->ctl) +
               launch_dense_residual(d, st, h->buf.r64, h->ctl, h->red, true);
    }
    return 0;
  }
  if (h->grid) {
    const Grid &G = *h->grid;
    Buffers B = h->buf;
    if (G.colour) {   // red-black: one in-place pass per class
      B.m64[1] = B.m64[0];
      B.m32[1] = B.m32[0];
      B.e[1] = B.e[0];
    }
    auto passes = [&](auto launch) {
      return G.colour ? launch(G.pass_view(0)) + launch(G.pass_view(1)) : launch(G.pass_view(-1));
    };
    switch (phase) {
      case PH_FULL64:
        return passes([&](const GridView &v) { return launch_grid_full64(v, st, B, h->ctl, h->red); });
      case PH_CHECK64:   // (Aitken: the extrapolated means first)
        return (h->opt.aitken > 0 ? launch_aitken(g.n, st, h->ctl, nullptr) : 0) +
               launch_grid_residual(G.v, st, nullptr, h->ctl, h->red, false);
      case PH_FULL32:
        return passes([&](const GridView &v) {
          return launch_grid_full32(v, st, B, h->ctl, h->red, is_bf16(h));
        });
      case PH_MEAN:
        return passes([&](const GridView &v) {
          return launch_grid_mean(v, st, B, h->ctl, h->red, is_bf16(h));
        });
      case PH_MEANW: {   // FP32 mean messages after the ladder climbed
        Buffers W = B;
        W.e[0] = B.e32[0];
        W.e[1] = G.colour ? B.e32[0] : B.e32[1];
        return passes([&](const GridView &v) {
          return launch_grid_mean(v, st, W, h->ctl, h->red, false);
        });
      }
      case PH_REFINE: {
        const int k = launch_refine_update(g.n, st, h->buf, h->ctl) +
                      launch_grid_residual(G.v, st, h->buf.r64, h->ctl, h->red, true);
        if (G.colour) zero_messages(h, st, false);   // the next inner solve starts from zero
        return k;
      }
    }
    return 0;
  }
  if (phase == PH_MEANR || phase == PH_MEANWR)   // the sweep, then its Aitken records
    return launch_phase(h, st, phase == PH_MEANR ? PH_MEAN : PH_MEANW) +
           launch_ait_record(g.n, st, h->buf, h->ctl);
  if (g.ncol > 0 && (phase == PH_FULL64 || phase == PH_FULL32 || phase == PH_MEAN ||
                    phase == PH_MEANK || phase == PH_MEANW)) {
    // colour schedule: one in-place pass per class (both parities alias one buffer)
    Buffers B = h->buf;
    B.m64[1] = B.m64[0];
    B.m32[1] = B.m32[0];
    B.e[1] = B.e[0];
    B.eK[1] = B.eK[0];
    int k = 0;
    for (int c = 0; c < g.ncol; ++c) {
      const GraphView v = g.colour_view(c);
      if (phase == PH_FULL64) k += launch_sweep64(g, st, B, h->ctl, h->red, &v);
      else if (phase == PH_FULL32) k += launch_sweep32(g, st, B, h->ctl, h->red, is_bf16(h), &v);
      else if (phase == PH_MEAN) k += launch_mean(g, st, B, h->ctl, h->red, is_bf16(h), &v);
      else if (phase == PH_MEANW) {   // FP32 mean messages after the ladder climbed
        Buffers W = B;
        W.e[0] = W.e[1] = B.e32[0];
        k += launch_mean(g, st, W, h->ctl, h->red, false, &v);
      }
      else k += launch_mean_multi(g, st, B, h->ctl, h->red, h->graph_K, &v);
    }
    return k;
  }
  switch (phase) {
    case PH_FULL64:
      return g.naive ? launch_naive64(g, st, h->buf, h->ctl, h->red)
                     : launch_sweep64(g, st, h->buf, h->ctl, h->red);
    case PH_CHECK64:
      return launch_check64(g, st, h->buf, h->ctl, h->red,
                            h->opt.aitken > 0 && h->opt.precision == GABP_PREC_FP64);
    case PH_FULL32: return launch_sweep32(g, st, h->buf, h->ctl, h->red, is_bf16(h));
    case PH_MEAN:
      return h->win.nwin > 0 ? launch_mean_win(g, h->win, st, h->buf, h->ctl, h->red, is_bf16(h))
                             : launch_mean(g, st, h->buf, h->ctl, h->red, is_bf16(h));
    case PH_MEANW: {   // FP32 mean messages after the ladder climbed (tile form)
      Buffers W = h->buf;
      W.e[0] = W.e32[0];
      W.e[1] = W.e32[1];
      return launch_mean(g, st, W, h->ctl, h->red, false);
    }
    case PH_REFINE: {
      const int k = launch_refine(g, st, h->buf, h->ctl, h->red);
      if (g.ncol > 0) zero_messages(h, st, false);   // the next inner solve starts from zero
      return k;
    }
    case PH_MEANK: return launch_mean_multi(g, st, h->buf, h->ctl, h->red, h->graph_K);
    case PH_REFINEK: {
      const int k = launch_refine_multi(g, st, h->buf, h->ctl, h->red, h->graph_K);
      if (g.ncol > 0) zero_multi_messages(h, st);   // the next inner solves start from zero
      return k;
    }
  }
  return 0;
}

// Colour schedule: the in-place passes read their message buffer from the
// start of an inner solve on, so it must hold zeros then.
void zero_messages(gabp_handle h, cudaStream_t st, bool full) {
  const size_t E = message_entries(h) + kPad;
  const Buffers &B = h->buf;
  if (full && B.m64[0]) CK(cudaMemsetAsync(B.m64[0], 0, sizeof(double2) * E, st));
  if (full && B.m32[0]) CK(cudaMemsetAsync(B.m32[0], 0, sizeof(float2) * E, st));
  if (B.e[0]) CK(cudaMemsetAsync(B.e[0], 0, (is_bf16(h) ? 2 : 4) * E, st));
  if (B.e32[0]) CK(cudaMemsetAsync(B.e32[0], 0, 4 * E, st));
}

// The K-column mean messages of the multi right-hand-side solve (colour schedule).
void zero_multi_messages(gabp_handle h, cudaStream_t st) {
  CK(cudaMemsetAsync(h->buf.eK[0], 0, sizeof(float) * h->g.E * h->graph_K, st));
}

// Launches of one message sweep: one, or one per colour class.
int passes_per_sweep(gabp_handle h) {
  if (h->grid) return h->grid->colour ? 2 : 1;
  return std::max(1, h->g.ncol);
}

int launch_mode_init(gabp_handle h, cudaStream_t st, int mode) {
  if (mode == CTL_MULTI) {
    if (h->g.ncol > 0) zero_multi_messages(h, st);
    return launch_init_multi(h->g, st, h->buf, h->ctl, h->red, h->graph_K);
  }
  if (h->g.ncol > 0 || (h->grid && h->grid->colour)) zero_messages(h, st, true);
  return launch_init(h->g, st, h->buf, h->ctl, h->red);
}

// The FP32-storage mean phase of the precision ladder: BF16 handles whose
// ladder is climbed by the controller (every form but a dense batch under
// per-system control, whose systems climb inside the sweeps).
bool ladder_phase(gabp_handle h) {
  return is_bf16(h) && !(h->dense && h->opt.batch_control == 0);
}

// The mean phases followed by the Aitken records: CSR handles of mixed
// solves with aitken > 0 (grid mean sweeps take their records themselves;
// dense handles have none).
bool ait_record_phase(gabp_handle h) {
  return !h->dense && !h->grid && h->buf.ait32 != nullptr;
}

bool phase_used(int mode, int p) {
  switch (mode) {
    case CTL_FP64: return p == PH_FULL64 || p == PH_CHECK64;
    case CTL_MIXED:
      return p == PH_FULL32 || p == PH_MEAN || p == PH_REFINE || p == PH_MEANW || p == PH_MEANR ||
             p == PH_MEANWR;
    case CTL_PREC: return p == PH_FULL32;
    case CTL_MULTI: return p == PH_MEANK || p == PH_REFINEK;
  }
  return false;
}

int phase_kind(int phase) {
  switch (phase) {
    case PH_FULL64: case PH_FULL32: return K_FULL;
    case PH_MEAN: case PH_MEANK: case PH_MEANW: case PH_MEANR: case PH_MEANWR: return K_MEAN;
    case PH_CHECK64: case PH_REFINE: case PH_REFINEK: return K_RES;
  }
  return K_OTHER;
}

// Records the solve graph of one control mode:
//   init -> WHILE(h_while) { SWITCH(h_phase) { phase bodies } }
void build_solve_graph(gabp_handle h, int mode) {
  cudaGraph_t graph;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle hw, hp;
  CK(cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&hp, graph, 0, cudaGraphCondAssignDefault));
  cudaStream_t cs = h->cap_stream;

  CK(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_mode_init(h, cs, mode);
  cudaGraph_t captured;
  CK(cudaStreamEndCapture(cs, &captured));
  size_t nn = 0;
  CK(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> roots(nn);
  CK(cudaGraphGetNodes(graph, roots.data(), &nn));

  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, graph, roots.data(), nullptr, nn, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];

  cudaGraphNodeParams sp{};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hp;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = PH_COUNT;
  cudaGraphNode_t snode;
  CK(cudaGraphAddNode(&snode, body, nullptr, nullptr, 0, &sp));
  for (int p = 0; p < PH_COUNT; ++p) {
    cudaGraph_t pb = sp.conditional.phGraph_out[p];
    if (!phase_used(mode, p) || ((p == PH_MEANW || p == PH_MEANWR) && !ladder_phase(h)) ||
        ((p == PH_MEANR || p == PH_MEANWR) && !ait_record_phase(h))) {
      cudaGraphNode_t e;
      CK(cudaGraphAddEmptyNode(&e, pb, nullptr, 0));
      continue;
    }
    CK(cudaStreamBeginCaptureToGraph(cs, pb, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_phase(h, cs, p);
    cudaGraph_t out;
    CK(cudaStreamEndCapture(cs, &out));
  }
  CK(cudaGraphInstantiate(&h->exec[mode], graph, 0));
  h->graph[mode] = graph;
  h->cond[mode][0] = hw;
  h->cond[mode][1] = hp;
}

// Control block of a solve, in the pinned host mirror.
void init_ctl(gabp_handle h, int mode, const double *b, double *x, double tol, int32_t max_iter,
              bool in_graph) {
  Ctl &c = *h->ctl_host;
  std::memset(&c, 0, sizeof(Ctl));
  c.b = b;
  c.x = x;
  c.tol = tol;
  c.rel = h->opt.residual_kind == GABP_RESIDUAL_REL;
  c.mode = mode;
  c.max_iter = max_iter;
  c.check_every = h->opt.check_every > 0 ? h->opt.check_every : 4;
  c.inner_tol = h->opt.inner_tol > 0 ? h->opt.inner_tol : (h->g.nsys > 0 ? 1e-6 : 1e-7);
  c.inner_goal = c.inner_tol;
  c.damping = h->opt.damping;
  c.in_graph = in_graph ? 1 : 0;
  if (in_graph) {
    c.h_while = h->cond[mode][0];
    c.h_phase = h->cond[mode][1];
  }
  c.xw = x;
  // Aitken's Delta^2 on the FP64 tentative means (per-sweep CSR path)
  if (h->opt.aitken > 0 && h->opt.precision == GABP_PREC_FP64 && !h->dense &&
      (mode == CTL_FP64 || mode == CTL_ROUNDS)) {
    const int s = h->opt.aitken;
    for (int k = 0; k < 3; ++k) {
      ensure(&h->ring[k], h->g.n);
      c.ring[k] = h->ring[k];
    }
    c.aitken = s;
    int ce = std::max(c.check_every, 2 * s);
    c.check_every = (ce + s - 1) / s * s;
  }
  c.first = 1;
  c.prev_dd = std::numeric_limits<double>::infinity();
  c.best_dd = std::numeric_limits<double>::infinity();
  // BF16 mean messages carry ~3 significant digits: inner solves level off
  // near 1e-2 relative change, where the refinement takes over
  c.floor_dd = is_bf16(h) ? 3e-2 : 1e-4;
  c.plateau = is_bf16(h) ? 16 : 0;
  // BF16 storage climbs to FP32 at the first stalled refinement step
  c.ladder = is_bf16(h) && mode == CTL_MIXED;
  c.floor_dd_wide = 1e-4;
  // Aitken on the inner solves of mixed grid solves
  c.ait_mixed = mode == CTL_MIXED && h->opt.aitken > 0 && h->buf.ait32 != nullptr;
  c.ait_rec = c.ait_mixed && ait_record_phase(h);
  c.ait_ok = 1;
  c.prev_dP = std::numeric_limits<double>::infinity();
  c.status = GABP_ERR_NOT_CONVERGED;
}

void finish_stats(gabp_handle h) {
  const Ctl &c = *h->ctl_host;
  gabp_stats &S = h->stats;
  S.sweeps_total = c.sweeps;
  S.sweeps_full = c.sweeps_full;
  S.sweeps_mean = c.sweeps_mean;
  S.outer_steps = (c.mode == CTL_MIXED || c.mode == CTL_MULTI) ? c.outer : 1;
  S.residual_checks = c.checks;
  S.status = c.status;
  S.residual = c.residual;
  S.rhs_norm = c.bnorm;
  S.n = h->g.n;
  S.edges = h->g.E;
  S.positions_swept = h->dense ? static_cast<int64_t>(c.positions) : 0;
  S.sweeps_wide = c.sweeps_wide;
  S.aitken_steps = c.ait_steps;
}

// Runs one control mode whose control block has been filled in the pinned
// mirror (init_ctl + mode fields): graph driver or, with profiling, host
// driver.  Leaves the final control block in the mirror.
void run_mode(gabp_handle h, int mode, int32_t max_iter) {
  cudaStream_t st = h->stream;
  const bool host_driver = h->opt.profile != 0;
  if (!host_driver) {
    if (mode == CTL_MULTI && h->exec[mode] && h->graph_K != h->ctl_host->K) {
      cudaGraphExecDestroy(h->exec[mode]);
      cudaGraphDestroy(h->graph[mode]);
      h->exec[mode] = nullptr;
      h->graph[mode] = nullptr;
    }
    if (mode == CTL_MULTI) h->graph_K = h->ctl_host->K;
    if (!h->exec[mode]) build_solve_graph(h, mode);
    h->ctl_host->in_graph = 1;
    h->ctl_host->h_while = h->cond[mode][0];
    h->ctl_host->h_phase = h->cond[mode][1];
  } else {
    if (mode == CTL_MULTI) h->graph_K = h->ctl_host->K;
    h->ctl_host->in_graph = 0;
  }
  CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h->red, 0, sizeof(DevScalars), st));
  if (!host_driver) {
    CK(cudaGraphLaunch(h->exec[mode], st));
    CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const Ctl &c = *h->ctl_host;
    const int per_check = (mode == CTL_MIXED || mode == CTL_MULTI) ? 2 : 1;
    if (c.retire)   // per-system control: refinement steps run inside the sweeps
      h->stats.kernel_launches += 1 + static_cast<int64_t>(c.sweeps) +
                                  (mode == CTL_FP64 ? static_cast<int64_t>(c.checks) : 0);
    else
      h->stats.kernel_launches += 1 + static_cast<int64_t>(c.sweeps) * passes_per_sweep(h) +
                                  static_cast<int64_t>(c.checks) * per_check;
  } else {
    run(h, K_OTHER, [&] { return launch_mode_init(h, st, mode); });
    const int64_t cap = 4 * static_cast<int64_t>(max_iter) + 128;
    for (int64_t it = 0; it < cap; ++it) {
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      prof_flush(h);
      if (h->ctl_host->done) break;
      const int phase = h->ctl_host->phase;
      run(h, phase_kind(phase), [&] { return launch_phase(h, st, phase); });
    }
  }
  CK(cudaGetLastError());
}

gabp_status report(gabp_handle h, const char *what) {
  const Ctl &c = *h->ctl_host;
  if (!c.done) return fail(h, GABP_ERR_NOT_CONVERGED, std::string(what) + ": controller did not finish");
  const gabp_status status = static_cast<gabp_status>(c.status);
  if (status != GABP_OK)
    return fail(h, status, std::string(what) + ": " + gabp_status_string(status) + ", residual " +
                               std::to_string(c.residual) + " after " + std::to_string(c.sweeps) +
                               " sweeps");
  return GABP_OK;
}

gabp_status solve_impl(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                       int32_t *iters) {
  const bool mixed = h->opt.precision != GABP_PREC_FP64;
  const int mode = mixed ? CTL_MIXED : CTL_FP64;
  double *x_out = x;
  if (h->perm) {   // colour schedule or grid form: solve in the renumbered order
    launch_permute(h->g.n, 1, h->stream, h->perm, b, h->bperm, false);
    b = h->bperm;
    x = h->xperm;
  }
  if (!mixed && h->res.C > 0 && !h->opt.profile && h->g.nsys == 0 && !h->dense) {
    bool ran = false;
    const gabp_status s = resident_solve(h, b, x, tol, max_iter, iters, &ran);
    if (ran) {
      if (h->perm) {
        launch_permute(h->g.n, 1, h->stream, h->perm, h->xperm, x_out, true);
        CK(cudaStreamSynchronize(h->stream));
      }
      return s;
    }
  }
  if (mixed) ensure32(h); else ensure64(h);
  h->stats = gabp_stats{};
  init_ctl(h, mode, b, x, tol, max_iter, false);
  if (h->g.nsys > 0) {
    h->ctl_host->batched = 1;
    CK(cudaMemsetAsync(h->g.sys_bmax, 0, sizeof(unsigned long long) * h->g.nsys, h->stream));
  }
  if (h->dense && h->opt.batch_control == 0) {   // per-system control
    Ctl &c = *h->ctl_host;
    c.retire = 1;
    c.nsys = c.sys_unfrozen = h->dense->nsys;
    CK(cudaMemsetAsync(h->dense->v.sysctl, 0, sizeof(SysCtl) * h->dense->nsys, h->stream));
  }
  run_mode(h, mode, max_iter);
  if (h->perm) {
    launch_permute(h->g.n, 1, h->stream, h->perm, h->xperm, x_out, true);
    CK(cudaStreamSynchronize(h->stream));
  }
  finish_stats(h);
  if (iters) *iters = h->ctl_host->sweeps;
  return report(h, mixed ? "mixed solve" : "FP64 solve");
}

// Section VII systems given psi_s = 0 (the Moore-Penrose solution; the
// reading and the kernels are in gabp_pinv.cu): iterated Tikhonov around the
// augmented solve.  Step 0 solves every system with [0; y]; from then on
// only the psi_s = 0 systems go on, with [S^T (y - S x^); 0] and the x^ part
// scaled by 1 / psi_0 (the others get a zero right-hand side, so their
// solutions stay as step 0 left them).  Ends when
// every such system has ||S^T (y - S x^)||_inf <= tol ||S^T y||_inf, with
// GABP_ERR_NOT_CONVERGED when the sweeps reach max_iter or the steps
// kPinvSteps, or with the status of a failed augmented solve.  Statistics:
// sweeps, checks, launches and profiled kernel times summed over the
// augmented solves; outer_steps =
// their number; residual / rhs_norm = the largest ||S^T (y - S x^)||_inf /
// ||S^T y||_inf of the psi_s = 0 systems.
constexpr int kPinvSteps = 500;

gabp_status lsq_pinv_solve(gabp_handle h, const double *y, double *xhat, double tol, int32_t max_iter,
                           int32_t *iters) {
  cudaStream_t st = h->stream;
  const int64_t n = h->g.n;
  const int32_t nsys = h->g.nsys;
  const int32_t *sor = h->g.sys_of_row;
  ensure(&h->lsq_u, n);
  ensure(&h->lsq_v, n);
  ensure(&h->lsq_gmax, nsys);
  std::vector<unsigned long long> gbits(nsys);
  auto offdiag = [&](const double *v, double *u) {
    if (h->dense) launch_dense_offdiag(*h->dense, st, v, u);
    else launch_csr_offdiag(h->g, st, v, u);
  };
  auto sysmax = [&](const double *u, std::vector<double> &out) {
    CK(cudaMemsetAsync(h->lsq_gmax, 0, sizeof(unsigned long long) * nsys, st));
    launch_pinv_sysmax(st, n, sor, h->lsq_aug_off, h->lsq_K, u, h->lsq_gmax);
    CK(cudaMemcpyAsync(gbits.data(), h->lsq_gmax, sizeof(unsigned long long) * nsys,
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out.resize(nsys);
    for (int32_t q = 0; q < nsys; ++q) out[q] = bits_to_double(gbits[q]);
  };
  // ||S^T y|| per system, and the first right-hand side [0; y]
  launch_lsq_rhs(st, n, sor, h->lsq_aug_off, h->lsq_K, h->lsq_y_off, y, h->lsq_rhs);
  offdiag(h->lsq_rhs, h->lsq_u);
  std::vector<double> g0, g;
  sysmax(h->lsq_u, g0);
  CK(cudaMemsetAsync(xhat, 0, sizeof(double) * h->lsq_nx, st));
  gabp_stats sum{};
  int64_t launches = 4;
  gabp_status status = GABP_ERR_NOT_CONVERGED;
  std::string why = "lsq solve: " + std::to_string(kPinvSteps) + " augmented solves";
  double worst = 0.0, worst_ref = 0.0;
  int steps = 0;
  while (steps < kPinvSteps && sum.sweeps_total < max_iter) {
    int32_t it = 0;
    const gabp_status s = solve_impl(h, h->lsq_rhs, h->lsq_x, tol, max_iter - sum.sweeps_total, &it);
    ++steps;
    sum.sweeps_total += h->stats.sweeps_total;
    sum.sweeps_full += h->stats.sweeps_full;
    sum.sweeps_mean += h->stats.sweeps_mean;
    sum.residual_checks += h->stats.residual_checks;
    sum.ms_full += h->stats.ms_full;
    sum.ms_mean += h->stats.ms_mean;
    sum.ms_residual += h->stats.ms_residual;
    sum.ms_other += h->stats.ms_other;
    launches += h->stats.kernel_launches;
    if (s != GABP_OK) {
      status = s;
      why = h->last_error;
      break;
    }
    // the first solve is x^ itself; a later one, from [g; 0], is psi_0 times the step
    launch_pinv_update(st, n, sor, h->lsq_aug_off, h->lsq_K, h->lsq_x_off,
                       steps == 1 ? nullptr : h->lsq_inv_psi0, h->lsq_x, xhat);
    // g = S^T (y - S x^) of the psi_s = 0 systems (zero for the others): the
    // stop rule's residual and, as [g; 0], the next right-hand side
    launch_pinv_embed(st, n, sor, h->lsq_aug_off, h->lsq_K, h->lsq_x_off, xhat, h->lsq_v);
    offdiag(h->lsq_v, h->lsq_u);
    launch_pinv_rhs(st, n, sor, h->lsq_aug_off, h->lsq_K, h->lsq_y_off, y, h->lsq_u, h->lsq_pinv,
                    h->lsq_v);
    offdiag(h->lsq_v, h->lsq_rhs);
    sysmax(h->lsq_rhs, g);
    launches += 6;
    bool done = true;
    worst = worst_ref = 0.0;
    for (int32_t q = 0; q < nsys; ++q) {
      if (!h->lsq_pinv_host[q]) continue;
      if (g0[q] > 0.0 && g[q] > tol * g0[q]) done = false;   // S^T y = 0: x^ = 0 from step 0
      if (g0[q] > 0.0 && g[q] / g0[q] >= worst / std::max(worst_ref, DBL_MIN)) {
        worst = g[q];
        worst_ref = g0[q];
      }
    }
    if (done) {
      status = GABP_OK;
      break;
    }
    why = "lsq solve: normal-equation residual " + std::to_string(worst) + " of " +
          std::to_string(worst_ref) + " after " + std::to_string(steps) + " augmented solves";
  }
  sum.outer_steps = steps;
  sum.status = status;
  sum.residual = worst;
  sum.rhs_norm = worst_ref;
  sum.n = h->g.n;
  sum.edges = h->g.E;
  sum.kernel_launches = launches;
  h->stats = sum;
  if (iters) *iters = sum.sweeps_total;
  return status == GABP_OK ? GABP_OK : fail(h, status, why);
}

void ensure_multi(gabp_handle h, int K) {
  if (h->capK >= static_cast<size_t>(K)) return;
  Buffers &B = h->buf;
  cudaFree(B.eK[0]); cudaFree(B.eK[1]); cudaFree(B.dK); cudaFree(B.rhsK); cudaFree(B.rK);
  B.eK[0] = B.eK[1] = B.dK = B.rhsK = nullptr;
  B.rK = nullptr;
  MultiCols &C = h->cols;
  cudaFree(C.bnorm); cudaFree(C.thr); cudaFree(C.rn); cudaFree(C.inv_rn);
  cudaFree(C.bmax); cudaFree(C.rmax);
  C = MultiCols{};
  h->capK = 0;
  const size_t n = h->g.n, E = h->g.E;
  ensure(&B.eK[0], E * K); ensure(&B.eK[1], E * K);
  ensure(&B.dK, n * K); ensure(&B.rhsK, n * K); ensure(&B.rK, n * K);
  ensure(&C.bnorm, K); ensure(&C.thr, K); ensure(&C.rn, K); ensure(&C.inv_rn, K);
  ensure(&C.bmax, K); ensure(&C.rmax, K);
  h->capK = K;
}

// Mixed-mode multi right-hand-side solve: precisions once (CTL_PREC), then
// all K columns together (CTL_MULTI).
gabp_status solve_multi_mixed(gabp_handle h, const double *B, double *X, int32_t K, double tol,
                              int32_t max_iter, int32_t *iters) {
  ensure32(h);
  ensure_multi(h, K);
  h->stats = gabp_stats{};
  init_ctl(h, CTL_PREC, nullptr, nullptr, tol, max_iter, false);
  run_mode(h, CTL_PREC, max_iter);
  const int prec_sweeps = h->ctl_host->sweeps;
  gabp_status s = report(h, "precision phase");
  if (s != GABP_OK) {
    finish_stats(h);
    if (iters) *iters = prec_sweeps;
    return s;
  }
  double *X_user = X;
  if (h->g.ncol > 0) {   // colour schedule: the columns in the renumbered row order
    const size_t nk = static_cast<size_t>(h->g.n) * K;
    if (h->capKperm < nk) {
      cudaFree(h->bKperm);
      cudaFree(h->xKperm);
      h->bKperm = h->xKperm = nullptr;
      h->capKperm = 0;
      ensure(&h->bKperm, nk);
      ensure(&h->xKperm, nk);
      h->capKperm = nk;
    }
    launch_permute(h->g.n, K, h->stream, h->perm, B, h->bKperm, false);
    B = h->bKperm;
    X = h->xKperm;
  }
  init_ctl(h, CTL_MULTI, nullptr, nullptr, tol, std::max(1, max_iter - prec_sweeps), false);
  Ctl &c = *h->ctl_host;
  c.K = K;
  c.Bm = B;
  c.Xm = X;
  c.cols = h->cols;
  c.frozen = 1;
  run_mode(h, CTL_MULTI, max_iter);
  if (h->g.ncol > 0) launch_permute(h->g.n, K, h->stream, h->perm, X, X_user, true);
  finish_stats(h);
  h->stats.sweeps_full = prec_sweeps;
  h->stats.sweeps_total = prec_sweeps + h->ctl_host->sweeps;
  if (iters) *iters = prec_sweeps + h->ctl_host->sweeps;
  return report(h, "multi right-hand-side solve");
}

// Section VII: the symmetric augmented system of every S_s (N_s x K_s,
// row-major at S + sum of earlier N_t K_t):
//   [ I_K   S^T  ] [x^]   [0]
//   [ S    -psi I] [z ] = [y]
// stored as one block-diagonal CSR, rows of x^ first in every block.
void build_lsq_csr(int32_t nsys, const int32_t *K, const int32_t *N, const double *S,
                   const double *psi, std::vector<int64_t> &row_ptr, std::vector<int32_t> &col,
                   std::vector<double> &val, std::vector<int64_t> &sys_off) {
  row_ptr.assign(1, 0);
  sys_off.assign(1, 0);
  int64_t soff = 0, base = 0;
  for (int32_t s = 0; s < nsys; ++s) {
    const int32_t k = K[s], m = N[s];
    const double *Ss = S + soff;
    for (int32_t r = 0; r < k; ++r) {   // x^_r: 1 on the diagonal, S_{j r} towards z_j
      col.push_back(static_cast<int32_t>(base + r));
      val.push_back(1.0);
      for (int32_t j = 0; j < m; ++j) {
        const double v = Ss[static_cast<int64_t>(j) * k + r];
        if (v != 0.0) { col.push_back(static_cast<int32_t>(base + k + j)); val.push_back(v); }
      }
      row_ptr.push_back(static_cast<int64_t>(col.size()));
    }
    for (int32_t j = 0; j < m; ++j) {   // z_j: S_{j r} towards x^_r, -psi on the diagonal
      for (int32_t r = 0; r < k; ++r) {
        const double v = Ss[static_cast<int64_t>(j) * k + r];
        if (v != 0.0) { col.push_back(static_cast<int32_t>(base + r)); val.push_back(v); }
      }
      col.push_back(static_cast<int32_t>(base + k + j));
      val.push_back(-psi[s]);
      row_ptr.push_back(static_cast<int64_t>(col.size()));
    }
    soff += static_cast<int64_t>(k) * m;
    base += k + m;
    sys_off.push_back(base);
  }
}

void release(gabp_handle h) {
  if (h->grid) {
    free_grid(*h->grid);
    delete h->grid;
    h->grid = nullptr;
  }
  for (int m = 0; m < CTL_MODES; ++m) {
    if (h->exec[m]) cudaGraphExecDestroy(h->exec[m]);
    if (h->graph[m]) cudaGraphDestroy(h->graph[m]);
  }
  cudaFree(h->buf.eK[0]); cudaFree(h->buf.eK[1]); cudaFree(h->buf.dK);
  cudaFree(h->buf.rhsK); cudaFree(h->buf.rK);
  cudaFree(h->cols.bnorm); cudaFree(h->cols.thr); cudaFree(h->cols.rn);
  cudaFree(h->cols.inv_rn); cudaFree(h->cols.bmax); cudaFree(h->cols.rmax);
  free_graph(h->g);
  free_windows(h->win);
  Buffers &B = h->buf;
  cudaFree(B.m64[0]); cudaFree(B.m64[1]);
  cudaFree(B.m32[0]); cudaFree(B.m32[1]); cudaFree(B.e[0]); cudaFree(B.e[1]);
  cudaFree(B.e32[0]); cudaFree(B.e32[1]);
  cudaFree(B.ait32);
  cudaFree(B.c32); cudaFree(B.invP32); cudaFree(B.mon32[0]); cudaFree(B.mon32[1]);
  cudaFree(B.tot32[0]); cudaFree(B.tot32[1]);
  cudaFree(B.r64); cudaFree(B.rhs32);
  cudaFree(h->red); cudaFree(h->ctl);
  cudaFree(h->bbuf); cudaFree(h->xbuf);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  cudaFree(h->lsq_K); cudaFree(h->lsq_aug_off); cudaFree(h->lsq_y_off); cudaFree(h->lsq_x_off);
  cudaFree(h->lsq_rhs); cudaFree(h->lsq_x);
  cudaFree(h->lsq_pinv); cudaFree(h->lsq_inv_psi0); cudaFree(h->lsq_u); cudaFree(h->lsq_v);
  cudaFree(h->lsq_gmax);
  cudaFree(h->diag_ns);
  if (h->dense) {
    DenseView &v = h->dense->v;
    for (int k = 0; k < 2; ++k) {
      cudaFree(v.M32[k]); cudaFree(v.Mz64[k]); cudaFree(v.Mx64[k]); cudaFree(v.H[k]);
      cudaFree(v.H32[k]);
      cudaFree(v.sum32[k]); cudaFree(v.sum64[k]); cudaFree(v.sumE[k]);
    }
    cudaFree(v.C32);
    cudaFree(const_cast<float *>(v.S32));
    cudaFree(const_cast<double *>(v.S64));
    cudaFree(h->dense->sys);
    cudaFree(v.sysctl);
    delete h->dense;
    h->dense = nullptr;
  }
  free_resident(h->res);
  for (double *&r : h->ring) { cudaFree(r); r = nullptr; }
  cudaFree(h->perm); cudaFree(h->bperm); cudaFree(h->xperm);
  cudaFree(h->bKperm); cudaFree(h->xKperm);
  h->perm = nullptr;
  h->bperm = h->xperm = h->bKperm = h->xKperm = nullptr;
  h->capKperm = 0;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
}

// Dense bipartite form of a Section VII batch: S uploaded as given (row-major
// N_s x K_s per system, which is the grid layout of the dense kernels) in FP64
// for the residual and FP32 for the sweeps; systems listed largest first so
// that the CTAs that claim them finish together.
void build_dense(gabp_handle h, int32_t nsys, const int32_t *K, const int32_t *N, const double *S,
                 const double *psi, const std::vector<int64_t> &node_off) {
  Dense *d = new Dense;
  h->dense = d;
  std::vector<DenseSys> sys(nsys);
  int64_t pairs = 0, nodes = 0;
  for (int32_t s = 0; s < nsys; ++s) {
    sys[s] = DenseSys{K[s], N[s], s, 0, pairs, nodes, psi[s]};
    pairs += static_cast<int64_t>(K[s]) * N[s];
    nodes += K[s] + N[s];
    d->maxK = std::max(d->maxK, K[s]);
    d->maxN = std::max(d->maxN, N[s]);
  }
  int64_t nnz = 0;
  std::vector<float> S32(pairs);
  for (int64_t p = 0; p < pairs; ++p) {
    S32[p] = static_cast<float>(S[p]);
    nnz += S[p] != 0.0;
  }
  std::stable_sort(sys.begin(), sys.end(), [](const DenseSys &a, const DenseSys &b) {
    return static_cast<int64_t>(a.K) * a.N > static_cast<int64_t>(b.K) * b.N;
  });
  std::vector<int32_t> sys_of_row(nodes);
  for (int32_t s = 0; s < nsys; ++s)
    for (int64_t i = node_off[s]; i < node_off[s + 1]; ++i) sys_of_row[i] = s;
  d->nsys = nsys;
  d->pairs = pairs;
  d->nodes = nodes;
  Graph &g = h->g;
  g.n = static_cast<int32_t>(nodes);
  g.E = 2 * nnz;
  g.nsys = nsys;
  g.h_sys_row_off = node_off;
  cudaStream_t st = h->stream;
  CK(cudaMalloc(reinterpret_cast<void **>(&g.sys_of_row), sizeof(int32_t) * nodes));
  CK(cudaMemcpyAsync(g.sys_of_row, sys_of_row.data(), sizeof(int32_t) * nodes,
                     cudaMemcpyHostToDevice, st));
  CK(cudaMalloc(reinterpret_cast<void **>(&g.sys_bmax), sizeof(unsigned long long) * nsys));
  CK(cudaMemsetAsync(g.sys_bmax, 0, sizeof(unsigned long long) * nsys, st));
  CK(cudaMalloc(reinterpret_cast<void **>(&d->sys), sizeof(DenseSys) * nsys));
  CK(cudaMemcpyAsync(d->sys, sys.data(), sizeof(DenseSys) * nsys, cudaMemcpyHostToDevice, st));
  CK(cudaMalloc(reinterpret_cast<void **>(&d->v.sysctl), sizeof(SysCtl) * nsys));
  CK(cudaMemsetAsync(d->v.sysctl, 0, sizeof(SysCtl) * nsys, st));
  float *S32d = nullptr;
  double *S64d = nullptr;
  ensure(&S32d, pairs);
  ensure(&S64d, pairs);
  d->v.S32 = S32d;   // owned by the handle from here on
  d->v.S64 = S64d;
  CK(cudaMemcpyAsync(S32d, S32.data(), sizeof(float) * pairs, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(S64d, S, sizeof(double) * pairs, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  d->v.sys = d->sys;
  d->v.nsys = nsys;
  d->v.pairs = pairs;
  d->v.sys_of_row = g.sys_of_row;
  d->v.sys_bmax = g.sys_bmax;
  prepare_dense_kernels(is_bf16(h));
}

// ---- small FP64 systems: the whole solve in one cluster launch ----
// Rows cut into C parts of about E / C slots each (cut points on the slot
// prefix sums); false if a part exceeds the per-CTA limits.
bool plan_resident(const Graph &g, int C, std::vector<int32_t> &row0, int *smax, int *rmax) {
  const int64_t n = g.n, E = g.E;
  row0.assign(C + 1, 0);
  for (int c = 1; c < C; ++c) {
    const int64_t target = E * c / C;
    const int64_t r = std::lower_bound(g.h_rp.begin(), g.h_rp.begin() + n + 1, target) - g.h_rp.begin();
    row0[c] = static_cast<int32_t>(std::max<int64_t>(row0[c - 1], std::min<int64_t>(r, n)));
  }
  row0[C] = static_cast<int32_t>(n);
  *smax = *rmax = 0;
  for (int c = 0; c < C; ++c) {
    *rmax = std::max(*rmax, row0[c + 1] - row0[c]);
    *smax = std::max(*smax, g.h_rp[row0[c + 1]] - g.h_rp[row0[c]]);
  }
  return *rmax <= kResidentMaxRows && *smax <= kResidentMaxSlots && *smax >= 1;
}

void free_resident(Resident &r) {
  cudaFree(r.row0); cudaFree(r.dst); cudaFree(r.colp); cudaFree(r.out);
  r = Resident{};
}

// Builds the cluster-resident layout for C CTAs; returns false (and leaves
// the handle without one) if the system does not fit.
bool build_resident(gabp_handle h, int C) {
  const Graph &g = h->g;
  std::vector<int32_t> row0;
  int smax = 0, rmax = 0;
  if (C < 1 || C > kResidentMaxCluster || !plan_resident(g, C, row0, &smax, &rmax)) return false;
  const int64_t n = g.n, E = g.E;
  std::vector<int32_t> part(n);
  for (int c = 0; c < C; ++c)
    for (int32_t i = row0[c]; i < row0[c + 1]; ++i) part[i] = c;
  std::vector<int32_t> dst(E), colp(E);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t s = g.h_rp[i]; s < g.h_rp[i + 1]; ++s) {
      const int32_t j = g.h_col[s], pj = part[j];
      dst[s] = (pj << 24) | (g.h_rev[s] - g.h_rp[row0[pj]]);
      colp[s] = (pj << 16) | (j - row0[pj]);
    }
  free_resident(h->res);
  Resident &r = h->res;
  ensure(&r.row0, C + 1);
  ensure(&r.dst, E);
  ensure(&r.colp, E);
  ensure(&r.out, 1);
  CK(cudaMemcpyAsync(r.row0, row0.data(), sizeof(int32_t) * (C + 1), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(r.dst, dst.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(r.colp, colp.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  r.C = C;
  r.smax = smax;
  r.rmax = rmax;
  return true;
}

// Default cluster: about 512 slots per CTA (2 .. 16 CTAs), grown until the
// parts fit.
void setup_resident(gabp_handle h) {
  const Graph &g = h->g;
  if (h->opt.small_form != 0 || h->g.ncol > kResidentMaxColours || g.E < 1 ||
      g.E > static_cast<int64_t>(kResidentMaxCluster) * kResidentMaxSlots ||
      g.n > kResidentMaxCluster * kResidentMaxRows)
    return;
  if (h->opt.cluster_ctas > 0) {
    build_resident(h, h->opt.cluster_ctas);
    return;
  }
  int C = 2;
  while (C < kResidentMaxCluster && g.E > static_cast<int64_t>(C) * 512) C *= 2;
  for (; C <= kResidentMaxCluster; C *= 2)
    if (build_resident(h, C)) return;
}

ResidentView resident_view(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                           int check_every) {
  const Graph &g = h->g;
  const Resident &r = h->res;
  ResidentView v{};
  v.row0 = r.row0;
  v.rp = g.rp;
  v.a64 = g.a64;
  v.diag64 = g.diag64;
  v.dst = r.dst;
  v.colp = r.colp;
  v.b = b;
  v.x = x;
  v.smax = r.smax;
  v.rmax = r.rmax;
  v.check_every = check_every;
  v.max_iter = max_iter;
  v.rel = h->opt.residual_kind == GABP_RESIDUAL_REL;
  v.tol = tol;
  v.damping = h->opt.damping;
  v.out = r.out;
  v.ncol = g.ncol;   // colour schedule: one pass per class (col_rows is empty without one)
  v.damp_last = g.damp_last;
  if (g.ncol > 0)
    for (int c = 0; c <= g.ncol; ++c) v.cb[c] = g.col_rows[c];
  return v;
}

// One-launch FP64 solve.  *ran = false when the device cannot place the
// cluster (the handle then keeps to the per-sweep path).
gabp_status resident_solve(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                           int32_t *iters, bool *ran) {
  int check_every = h->opt.check_every > 0 ? h->opt.check_every : 4;
  const int ait = h->opt.aitken;
  if (ait > 0) check_every = (std::max(check_every, 2 * ait) + ait - 1) / ait * ait;
  ResidentView v = resident_view(h, b, x, tol, max_iter, check_every);
  v.aitken = ait;
  const cudaError_t ce = launch_resident64(v, h->res.C, h->stream);
  if (ce == cudaErrorInvalidConfiguration) {
    free_resident(h->res);
    h->tuning.cluster_ctas = 0;
    *ran = false;
    return GABP_OK;
  }
  CK(ce);
  *ran = true;
  ResidentOut o{};
  CK(cudaMemcpyAsync(&o, h->res.out, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  gabp_stats &S = h->stats;
  S = gabp_stats{};
  S.sweeps_total = S.sweeps_full = o.sweeps;
  S.outer_steps = 1;
  S.residual_checks = o.checks;
  S.status = o.status;
  S.residual = o.residual;
  S.rhs_norm = o.bnorm;
  S.n = h->g.n;
  S.edges = h->g.E;
  S.kernel_launches = 1;
  if (iters) *iters = o.sweeps;
  const gabp_status st = static_cast<gabp_status>(o.status);
  if (st != GABP_OK)
    return fail(h, st, std::string("FP64 solve: ") + gabp_status_string(st) + ", residual " +
                           std::to_string(o.residual) + " after " + std::to_string(o.sweeps) +
                           " sweeps");
  return GABP_OK;
}

// ---- autotuner ----
int64_t num_sms_host() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// Milliseconds per launch of `launch` (CUDA events on the handle's stream,
// after one untimed launch).
template <class F>
float time_launches(gabp_handle h, int reps, F &&launch) {
  cudaEvent_t a, z;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&z));
  launch();
  CK(cudaEventRecord(a, h->stream));
  for (int k = 0; k < reps; ++k) launch();
  CK(cudaEventRecord(z, h->stream));
  CK(cudaEventSynchronize(z));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, z));
  CK(cudaEventDestroy(a));
  CK(cudaEventDestroy(z));
  CK(cudaGetLastError());
  return ms / reps;
}

// Control block for timing sweeps outside a solve: mixed mode, frozen
// precisions, not the first sweep (so every launch streams its inputs), b and
// x pointing at a scratch vector that the timed kernels never write.
void tuning_ctl(gabp_handle h) {
  ensure(&h->bbuf, h->g.n);
  init_ctl(h, CTL_MIXED, h->bbuf, h->bbuf, 1e-10, 1 << 30, false);
  Ctl &c = *h->ctl_host;
  c.first = 0;
  c.frozen = 1;
  c.rn = 1.0;
  c.inv_rn = 1.0;
  c.check_every = 1 << 30;
  CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->red, 0, sizeof(DevScalars), h->stream));
}

void fill_tuning(gabp_handle h) {
  gabp_tuning &t = h->tuning;
  t.tile_slots = h->g.tile_slots;
  t.tile_rows = h->g.tile_rows;
  t.heavy_degree = h->g.heavy_degree;
  t.group_lanes = h->g.group;
  t.pull_lanes = h->g.pull_lanes;
  t.mean_window = h->win.nwin > 0 ? h->win.target : 0;
  t.windows = h->win.nwin;
  const bool rows = h->dense && !h->dense->serial;   // the serial kernels take whole rows
  t.dense_rows_mean = rows ? h->dense->rows_mean : 0;
  t.dense_rows_full = rows ? h->dense->rows_full : 0;
  t.cluster_ctas = h->res.C;
}

// Times the candidate launch shapes on the handle's own matrix (zero
// messages: the traffic and the work per launch do not depend on the values)
// and keeps the fastest.  Runs at create, before any solve graph is recorded.
void autotune(gabp_handle h) {
  const auto t0 = std::chrono::steady_clock::now();
  gabp_tuning &T = h->tuning;
  Graph &g = h->g;
  const bool mixed = h->opt.precision != GABP_PREC_FP64;
  const bool bf16 = is_bf16(h);
  if (h->dense) {
    if (mixed && h->opt.dense_rows == 0 && !h->dense->serial) {
      Dense &d = *h->dense;
      ensure32(h);
      float best = 1e30f;
      int pick = 2;
      for (int u : {1, 2, 4}) {
        d.rows_mean = u;
        tuning_ctl(h);
        const float ms = time_launches(h, 3, [&] { launch_dense_mean(d, h->stream, h->buf, h->ctl, h->red, bf16); });
        ++T.candidates;
        if (ms < best) { best = ms; pick = u; }
      }
      d.rows_mean = pick;
      best = 1e30f;
      pick = 2;
      for (int u : {1, 2, 4}) {
        d.rows_full = u;
        tuning_ctl(h);
        const float ms = time_launches(h, 2, [&] { launch_dense_full32(d, h->stream, h->buf, h->ctl, h->red, bf16); });
        ++T.candidates;
        if (ms < best) { best = ms; pick = u; }
      }
      d.rows_full = pick;
    }
  } else if (mixed) {
    ensure32(h);
    auto score = [&](int slots, int rows, int heavy) {
      CK(set_row_tiles(g, slots, rows, heavy, h->stream));
      tuning_ctl(h);
      const float tm = time_launches(h, 3, [&] { launch_mean(g, h->stream, h->buf, h->ctl, h->red, bf16); });
      const float tf = time_launches(h, 2, [&] { launch_sweep32(g, h->stream, h->buf, h->ctl, h->red, bf16); });
      ++T.candidates;
      return 4.0 * tm + tf;
    };
    const int slots0 = g.tile_slots, rows0 = g.tile_rows;
    double best = 1e300;
    int heavy = g.heavy_degree;
    if (h->opt.heavy_degree == 0) {
      for (int hd : {16, 32, 64, 128, 1 << 30}) {
        const double sc = score(slots0, rows0, hd);
        if (sc < best) { best = sc; heavy = hd; }
      }
    } else {
      best = score(slots0, rows0, heavy);
    }
    int slots = slots0, rows = rows0;
    if (h->opt.tile_slots == 0 && h->opt.tile_rows == 0) {
      const int shapes[][2] = {{512, 256}, {512, 128}, {256, 64}};
      for (const auto &sh : shapes) {
        const double sc = score(sh[0], sh[1], heavy);
        if (sc < best) { best = sc; slots = sh[0]; rows = sh[1]; }
      }
    }
    CK(set_row_tiles(g, slots, rows, heavy, h->stream));
    // form of the FP32 full sweep: scatter (on the tiles just chosen) or
    // in place with 2..32 lanes per row (synchronous, undamped handles)
    if (h->opt.pull_lanes == 0 && g.ncol == 0 && h->opt.damping == 0.0) {
      g.pull_lanes = 0;
      tuning_ctl(h);
      float best_f = time_launches(h, 2, [&] { launch_sweep32(g, h->stream, h->buf, h->ctl, h->red, bf16); });
      int pick = 0;
      for (int G : {2, 4, 8, 16, 32}) {
        g.pull_lanes = G;
        // positive node totals of "earlier rounds" (bytes 0x3F: 0.75f), so
        // that the timed rounds divide by ordinary numbers
        CK(cudaMemsetAsync(h->buf.tot32[0], 0x3F, sizeof(float2) * g.n, h->stream));
        CK(cudaMemsetAsync(h->buf.tot32[1], 0x3F, sizeof(float2) * g.n, h->stream));
        tuning_ctl(h);
        const float ms = time_launches(h, 2, [&] { launch_sweep32(g, h->stream, h->buf, h->ctl, h->red, bf16); });
        ++T.candidates;
        if (ms < best_f) { best_f = ms; pick = G; }
      }
      g.pull_lanes = pick;
    }
    // form of the mean sweep: the tiles just chosen, or windows of about
    // E / (SMs x m) slots (synchronous schedule)
    if (h->opt.mean_window == 0 && g.ncol == 0 && g.E > 0) {
      free_windows(h->win);
      tuning_ctl(h);
      float best_m = time_launches(h, 3, [&] { launch_mean(g, h->stream, h->buf, h->ctl, h->red, bf16); });
      int32_t pick = 0;
      const int64_t sms = num_sms_host();
      std::vector<int32_t> targets;
      for (int m : {3, 4, 6, 8}) {
        const int64_t t = std::min<int64_t>(24000, std::max<int64_t>(256, (g.E + sms * m - 1) / (sms * m)));
        if (std::find(targets.begin(), targets.end(), static_cast<int32_t>(t)) == targets.end())
          targets.push_back(static_cast<int32_t>(t));
      }
      for (int32_t t : targets) {
        std::string msg;
        if (build_windows(g, t, bf16, h->win, h->stream, &msg) != GABP_OK) continue;
        tuning_ctl(h);
        const float ms = time_launches(h, 3, [&] {
          launch_mean_win(g, h->win, h->stream, h->buf, h->ctl, h->red, bf16);
        });
        ++T.candidates;
        if (ms < best_m) { best_m = ms; pick = t; }
      }
      free_windows(h->win);
      if (pick > 0) {
        std::string msg;
        if (build_windows(g, pick, bf16, h->win, h->stream, &msg) != GABP_OK) free_windows(h->win);
      }
    }
  }
  if (!mixed && h->res.C > 0 && h->opt.cluster_ctas == 0) {
    // cluster size of the one-launch FP64 solve: 64 sweeps each, no early stop
    ensure(&h->bbuf, g.n);
    float best = 1e30f;
    int pick = h->res.C;
    for (int C : {2, 4, 8, 16}) {
      if (!build_resident(h, C)) continue;
      const ResidentView v = resident_view(h, h->bbuf, h->bbuf, 0.0, 64, 64);
      bool placed = true;
      const float ms = time_launches(h, 2, [&] {
        if (placed && launch_resident64(v, C, h->stream) == cudaErrorInvalidConfiguration) placed = false;
      });
      CK(cudaGetLastError());
      ++T.candidates;
      if (placed && ms < best) { best = ms; pick = C; }
    }
    if (!build_resident(h, pick)) free_resident(h->res);
  }
  if (h->dense || mixed || g.naive) {   // (Algorithm 1 has no lanes to tune)
  } else if (h->opt.group_lanes == 0) {
    ensure64(h);
    float best = 1e30f;
    int pick = g.group;
    for (int G : {2, 4, 8, 16, 32}) {
      g.group = G;
      prepare_kernels(G, false);
      tuning_ctl(h);
      const float ms = time_launches(h, 3, [&] { launch_sweep64(g, h->stream, h->buf, h->ctl, h->red); });
      ++T.candidates;
      if (ms < best) { best = ms; pick = G; }
    }
    g.group = pick;
  }
  T.tuned = 1;
  fill_tuning(h);
  T.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Colour schedule: greedy colouring in the caller's row order (the lowest
// colour no earlier neighbour holds; every off-diagonal CSR entry counts as
// an edge), then rows renumbered by (colour, row).  Fills the renumbered CSR
// (columns sorted), the class row offsets, the permutation and, per
// renumbered entry, the caller's entry.
struct ColourPlan {
  std::vector<int32_t> perm, iperm, bounds, col;
  std::vector<int64_t> rp, pos;
  std::vector<double> val;
};

bool plan_colours(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                  const double *val, ColourPlan &p, std::string *msg) {
  if (n < 1 || !row_ptr || !col || !val || row_ptr[0] != 0 || row_ptr[n] != nnz) {
    *msg = "invalid CSR";
    return false;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) { *msg = "row_ptr not monotone"; return false; }
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] < 0 || col[e] >= n) { *msg = "column index out of range"; return false; }
  }
  std::vector<int32_t> colour(n, -1), stamp;
  int32_t ncol = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t c = col[e] != i ? colour[col[e]] : -1;
      if (c >= 0) {
        if (static_cast<size_t>(c) >= stamp.size()) stamp.resize(c + 1, -1);
        stamp[c] = static_cast<int32_t>(i);
      }
    }
    int32_t c = 0;
    while (static_cast<size_t>(c) < stamp.size() && stamp[c] == i) ++c;
    colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  p.bounds.assign(ncol + 1, 0);
  for (int64_t i = 0; i < n; ++i) p.bounds[colour[i] + 1]++;
  for (int32_t c = 0; c < ncol; ++c) p.bounds[c + 1] += p.bounds[c];
  p.perm.resize(n);
  p.iperm.resize(n);
  std::vector<int32_t> next(p.bounds.begin(), p.bounds.end() - 1);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t k = next[colour[i]]++;
    p.perm[k] = static_cast<int32_t>(i);
    p.iperm[i] = k;
  }
  p.rp.assign(1, 0);
  p.col.clear(); p.val.clear(); p.pos.clear();
  p.col.reserve(nnz); p.val.reserve(nnz); p.pos.reserve(nnz);
  std::vector<std::pair<int32_t, int64_t>> row;
  for (int64_t k = 0; k < n; ++k) {
    const int32_t i = p.perm[k];
    row.clear();
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) row.emplace_back(p.iperm[col[e]], e);
    std::sort(row.begin(), row.end());
    for (const auto &ce : row) {
      p.col.push_back(ce.first);
      p.val.push_back(val[ce.second]);
      p.pos.push_back(ce.second);
    }
    p.rp.push_back(static_cast<int64_t>(p.col.size()));
  }
  return true;
}

// A handle with validated options and no matrix yet.
gabp_status new_handle(const gabp_options *opt, gabp_handle *out) {
  gabp_handle h = new (std::nothrow) gabp_s;
  if (!h) return GABP_ERR_OOM;
  if (opt) h->opt = *opt; else gabp_default_options(&h->opt);
  if (h->opt.precision < GABP_PREC_FP64 || h->opt.precision > GABP_PREC_MIXED_BF16) {
    delete h;
    g_create_error = "unknown precision mode";
    return GABP_ERR_INVALID_ARG;
  }
  if (!(h->opt.damping >= 0.0 && h->opt.damping < 1.0)) {
    delete h;
    g_create_error = "damping must lie in [0, 1)";
    return GABP_ERR_INVALID_ARG;
  }
  const gabp_options &o = h->opt;
  if (o.tile_slots < 0 || (o.tile_slots > 0 && (o.tile_slots < 32 || o.tile_slots > 1024)) ||
      o.tile_rows < 0 || o.tile_rows > 256 || o.heavy_degree < 0 ||
      !(o.cluster_ctas == 0 || o.cluster_ctas == 2 || o.cluster_ctas == 4 || o.cluster_ctas == 8 ||
        o.cluster_ctas == 16) || o.aitken < 0 || o.aitken > 64 || o.schedule < 0 || o.schedule > 1 ||
      !(o.dense_rows == 0 || o.dense_rows == 1 || o.dense_rows == 2 || o.dense_rows == 4)) {
    delete h;
    g_create_error = "launch shape out of range (tile_slots 32..1024, tile_rows 1..256, "
                     "heavy_degree >= 1, dense_rows 1, 2 or 4, cluster_ctas 2..16, aitken 0..64, schedule 0..1; "
                     "0 = automatic)";
    return GABP_ERR_INVALID_ARG;
  }
  if (o.damp_scope < 0 || o.damp_scope > 1 || (o.damp_scope == 1 && o.schedule != 1)) {
    delete h;
    g_create_error = "damp_scope must be 0, or 1 with schedule = 1";
    return GABP_ERR_INVALID_ARG;
  }
  if (!(o.naive == 0 || o.naive == 1) ||
      (o.naive == 1 && (o.schedule != 0 || o.damping != 0.0 || o.precision != GABP_PREC_FP64))) {
    delete h;
    g_create_error = "naive must be 0 or 1; Algorithm 1 (naive = 1) needs FP64, schedule 0 and damping 0";
    return GABP_ERR_INVALID_ARG;
  }
  if (o.batch_control < 0 || o.batch_control > 1) {
    delete h;
    g_create_error = "batch_control must be 0 (per system) or 1 (whole batch)";
    return GABP_ERR_INVALID_ARG;
  }
  if (o.mean_window < -1 || (o.mean_window > 0 && (o.mean_window < 256 || o.mean_window > 65536)) ||
      (o.mean_window > 0 && o.schedule != 0)) {
    delete h;
    g_create_error = "mean_window must be -1, 0 or 256..65536; the window form (> 0) needs schedule 0";
    return GABP_ERR_INVALID_ARG;
  }
  if (!(o.pull_lanes == -1 || o.pull_lanes == 0 || o.pull_lanes == 2 || o.pull_lanes == 4 ||
        o.pull_lanes == 8 || o.pull_lanes == 16 || o.pull_lanes == 32) ||
      (o.pull_lanes > 0 && (o.schedule != 0 || o.damping != 0.0))) {
    delete h;
    g_create_error = "pull_lanes must be -1, 0, 2, 4, 8, 16 or 32; the in-place form (> 0) needs "
                     "schedule 0 and damping 0";
    return GABP_ERR_INVALID_ARG;
  }
  h->stream = static_cast<cudaStream_t>(h->opt.stream);
  *out = h;
  return GABP_OK;
}

}  // namespace

extern "C" {

void gabp_default_options(gabp_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = GABP_PREC_FP64;
  opt->residual_kind = GABP_RESIDUAL_REL;
  opt->inner_tol = 0.0;   // automatic
}

gabp_status gabp_create(gabp_handle *out, int64_t n, int64_t nnz, const int64_t *row_ptr_host,
                        const int32_t *col_host, const double *val_host, const int64_t *rev_host,
                        const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID_ARG;
  *out = nullptr;
  g_create_error.clear();
  gabp_handle h = nullptr;
  if (const gabp_status s0 = new_handle(opt, &h); s0 != GABP_OK) return s0;
  h->user_nnz = nnz;
  gabp_status s = guarded(h, [&] {
    std::string msg;
    if (h->opt.schedule == 1) {
      // colour schedule: build the graph of the renumbered matrix
      ColourPlan cp;
      if (!plan_colours(n, nnz, row_ptr_host, col_host, val_host, cp, &msg)) {
        h->last_error = msg;
        return GABP_ERR_INVALID_ARG;
      }
      h->g.ncol = static_cast<int>(cp.bounds.size()) - 1;
      h->g.col_rows = cp.bounds;
      h->g.damp_last = h->opt.damp_scope == 1;
      gabp_status r = build_graph(h->g, n, nnz, cp.rp.data(), cp.col.data(), cp.val.data(), nullptr,
                                  h->opt, h->stream, &msg);
      if (r != GABP_OK) { h->last_error = msg; return r; }
      for (int64_t &q : h->g.h_user_pos) q = cp.pos[q];   // message export: the caller's entries
      ensure(&h->perm, n);
      ensure(&h->bperm, n);
      ensure(&h->xperm, n);
      CK(cudaMemcpyAsync(h->perm, cp.perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      return GABP_OK;
    }
    gabp_status r = build_graph(h->g, n, nnz, row_ptr_host, col_host, val_host, rev_host, h->opt,
                                h->stream, &msg);
    if (r != GABP_OK) h->last_error = msg;
    return r;
  });
  if (s == GABP_OK) {
    s = guarded(h, [&] {
      if (h->opt.precision == GABP_PREC_FP64 && !h->opt.naive) setup_resident(h);
      return GABP_OK;
    });
  }
  if (s == GABP_OK && h->opt.mean_window > 0 && h->opt.precision != GABP_PREC_FP64) {
    s = guarded(h, [&] {
      std::string msg;
      const gabp_status r = build_windows(h->g, h->opt.mean_window, is_bf16(h), h->win, h->stream, &msg);
      if (r != GABP_OK) h->last_error = msg;
      return r;
    });
  }
  if (s == GABP_OK) {
    if (h->opt.pull_lanes > 0) h->g.pull_lanes = h->opt.pull_lanes;
    h->g.naive = h->opt.naive == 1;
    fill_tuning(h);
    if (h->opt.autotune) s = guarded(h, [&] { autotune(h); return GABP_OK; });
  }
  if (s != GABP_OK) {
    g_create_error = h->last_error;
    release(h);
    delete h;
    return s;
  }
  *out = h;
  return GABP_OK;
}

gabp_status gabp_create_batched(gabp_handle *out, int32_t nsys, const int64_t *sys_row_off_host,
                                int64_t nnz, const int64_t *row_ptr_host, const int32_t *col_host,
                                const double *val_host, const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsys < 1 || !sys_row_off_host) {
    g_create_error = "gabp_create_batched: nsys < 1 or null offsets";
    return GABP_ERR_INVALID_ARG;
  }
  if (opt && opt->schedule != 0) {
    g_create_error = "gabp_create_batched: the colour schedule is not available for batched handles";
    return GABP_ERR_INVALID_ARG;
  }
  // block-diagonal structure is checked on the host before any device work
  const int64_t n = sys_row_off_host[nsys];
  if (sys_row_off_host[0] != 0 || n < 1 || !row_ptr_host || !col_host || row_ptr_host[n] != nnz) {
    g_create_error = "gabp_create_batched: offsets must run from 0 to n and row_ptr[n] == nnz";
    return GABP_ERR_INVALID_ARG;
  }
  for (int32_t sy = 0; sy < nsys; ++sy) {
    const int64_t r0 = sys_row_off_host[sy], r1 = sys_row_off_host[sy + 1];
    if (r1 <= r0) {
      g_create_error = "gabp_create_batched: every system needs at least one row";
      return GABP_ERR_INVALID_ARG;
    }
    for (int64_t i = r0; i < r1; ++i) {
      if (row_ptr_host[i] < 0 || row_ptr_host[i + 1] < row_ptr_host[i] || row_ptr_host[i + 1] > nnz) {
        g_create_error = "gabp_create_batched: row_ptr not monotone within [0, nnz]";
        return GABP_ERR_INVALID_ARG;
      }
      for (int64_t e = row_ptr_host[i]; e < row_ptr_host[i + 1]; ++e)
        if (col_host[e] < r0 || col_host[e] >= r1) {
          g_create_error = "gabp_create_batched: an entry couples two systems";
          return GABP_ERR_INVALID_ARG;
        }
    }
  }
  gabp_handle h = nullptr;
  gabp_status s = gabp_create(&h, n, nnz, row_ptr_host, col_host, val_host, nullptr, opt);
  if (s != GABP_OK) return s;
  s = guarded(h, [&] {
    std::string msg;
    gabp_status r = build_systems(h->g, nsys, sys_row_off_host, row_ptr_host, col_host, h->stream, &msg);
    if (r != GABP_OK) h->last_error = msg;
    return r;
  });
  if (s != GABP_OK) {
    g_create_error = h->last_error;
    gabp_destroy(h);
    return s;
  }
  *out = h;
  return GABP_OK;
}

gabp_status gabp_create_lsq_batched(gabp_handle *out, int32_t nsys, const int32_t *K_host,
                                    const int32_t *N_host, const double *S_host,
                                    const double *psi_host, const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsys < 1 || !K_host || !N_host || !S_host || !psi_host) {
    g_create_error = "gabp_create_lsq_batched: invalid argument";
    return GABP_ERR_INVALID_ARG;
  }
  for (int32_t s = 0; s < nsys; ++s)
    if (K_host[s] < 1 || N_host[s] < 1 || !(psi_host[s] >= 0.0) || !std::isfinite(psi_host[s])) {
      g_create_error = "gabp_create_lsq_batched: K_s, N_s >= 1 and psi_s >= 0 required";
      return GABP_ERR_INVALID_ARG;
    }
  const double shift = opt ? opt->pinv_shift : 0.0;
  if (!(shift >= 0.0) || !std::isfinite(shift)) {
    g_create_error = "gabp_create_lsq_batched: pinv_shift must be finite and >= 0";
    return GABP_ERR_INVALID_ARG;
  }
  // psi_s = 0 (the Moore-Penrose solution): the augmented matrix is built with
  // psi_0 = shift * (mean squared column norm of S_s) and the solve iterates
  // around it; every other system keeps its psi_s
  std::vector<double> psi_eff(psi_host, psi_host + nsys);
  std::vector<uint8_t> pinv(nsys, 0);
  bool any_pinv = false;
  {
    int64_t off = 0;
    for (int32_t s = 0; s < nsys; ++s) {
      const int64_t cnt = static_cast<int64_t>(K_host[s]) * N_host[s];
      if (psi_host[s] == 0.0) {
        double ss = 0.0;
        for (int64_t p = 0; p < cnt; ++p) ss += S_host[off + p] * S_host[off + p];
        const double col2 = ss / K_host[s];
        psi_eff[s] = (shift > 0.0 ? shift : 0.1) * (col2 > 0.0 ? col2 : 1.0);
        pinv[s] = 1;
        any_pinv = true;
      }
      off += cnt;
    }
  }
  psi_host = psi_eff.data();
  bool dense = !opt || opt->lsq_form == 0;
  for (int32_t s = 0; s < nsys && dense; ++s)
    dense = K_host[s] <= kDenseMaxK && N_host[s] <= kDenseMaxN;
  if (opt && opt->schedule != 0 && !dense) {
    g_create_error = "gabp_create_lsq_batched: the colour schedule needs the dense form (lsq_form 0, "
                     "K_s <= 256 and N_s <= 1024)";
    return GABP_ERR_INVALID_ARG;
  }
  gabp_handle h = nullptr;
  gabp_status s = GABP_OK;
  std::vector<int64_t> sys_off(1, 0);
  if (dense) {
    int64_t nodes = 0;
    for (int32_t k = 0; k < nsys; ++k) sys_off.push_back(nodes += K_host[k] + N_host[k]);
    if (nodes >= (int64_t{1} << 31) - 64) {
      g_create_error = "gabp_create_lsq_batched: more than 2^31 - 64 unknowns";
      return GABP_ERR_INVALID_ARG;
    }
    s = new_handle(opt, &h);
    if (s != GABP_OK) return s;
    s = guarded(h, [&] {
      build_dense(h, nsys, K_host, N_host, S_host, psi_host, sys_off);
      h->dense->serial = h->opt.schedule == 1;
      h->dense->v.damp_scope = h->opt.damp_scope;
      if (h->opt.dense_rows > 0) h->dense->rows_mean = h->dense->rows_full = h->opt.dense_rows;
      fill_tuning(h);
      if (h->opt.autotune) autotune(h);
      return GABP_OK;
    });
    if (s != GABP_OK) {
      g_create_error = h->last_error;
      gabp_destroy(h);
      return s;
    }
  } else {
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    try {
      build_lsq_csr(nsys, K_host, N_host, S_host, psi_host, row_ptr, col, val, sys_off);
    } catch (const std::bad_alloc &) {
      return GABP_ERR_OOM;
    }
    s = gabp_create_batched(&h, nsys, sys_off.data(), static_cast<int64_t>(col.size()),
                            row_ptr.data(), col.data(), val.data(), opt);
    if (s != GABP_OK) return s;
  }
  s = guarded(h, [&] {
    h->lsq_pinv_host = pinv;
    if (any_pinv) {
      std::vector<double> inv_psi0(nsys, 0.0);
      for (int32_t q = 0; q < nsys; ++q)
        if (pinv[q]) inv_psi0[q] = 1.0 / psi_eff[q];
      ensure(&h->lsq_pinv, nsys);
      ensure(&h->lsq_inv_psi0, nsys);
      CK(cudaMemcpyAsync(h->lsq_pinv, pinv.data(), nsys, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->lsq_inv_psi0, inv_psi0.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    std::vector<int64_t> y_off(nsys + 1, 0), x_off(nsys + 1, 0);
    for (int32_t k = 0; k < nsys; ++k) {
      y_off[k + 1] = y_off[k] + N_host[k];
      x_off[k + 1] = x_off[k] + K_host[k];
    }
    h->lsq_ny = y_off[nsys];
    h->lsq_nx = x_off[nsys];
    ensure(&h->lsq_K, nsys);
    ensure(&h->lsq_aug_off, nsys + 1);
    ensure(&h->lsq_y_off, nsys + 1);
    ensure(&h->lsq_x_off, nsys + 1);
    ensure(&h->lsq_rhs, h->g.n);
    ensure(&h->lsq_x, h->g.n);
    CK(cudaMemcpyAsync(h->lsq_K, K_host, sizeof(int32_t) * nsys, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->lsq_aug_off, sys_off.data(), sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->lsq_y_off, y_off.data(), sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->lsq_x_off, x_off.data(), sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GABP_OK;
  });
  if (s != GABP_OK) {
    g_create_error = h->last_error;
    gabp_destroy(h);
    return s;
  }
  *out = h;
  return GABP_OK;
}

gabp_status gabp_create_grid(gabp_handle *out, int32_t ndim, const int32_t *dims, int64_t nnz,
                             const int64_t *row_ptr_host, const int32_t *col_host,
                             const double *val_host, const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID_ARG;
  *out = nullptr;
  gabp_handle h = nullptr;
  gabp_status s = new_handle(opt, &h);
  if (s != GABP_OK) return s;
  s = guarded(h, [&] {
    h->grid = new Grid;
    std::vector<int32_t> perm;
    std::string msg;
    const gabp_status r = build_grid(*h->grid, ndim, dims, nnz, row_ptr_host, col_host, val_host,
                                     h->stream, perm, &msg);
    if (r != GABP_OK) {
      h->last_error = msg;
      return r;
    }
    Grid &G = *h->grid;
    G.colour = h->opt.schedule == 1;
    G.damp_last = h->opt.damp_scope == 1;
    const int64_t n = G.slots();
    h->g.n = static_cast<int32_t>(n);
    h->g.E = nnz - n;   // directed off-diagonal edges (the diagonal is in every row)
    h->user_nnz = nnz;
    ensure(&h->perm, n);
    ensure(&h->bperm, n);
    ensure(&h->xperm, n);
    CK(cudaMemcpyAsync(h->perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    fill_tuning(h);
    return GABP_OK;
  });
  if (s != GABP_OK) {
    g_create_error = h->last_error;
    gabp_destroy(h);
    return s;
  }
  *out = h;
  return GABP_OK;
}

gabp_status gabp_solve_lsq_batched(gabp_handle h, const double *y_dev, double *xhat_dev, double tol,
                                   int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!h->lsq_K) return fail(h, GABP_ERR_INVALID_ARG, "handle was not made by gabp_create_lsq_batched");
  if (!y_dev || !xhat_dev || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_lsq_batched: invalid argument");
  return guarded(h, [&] {
    cudaStream_t st = h->stream;
    if (h->lsq_pinv) return lsq_pinv_solve(h, y_dev, xhat_dev, tol, max_iter, iters);
    launch_lsq_rhs(st, h->g.n, h->g.sys_of_row, h->lsq_aug_off, h->lsq_K, h->lsq_y_off, y_dev,
                   h->lsq_rhs);
    const gabp_status s = solve_impl(h, h->lsq_rhs, h->lsq_x, tol, max_iter, iters);
    launch_lsq_extract(st, h->g.n, h->g.sys_of_row, h->lsq_aug_off, h->lsq_K, h->lsq_x_off,
                       h->lsq_x, xhat_dev);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    h->stats.kernel_launches += 2;
    return s;
  });
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
  if (!b_dev || !x_dev || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve: null pointer, invalid tol or max_iter < 1");
  return guarded(h, [&] { return solve_impl(h, b_dev, x_dev, tol, max_iter, iters); });
}

gabp_status gabp_solve_host(gabp_handle h, const double *b_host, double *x_host, double tol,
                            int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!b_host || !x_host || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_host: null pointer, invalid tol or max_iter < 1");
  return guarded(h, [&] {
    const size_t bytes = sizeof(double) * h->g.n;
    ensure(&h->bbuf, h->g.n);
    ensure(&h->xbuf, h->g.n);
    CK(cudaMemcpyAsync(h->bbuf, b_host, bytes, cudaMemcpyHostToDevice, h->stream));
    const gabp_status s = solve_impl(h, h->bbuf, h->xbuf, tol, max_iter, iters);
    CK(cudaMemcpyAsync(x_host, h->xbuf, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return s;
  });
}

gabp_status gabp_solve_multi(gabp_handle h, const double *B_dev, double *X_dev, int32_t nrhs,
                             double tol, int32_t max_iter, int32_t *iters) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!B_dev || !X_dev || nrhs < 1 || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_multi: invalid argument");
  // dense Section VII batches and grid handles solve the columns one after another
  const bool shared_precisions = h->opt.precision != GABP_PREC_FP64 && !h->dense && !h->grid;
  if (shared_precisions && nrhs > 256)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_solve_multi: at most 256 right-hand sides per call");
  if (shared_precisions)
    return guarded(h, [&] { return solve_multi_mixed(h, B_dev, X_dev, nrhs, tol, max_iter, iters); });
  return guarded(h, [&] {
    const int64_t n = h->g.n;
    ensure(&h->bbuf, n);
    ensure(&h->xbuf, n);
    int32_t total = 0;
    gabp_status worst = GABP_OK;
    std::string msg;
    for (int32_t k = 0; k < nrhs; ++k) {
      CK(cudaMemcpy2DAsync(h->bbuf, sizeof(double), B_dev + k, sizeof(double) * nrhs,
                           sizeof(double), n, cudaMemcpyDeviceToDevice, h->stream));
      int32_t it = 0;
      const gabp_status s = solve_impl(h, h->bbuf, h->xbuf, tol, max_iter, &it);
      total += it;
      CK(cudaMemcpy2DAsync(X_dev + k, sizeof(double) * nrhs, h->xbuf, sizeof(double),
                           sizeof(double), n, cudaMemcpyDeviceToDevice, h->stream));
      if (s != GABP_OK && worst == GABP_OK) { worst = s; msg = h->last_error; }
    }
    CK(cudaStreamSynchronize(h->stream));
    if (iters) *iters = total;
    if (worst != GABP_OK) h->last_error = msg;
    return worst;
  });
}

gabp_status gabp_set_profile(gabp_handle h, int32_t on) {
  if (!h || (on != 0 && on != 1)) return GABP_ERR_INVALID_ARG;
  h->opt.profile = on;
  return GABP_OK;
}

gabp_status gabp_get_tuning(gabp_handle h, gabp_tuning *tuning) {
  if (!h || !tuning) return GABP_ERR_INVALID_ARG;
  *tuning = h->tuning;
  return GABP_OK;
}

gabp_status gabp_check_wait_limit(gabp_handle h, int32_t limit_us, double *seconds_waited) {
  if (!h) return GABP_ERR_INVALID_ARG;
  constexpr int64_t kMaxUs = static_cast<int64_t>(kWaitLimitNs / 1000);
  if (limit_us < 0 || limit_us > kMaxUs)
    return fail(h, GABP_ERR_INVALID_ARG,
                "gabp_check_wait_limit: limit_us must be 0 (the library's limit) or 1.." +
                    std::to_string(kMaxUs));
  const unsigned long long limit_ns =
      limit_us == 0 ? kWaitLimitNs : static_cast<unsigned long long>(limit_us) * 1000ull;
  return guarded(h, [&] {
    cudaStream_t st = h->stream;
    ensure_common(h);   // control block and reductions (a fresh handle has none yet)
    ensure(&h->bbuf, h->g.n);
    ensure(&h->diag_ns, 1);
    init_ctl(h, CTL_FP64, h->bbuf, h->bbuf, 0.0, 1, false);
    CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->red, 0, sizeof(DevScalars), st));
    launch_wait_limit(st, h->ctl, h->red, limit_ns, h->diag_ns);
    CK(cudaGetLastError());
    unsigned long long ns = 0;
    CK(cudaMemcpyAsync(&ns, h->diag_ns, sizeof(ns), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (seconds_waited) *seconds_waited = 1e-9 * static_cast<double>(ns);
    return report(h, "wait-limit check");
  });
}

gabp_status gabp_get_stats(gabp_handle h, gabp_stats *stats) {
  if (!h || !stats) return GABP_ERR_INVALID_ARG;
  *stats = h->stats;
  return GABP_OK;
}

gabp_status gabp_get_system_sweeps(gabp_handle h, int32_t *sweeps_host, int32_t nsys) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!sweeps_host || h->g.nsys <= 0 || nsys != h->g.nsys)
    return fail(h, GABP_ERR_INVALID_ARG,
                "gabp_get_system_sweeps: not a batched handle, or nsys is not its number of systems");
  return guarded(h, [&] {
    if (h->dense && h->ctl_host->retire) {
      std::vector<SysCtl> sc(nsys);
      CK(cudaMemcpyAsync(sc.data(), h->dense->v.sysctl, sizeof(SysCtl) * nsys,
                         cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int32_t s = 0; s < nsys; ++s) sweeps_host[s] = sc[s].sweeps;
    } else {
      for (int32_t s = 0; s < nsys; ++s) sweeps_host[s] = h->stats.sweeps_total;
    }
    return GABP_OK;
  });
}

gabp_status gabp_run_rounds(gabp_handle h, const double *b_dev, int32_t rounds, double *x_dev) {
  if (!h) return GABP_ERR_INVALID_ARG;
  if (!b_dev || !x_dev || rounds < 0)
    return fail(h, GABP_ERR_INVALID_ARG, "gabp_run_rounds: invalid argument");
  return guarded(h, [&] {
    cudaStream_t st = h->stream;
    ensure64(h);
    double *x_user = x_dev;
    const bool in_place = h->g.ncol > 0 || (h->grid && h->grid->colour);
    if (h->perm) {   // colour schedule or grid form: the renumbered order
      launch_permute(h->g.n, 1, st, h->perm, b_dev, h->bperm, false);
      b_dev = h->bperm;
      x_dev = h->xperm;
    }
    if (in_place)    // one message buffer, read before it is written: from zero
      CK(cudaMemsetAsync(h->buf.m64[0], 0, sizeof(double2) * (message_entries(h) + kPad), st));
    init_ctl(h, CTL_ROUNDS, b_dev, x_dev, 0.0, rounds, false);
    Ctl &c = *h->ctl_host;
    c.rounds_target = rounds;
    // Aitken: the means of rounds R - 2s, R - s and R go to the ring
    const bool ait = c.aitken > 0 && rounds >= 2 * c.aitken;
    c.write_x = ait && (rounds == 2 * c.aitken);   // round 0 = R - 2s
    c.xw = ait ? c.ring[0] : x_dev;
    CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->red, 0, sizeof(DevScalars), st));
    // `rounds` message sweeps, then one pass that only writes the means.
    for (int32_t t = 0; t <= rounds; ++t) {
      if (h->dense) {
        launch_dense_full64(*h->dense, st, h->buf, h->ctl, h->red);
      } else if (h->grid && t < rounds) {
        launch_phase(h, st, PH_FULL64);   // one round: both classes, or the two passes
      } else if (h->grid) {
        Buffers B = h->buf;               // the means of the last round
        if (h->grid->colour) B.m64[1] = B.m64[0];
        launch_grid_full64(h->grid->pass_view(-1), st, B, h->ctl, h->red);
      } else if (h->g.ncol > 0 && t < rounds) {
        launch_phase(h, st, PH_FULL64);   // one round: the colour passes
      } else if (h->g.ncol > 0) {
        Buffers B = h->buf;               // the means of the last round: one buffer
        B.m64[1] = B.m64[0];
        launch_sweep64(h->g, st, B, h->ctl, h->red);
      } else if (h->g.naive) {
        launch_naive64(h->g, st, h->buf, h->ctl, h->red);   // (the last pass only infers)
      } else {
        launch_sweep64(h->g, st, h->buf, h->ctl, h->red);   // (the last pass only infers)
      }
    }
    if (ait) launch_aitken(h->g.n, st, h->ctl, x_dev);
    if (h->perm) launch_permute(h->g.n, 1, st, h->perm, h->xperm, x_user, true);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    DevScalars red{};
    CK(cudaMemcpyAsync(&red, h->red, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->m64_cur = h->g.ncol > 0 ? 0 : h->ctl_host->par_m;
    if (red.breakdown) return fail(h, GABP_ERR_BREAKDOWN, "breakdown during rounds");
    return GABP_OK;
  });
}

gabp_status gabp_get_messages(gabp_handle h, double *P_host, double *mu_host) {
  if (!h || !P_host || !mu_host) return GABP_ERR_INVALID_ARG;
  if (h->dense)
    return fail(h, GABP_ERR_INVALID_ARG,
                "gabp_get_messages: a dense Section VII batch has no caller CSR to lay messages out on");
  if (h->grid)
    return fail(h, GABP_ERR_INVALID_ARG,
                "gabp_get_messages: a grid handle keeps its messages per direction, not per CSR entry");
  return guarded(h, [&] {
    const Graph &g = h->g;
    std::memset(P_host, 0, sizeof(double) * h->user_nnz);
    std::memset(mu_host, 0, sizeof(double) * h->user_nnz);
    if (g.E == 0 || !h->have64) return GABP_OK;
    std::vector<double2> m(g.E);
    CK(cudaMemcpyAsync(m.data(), h->buf.m64[h->m64_cur], sizeof(double2) * g.E,
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

const char *gabp_version(void) { return "gabp-gb300 0.2 (sm_103a)"; }

}  // extern "C"
