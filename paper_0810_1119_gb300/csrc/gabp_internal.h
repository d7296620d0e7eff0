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
//
// Control: every solve is driven by a small control block (Ctl) in device
// memory.  Kernels read their buffer parities and flags from it, and the last
// block of each controlling launch runs the decision logic (convergence,
// precision freeze, refinement, stop) and writes the next phase back, so a
// whole solve can run as one CUDA graph (a WHILE node around a SWITCH on the
// phase) with a single host synchronisation at the end.
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

// Device-side reduction slots.  Maxima of non-negative doubles are kept with
// 64-bit atomicMax on their bit patterns (IEEE order and unsigned order agree
// for non-negative values; NaN compares above +inf and so reads as "not
// finite").  The controller zeroes what it consumed.
struct DevScalars {
  unsigned long long max_dx;      // max_i |x_i^t - x_i^{t-1}|   (or |d| change)
  unsigned long long max_x;       // max_i |x_i^t|
  unsigned long long max_dP;      // max_i |P~_i^t - P~_i^{t-1}|
  unsigned long long max_P;       // max_i |P~_i^t|
  unsigned long long max_r;       // max_i |r_i|
  unsigned long long max_b;       // max_i |b_i|
  unsigned long long max_rrel;    // batched: max_i |r_i| / ||b_sys(i)||_inf
  int breakdown;                  // set when P~_i - P_ji is zero or not finite
  int timeout;                    // set when a bounded wait gave up
  int pad[2];
};

// Solve phases (the SWITCH index of the solve graph).
enum Phase : int {
  PH_FULL64 = 0,    // FP64 full sweep
  PH_CHECK64 = 1,   // FP64 residual check
  PH_FULL32 = 2,    // FP32 full sweep (freezes when pending_freeze is set)
  PH_MEAN = 3,      // mean-only sweep with frozen precisions
  PH_REFINE = 4,    // x += ||r|| d, r = b - A x
  PH_MEANK = 5,     // mean-only sweep of K right-hand sides at once
  PH_REFINEK = 6,   // X += ||r_k|| D, R = B - A X for K columns
  PH_MEANW = 7,     // mean-only sweep in FP32 storage once a BF16 handle's ladder climbed
  PH_MEANR = 8,     // PH_MEAN, then the Aitken records of the sweep (CSR handles)
  PH_MEANWR = 9,    // PH_MEANW, then the Aitken records of the sweep (CSR handles)
  PH_COUNT = 10,
  PH_DONE = 15
};

// CTL_PREC converges and freezes the precisions only (zero right-hand
// side); CTL_MULTI then solves K right-hand sides with them.
enum CtlMode : int { CTL_ROUNDS = 0, CTL_FP64 = 1, CTL_MIXED = 2, CTL_PREC = 3, CTL_MULTI = 4,
                     CTL_MODES = 5 };

// Per-column state of a multi right-hand-side solve (device arrays of K).
struct MultiCols {
  double *bnorm, *thr, *rn, *inv_rn;
  unsigned long long *bmax, *rmax;   // reductions (bit patterns of maxima)
};

struct Ctl {
  // ---- set by the host before a solve ----
  const double *b;          // right-hand side (device)
  double *x;                // solution (device)
  double tol;
  int rel;                  // 1 = relative residual
  int mode;                 // CtlMode
  int max_iter;
  int check_every;
  double inner_tol;
  double inner_goal;            // accuracy asked of the current inner solve (<= what the stop rule needs)
  int in_graph;             // 1 = set the graph's conditional handles
  int batched;              // 1 = independent systems, relative rule per system
  double damping;           // gamma: eta <- gamma eta_old + (1 - gamma) eta_new
  int rounds_target;        // CTL_ROUNDS: sweeps before the infer-only pass
  unsigned long long h_while, h_phase;
  // ---- state ----
  int phase;
  int par_m, par_e, par_mon;    // buffer parities: in = buf[par], out = buf[par ^ 1]
  int first;                    // first sweep of an inner solve: incoming messages are zero
  int second;                   // the sweep after the first one (its round-t-2 messages are zero)
  int write_x;                  // FP64: this sweep writes the tentative means
  int frozen, pending_freeze;
  int k, stall, sweeps, sweeps_full, sweeps_mean, outer, checks, steps;
  double prev_dd, prev_dP;
  double best_dd;               // smallest relative change of d in this inner solve
  int since_best;               // sweeps since best_dd last shrank by 10 %
  int plateau;                  // > 0: an inner solve also ends after this many such sweeps
  double floor_dd;              // relative change below which a stall ends an inner solve
  // BF16 mean storage, precision ladder (ladder = 1): after the first
  // refinement step that fails to shrink the residual by 10 %, the inner
  // solves store their mean messages in FP32 (wide = 1), with the FP32
  // storage's inner rule (floor_dd_wide, no plateau).  sweeps_wide counts the
  // mean-only sweeps that ran with FP32 storage; wide_now is set by a dense
  // sweep in which some system (per-system control) stored FP32 messages.
  int ladder, wide, sweeps_wide, wide_now;
  double floor_dd_wide;
  // Mixed solves with Aitken (ait_mixed = 1; grid and CSR handles, one
  // right-hand side): the mean sweeps record d every 2^j sweeps
  // (j = kAitMinLevel ...) of an inner solve, the last three records per
  // level; at the end of an inner solve of k sweeps the controller picks the
  // widest spacing s with 6 s <= k whose last three records come after sweep
  // ait_k0 (level ait_level, m = k / s records), and
  // the refinement update extrapolates the last three (ait_use) unless the
  // last extrapolated step failed to shrink the residual by 10 % (ait_ok = 0).
  // ait_md: max |d| of the last sweep.
  // ait_rec: the records are taken by a kernel of their own (CSR handles),
  // so the controller picks PH_MEANR / PH_MEANWR for sweeps 64, 128, ...
  // ait_k0: the number of the freeze sweep within the first inner solve
  // (full sweeps take no records; later inner solves have none).
  int ait_mixed, ait_rec, ait_use, ait_level, ait_m, ait_ok, ait_steps, ait_k0;
  double ait_md;
  double best_rn;               // smallest FP64 residual of the refinement so far
  int outer_stall;              // refinement steps since best_rn last halved
  double bnorm, thr, rn, inv_rn, residual;
  int status, done;
  unsigned int blocks_done;     // last-block detection counter
  unsigned int work_next;       // dense batches: next system to claim (reset by the last block)
  // Aitken's Delta^2 on the tentative means (FP64 sweeps): every `aitken`
  // sweeps the means go to ring[nw % 3]; a check extrapolates the last three
  // into x.  aitken = 0: the means go straight to x.
  int aitken, nw;
  double *ring[3];
  double *xw;                   // where the next sweep that writes means writes them
  int check_now;                // the sweep just run is followed by a residual check
  int e_slots;                  // the mean messages in e[par_e] are in the slot layout (written
                                // by a freeze sweep); window handles read them so once
  // Section VII batches in dense form with per-system control (retire = 1),
  // kept by the kernels' atomics: systems whose precisions are not frozen
  // yet, systems done and failed, the largest failure status, and the
  // largest final |r| and |r| / ||b_s|| over the systems that finished.
  // Also the grid positions swept (every dense solve).
  int retire;
  int nsys;
  int sys_unfrozen, sys_done, sys_failed, sys_fail_status;
  unsigned long long sys_rmax, sys_rrelmax;
  unsigned long long positions;
  int K;                        // CTL_MULTI: right-hand sides
  const double *Bm;             // CTL_MULTI: n x K right-hand sides (row-major)
  double *Xm;                   // CTL_MULTI: n x K solutions (row-major)
  MultiCols cols;               // CTL_MULTI: per-column state
};

// Device buffers of a handle, passed to the kernels by value.
struct Buffers {
  double2 *m64[2];
  float2 *m32[2];
  void *e[2];               // mean messages: float or bf16 (per precision mode)
  void *e32[2];             // BF16 handles: FP32 mean messages once the ladder climbs
  float *ait32;             // mixed solves with Aitken: kAitLevels x 3 records of d (n each)
  float *c32;               // frozen coefficients c_ij (slot s of row i)
  float *invP32;            // frozen 1/P~_i
  float2 *mon32[2];         // (P~_i, d_i) of the last two sweeps
  float2 *tot32[2];         // in-place FP32 full sweep: (P~_i, h~_i) of the last two rounds
  double *r64;              // FP64 residual
  float *rhs32;             // r_i / ||r|| of the current inner solve
  // multi right-hand sides (K columns, row-major n x K / E x K)
  float *eK[2];             // mean messages of all columns
  float *dK;                // d of the last sweep
  float *rhsK;              // scaled right-hand sides of the inner solve
  double *rK;               // FP64 residuals
};

// Row tiles: tiles[t] = (first row, first slot) of tile t, tiles[ntiles] =
// (n, E).  A tile holds at most a fixed number of slots and rows, except a
// single row with more slots, which is a tile of its own.
struct GraphView {
  const int32_t *rp, *rev, *col;
  const double *a64, *diag64;
  const float *a32, *diag32;
  const int2 *tiles_big, *tiles_small;
  const uint16_t *lrow_big;     // tile-local row id of every slot (big tiles)
  const uint8_t *heavy_big;     // 1 if the big tile holds a row of degree > kHeavyDegree
  const uint8_t *rord;          // per tile: its rows' local indices, longest rows first
  int32_t ntiles_big, ntiles_small;
  int32_t n;
  // batched handles: system of every row, per-system max |b| (bit patterns)
  const int32_t *sys_of_row;
  unsigned long long *sys_bmax;
  // colour schedule: this launch is one colour class's pass over its tiles,
  // in place in a single message buffer; only a sweep's last pass controls;
  // with damping limited to the last class the other passes do not blend
  int32_t in_place, no_control, no_damp;
  int32_t row0, row1;           // rows of the row-per-warp kernels: [row0, row1)
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
  int2 *tiles_big = nullptr, *tiles_small = nullptr;
  uint16_t *lrow_big = nullptr;
  uint8_t *heavy_big = nullptr;
  uint8_t *rord = nullptr;
  int32_t ntiles_big = 0, ntiles_small = 0;
  int group = 8;                 // lanes per row in the sweep kernels
  bool naive = false;            // FP64 sweep: Algorithm 1 (cavity sums taken directly)
  int pull_lanes = 0;            // FP32 full sweep: 0 = scatter form, else lanes per row of the
                                 // in-place form (synchronous schedule without damping)
  int tile_slots = 0, tile_rows = 0, heavy_degree = 0;   // row tiles of the FP32 sweeps
  // colour schedule: rows renumbered by colour class; class c holds rows
  // [col_rows[c], col_rows[c+1]) and tiles [col_tiles_*[c], col_tiles_*[c+1])
  int ncol = 0;
  std::vector<int32_t> col_rows, col_tiles_big, col_tiles_small;
  bool damp_last = false;   // damping blends only what the last class sends
  int max_degree = 0;
  // batched handles (independent systems along the diagonal)
  int32_t nsys = 0;
  int32_t *sys_of_row = nullptr;
  unsigned long long *sys_bmax = nullptr;
  std::vector<int64_t> h_sys_row_off;

  GraphView view() const {
    return GraphView{rp,        rev,        col,          a64, diag64,     a32,     diag32,
                     tiles_big, tiles_small, lrow_big,    heavy_big, rord, ntiles_big,
                     ntiles_small, n,        sys_of_row, sys_bmax, 0,   0, 0,
                     0,         n};
  }
  // The view of colour class c's pass (colour schedule): its tiles only.
  GraphView colour_view(int c) const {
    GraphView v = view();
    const int32_t b0 = col_tiles_big[c], b1 = col_tiles_big[c + 1];
    const int32_t s0 = col_tiles_small[c], s1 = col_tiles_small[c + 1];
    v.tiles_big = tiles_big + b0;
    v.heavy_big = heavy_big + b0;
    v.ntiles_big = b1 - b0;
    v.tiles_small = tiles_small + s0;
    v.ntiles_small = s1 - s0;
    v.in_place = 1;
    v.no_control = c + 1 < ncol;
    v.no_damp = damp_last && c + 1 < ncol;
    v.row0 = col_rows[c];
    v.row1 = col_rows[c + 1];
    return v;
  }
};

// Window form of the mean-only sweep (gabp_window.cu).  Windows are ranges of
// consecutive rows: win[w] = (first row, first slot), win[nwin] = (n, E).
// Every window also owns a padded range [R0[w], R0[w+1]) (a multiple of 8
// positions) of a second index space.  There the messages live in receive
// order -- bins[.] holds at window J's range the messages bound for J,
// grouped by source window -- and p2[R0[J] + k] = the window-local slot of
// element k.  In the same space, the send order of window I: outmap[R0[I] +
// q] = the window-local slot whose row sends the message of send position q
// (positions sorted by destination slot), cq[R0[I] + q] = its coefficient.
// sruns[r], r in [srun_ptr[I], srun_ptr[I+1]) = (first send position of the
// run, window-local; its first receive position), one run per destination
// window.  heavy_rows lists the rows of degree > 64.
struct WinView {
  const int2 *win;
  const int32_t *R0;
  const uint16_t *p2, *outmap;
  const int32_t *srun_ptr;
  const int2 *sruns;
  const int32_t *heavy_ptr, *heavy_rows;
  float *cq;
  void *bins[2];                // receive-ordered messages (float or bf16), one per parity
  int32_t nwin;
  int32_t rcap;                 // most rows of a window
  int32_t off_om, off_cq, off_slot, off_rows, off_srt, off_bits;   // shared-memory layout (bytes)
  int32_t nbits;                // words of the run-start bitmap
};

struct Win {
  int32_t nwin = 0, wcap = 0, runcap = 0, target = 0, rcap = 0;
  int32_t off_om = 0, off_cq = 0, off_slot = 0, off_rows = 0, off_srt = 0, off_bits = 0, nbits = 0;
  int32_t blocks = 0, grid = 0;   // CTAs per SM; CTAs of a launch
  int64_t nruns = 0;
  size_t smem = 0;              // dynamic shared memory per CTA
  int2 *win = nullptr;
  int32_t *R0 = nullptr;
  uint16_t *p2 = nullptr, *outmap = nullptr;
  int32_t *srun_ptr = nullptr;
  int2 *sruns = nullptr;
  int32_t *heavy_ptr = nullptr, *heavy_rows = nullptr;
  float *cq = nullptr;
  void *bins[2] = {nullptr, nullptr};
  WinView view() const;
};

// Kernel launchers (gabp_kernels.cu).  Each returns the number of kernels it
// launched; the last kernel of every launcher runs the controller in its
// last block.
int launch_init(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red);
int launch_sweep64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                   const GraphView *view = nullptr);
int launch_check64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                   bool aitken);
int launch_sweep32(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, bool bf16,
                   const GraphView *view = nullptr);
int launch_mean(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, bool bf16,
                const GraphView *view = nullptr);
// Rows of `width` doubles: dst[i] = src[perm[i]] (gather) or dst[perm[i]] = src[i] (scatter).
int launch_permute(int32_t n, int32_t width, cudaStream_t st, const int32_t *perm, const double *src,
                   double *dst, bool scatter);
int launch_refine(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red);
int launch_init_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K);
int launch_mean_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K,
                      const GraphView *view = nullptr);
int launch_refine_multi(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red, int K);
void prepare_kernels(int group, bool bf16);
void tile_sizes(int *big_slots, int *big_rows, int *small_slots, int *small_rows);
double bits_to_double(unsigned long long u);

// Rows of degree above this make a tile "heavy": the FP32 sweeps and the
// residual then spread the tile's slots over the threads instead of giving
// each thread a row.
constexpr int kHeavyDegree = 64;

// Extra elements allocated past the end of every array the kernels stage
// into shared memory: the bulk copies round their ends up to 16 bytes.
constexpr size_t kPad = 32;

// ---- Section VII batches in dense bipartite form (gabp_dense.cu) ----
// System s of a batch: K unknowns x^_r, N observations z_j, its N x K grid of
// edge weights S_jr (row-major, like the S given by the caller) at pairs
// [pair0, pair0 + N K), its K + N augmented nodes at [node0, node0 + K + N)
// (x^ first), and its index in the caller's order.
struct DenseSys {
  int32_t K, N, orig, pad;
  int64_t pair0, node0;
  double psi;
};

// Per-system state of a batched solve with per-system control (device, one
// per system, caller's order).  Every rule the controller applies to a whole
// solve -- the precision freeze, the end of an inner solve, the scale of the
// refinement, the stop rule, the stall of the refinement -- is applied to
// each system on its own numbers, and each system refines as soon as its own
// inner solve ends:
//   state   0 = iterating, 2 = done (met the stop rule), 3 = failed
//           (diverged, or eight refinement steps without a 10 % smaller
//           stop measure);
//   frozen  0 = full sweeps, 1 = its next sweep freezes the precisions,
//           2 = mean-only sweeps;
//   rn      the scale ||r_s||_inf of its current inner solve (the first inner
//           solve uses ||b_s||_inf);
//   k, prev_dd, best_dd, since_best, stall, prev_dP: the inner solve's sweep
//           count (k = 0: its next sweep is the first of an inner solve) and
//           the history of the relative changes of d and P~;
//   goal    the accuracy asked of its current inner solve: inner_tol at
//           first, then min(1e-2, max(inner_tol, 0.3 tol / its stop
//           measure)), so that an inner solve shrinks the residual only by
//           the factor the system's own stop rule still needs (inner_tol
//           again after a step without a 10 % gain);
//   outer, best_prog, outer_stall: refinement steps, the smallest stop
//           measure after one, and steps since it last shrank by 10 %;
//   wide    BF16 handles: the system's ladder climbed (its first stalled
//           refinement step), and its inner solves store FP32 mean messages.
struct SysCtl {
  double rn;
  double prev_dd, best_dd, prev_dP;
  double best_prog;
  double goal;                  // accuracy asked of its current inner solve
  int32_t k, stall, since_best;
  int32_t state, frozen;
  int32_t sweeps;               // message sweeps of this system in the solve
  int32_t outer, outer_stall;
  int32_t wide;                 // BF16 handles: its inner solves store FP32 mean messages
  int32_t pad;
};

// Aitken records of the mixed grid solves: spacings 2^6 ... 2^12 sweeps.
constexpr int kAitMinLevel = 6;
constexpr int kAitLevels = 7;

constexpr int kDenseMaxK = 256;    // largest K_s (and N_s) the dense kernels take
constexpr int kDenseMaxN = 1024;

// Device arrays of the dense form.  Grid position p = pair0 + j K + r holds
// both directed messages of the edge (z_j, x^_r):
//   full sweeps:  (Pz, eta_z, Px, eta_x), Pz/eta_z = message x^_r -> z_j and
//                 Px/eta_x = message z_j -> x^_r;
//   mean sweeps:  (eta_z, eta_x) with frozen coefficients (c_z, c_x).
// Per node: the sums over its incoming messages of the round held in the
// buffer of the same parity (sumP, sum eta).  The serial schedule keeps the
// messages in place in the buffers of index 0, one plane per direction.
struct DenseView {
  const DenseSys *sys;
  int32_t nsys;
  int64_t pairs;
  int32_t damp_scope;           // 1: damping blends only the z -> x^ messages (serial)
  const float *S32;
  const double *S64;
  float4 *M32[2];
  double2 *Mz64[2], *Mx64[2];
  float2 *C32;
  void *H[2];                   // float2 or __nv_bfloat162 (eta_z, eta_x)
  void *H32[2];                 // BF16 handles: FP32 mean messages after the ladder climbs
  float2 *sum32[2];
  double2 *sum64[2];
  float *sumE[2];
  const int32_t *sys_of_row;
  unsigned long long *sys_bmax;
  SysCtl *sysctl;               // per-system control state (used when Ctl::retire = 1)
};

struct Dense {
  int32_t nsys = 0;
  int64_t pairs = 0, nodes = 0;
  int32_t maxK = 0, maxN = 0;
  DenseView v{};
  DenseSys *sys = nullptr;      // device, largest systems first
  bool have64 = false, have32 = false;
  int rows_mean = 2, rows_full = 2;   // grid rows each warp loads ahead (1, 2 or 4)
  bool serial = false;                // serial schedule, class x^ then class z
};

int launch_dense_full64(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red);
int launch_dense_full32(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                        bool bf16);
int launch_dense_mean(const Dense &d, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                      bool bf16);
int launch_dense_residual(const Dense &d, cudaStream_t st, double *r_out, Ctl *ctl,
                          DevScalars *red, bool refine);
int launch_refine_update(int32_t n, cudaStream_t st, Buffers B, Ctl *ctl);
int launch_ait_record(int32_t n, cudaStream_t st, Buffers B, const Ctl *ctl);
int launch_aitken(int32_t n, cudaStream_t st, Ctl *ctl, double *out);
void prepare_dense_kernels(bool bf16);

// ---- nearest-neighbour operators on a box in the grid form (gabp_grid.cu) ----
// Nodes of a p0 x p1 x p2 box (p0 even; x fastest) are split into the two
// colour classes of the box, c = (x + y + z) mod 2, and each class is kept as
// a half grid: H = x / 2 + h0 (y + p1 z), h0 = p0 / 2; slot c Nh + H.  Per
// class and direction d (0/1: +-x, 2/3: +-y, 4/5: +-z) one plane of Nh
// entries, index (c D + d) Nh + H, holds A to that neighbour and the message
// coming from it.  The neighbour of (c, H) in direction d is (1 - c, H +
// off(d)) with off = s, s - 1, +-h0, +-h0 p1 and s = (c + y + z) mod 2: every
// access is a contiguous run, no index arrays.
struct GridView {
  int32_t ndim, D;                 // axes, directions (2 ndim)
  int32_t h0, p1, p2;              // half-row length, dims[1], dims[2]
  // n / h0 and n / p1 for n < 2^31 as (n * m) >> s (division by an invariant
  // integer through multiplication, Granlund and Montgomery 1994)
  uint64_t m_h0, m_p1;
  int32_t s_h0, s_p1;
  int64_t Nh;                      // nodes per class
  const double *a64, *diag64;      // [2 D Nh], [2 Nh]
  const float *a32, *diag32;
  int32_t pass;                    // -1: both classes (synchronous); c: colour pass over class c
  int32_t in_place, no_control, no_damp;
};

struct Grid {
  GridView v{};
  double *a64 = nullptr, *diag64 = nullptr;   // owned device arrays
  float *a32 = nullptr, *diag32 = nullptr;
  int32_t dims[3] = {1, 1, 1};
  bool colour = false, damp_last = false;     // red-black schedule; damping on class 1 only
  bool have64 = false, have32 = false;
  int64_t slots() const { return 2 * v.Nh; }
  int64_t planes() const { return 2 * static_cast<int64_t>(v.D) * v.Nh; }
  // the view of one launch: pass -1 (synchronous) or colour pass c
  GridView pass_view(int c) const {
    GridView w = v;
    w.pass = c;
    w.in_place = c >= 0;
    w.no_control = c == 0;
    w.no_damp = c == 0 && damp_last;
    return w;
  }
};

int launch_grid_full64(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red);
int launch_grid_full32(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                       bool bf16);
int launch_grid_mean(const GridView &v, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red,
                     bool bf16);
int launch_grid_residual(const GridView &v, cudaStream_t st, double *r_out, Ctl *ctl,
                         DevScalars *red, bool refine);
// Host: checks that the CSR (natural order) couples only nearest neighbours of
// the box `dims`, builds the planes and returns the slot -> natural row map.
gabp_status build_grid(Grid &G, int32_t ndim, const int32_t *dims, int64_t nnz,
                       const int64_t *row_ptr, const int32_t *col, const double *val,
                       cudaStream_t st, std::vector<int32_t> &perm, std::string *msg);
void free_grid(Grid &G);

// ---- whole FP64 solves of small systems in one cluster launch (gabp_resident.cu) ----
constexpr int kResidentMaxCluster = 16;   // CTAs of the cluster (16 needs the non-portable size)
constexpr int kResidentMaxSlots = 3072;   // incoming-message slots per CTA
constexpr int kResidentMaxRows = 896;     // rows per CTA
constexpr int kResidentMaxColours = 16;   // colour classes of the colour schedule

struct ResidentOut {
  int32_t status, sweeps, checks, pad;
  double residual, bnorm;
};

// Rows [row0[c], row0[c+1]) belong to CTA c.  For every slot s (incoming
// message of its row): dst[s] = (CTA << 24) | local slot of rev[s] in that
// CTA, colp[s] = (CTA << 16) | local row of col[s].
struct ResidentView {
  int32_t aitken;                // Delta^2 stride over the tentative means (0 = off)
  const int32_t *row0;
  const int32_t *rp;
  const double *a64, *diag64;
  const int32_t *dst, *colp;
  const double *b;
  double *x;
  int32_t smax, rmax;
  int32_t check_every, max_iter, rel;
  double tol, damping;
  ResidentOut *out;
  // colour schedule (ncol > 0): rows [cb[c], cb[c+1]) form class c; one pass
  // per class, in place; damp_last: only the last class's messages blend
  int32_t ncol, damp_last;
  int32_t cb[kResidentMaxColours + 1];
};

struct Resident {
  int C = 0;                     // cluster size in use (0 = not eligible)
  int smax = 0, rmax = 0;
  int32_t *row0 = nullptr, *dst = nullptr, *colp = nullptr;
  ResidentOut *out = nullptr;    // device
};

uint32_t resident_smem_bytes(int smax, int rmax);
cudaError_t launch_resident64(const ResidentView &v, int C, cudaStream_t st);

// ---- graph builder (gabp_build.cu) ----
gabp_status build_graph(Graph &g, int64_t n, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col, const double *val, const int64_t *rev,
                        const gabp_options &opt, cudaStream_t st, std::string *msg);
// Marks the graph as `nsys` independent systems with row offsets
// sys_row_off[0..nsys] (checks that no entry couples two systems).
gabp_status build_systems(Graph &g, int32_t nsys, const int64_t *sys_row_off,
                          const int64_t *row_ptr, const int32_t *col, cudaStream_t st,
                          std::string *msg);
// Section VII systems with Psi = 0 (gabp_pinv.cu): u = offdiag(R~) v on the CSR
// or the dense form, v = [x^; 0], [0; y - S x^] for flagged systems, x^ +=
// (scaled) x^ part of an augmented solution, per-system max |u| over the x^ rows.
int launch_csr_offdiag(const Graph &g, cudaStream_t st, const double *v, double *u);
// FP64 sweep by Algorithm 1, the naive form (gabp_naive.cu; option naive).
int launch_naive64(const Graph &g, cudaStream_t st, Buffers B, Ctl *ctl, DevScalars *red);
// Diagnostics (gabp_selfcheck.cu): a bounded wait that runs out, reported as the sweeps report it.
// Time limit of every bounded device wait (the sweeps' shared-memory
// staging).  A copy that lands takes microseconds, so the limit only ever
// ends a wait whose copy will not come, and it frees the SM within a tenth
// of a second.
constexpr unsigned long long kWaitLimitNs = 100ull * 1000 * 1000;   // 100 ms
int launch_wait_limit(cudaStream_t st, Ctl *ctl, DevScalars *red, unsigned long long limit_ns,
                      unsigned long long *ns);
int launch_dense_offdiag(const Dense &d, cudaStream_t st, const double *v, double *u);
int launch_pinv_embed(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                      const int32_t *K, const int64_t *x_off, const double *xhat, double *v);
int launch_pinv_rhs(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                    const int32_t *K, const int64_t *y_off, const double *y, const double *u,
                    const uint8_t *flag, double *rhs);
int launch_pinv_update(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                       const int32_t *K, const int64_t *x_off, const double *scale, const double *x_aug,
                       double *xhat);
int launch_pinv_sysmax(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row, const int64_t *aug_off,
                       const int32_t *K, const double *u, unsigned long long *smax);
int launch_lsq_rhs(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row,
                   const int64_t *aug_off, const int32_t *K, const int64_t *y_off, const double *y,
                   double *rhs);
int launch_lsq_extract(cudaStream_t st, int64_t n_aug, const int32_t *sys_of_row,
                       const int64_t *aug_off, const int32_t *K, const int64_t *x_off,
                       const double *x_aug, double *xhat);
void free_graph(Graph &g);
// Window form (gabp_window.cu): windows of about `target` slots.
gabp_status build_windows(const Graph &g, int32_t target, bool bf16, Win &W, cudaStream_t st,
                          std::string *msg);
void free_windows(Win &W);
int launch_mean_win(const Graph &g, const Win &W, cudaStream_t st, Buffers B, Ctl *ctl,
                    DevScalars *red, bool bf16);
cudaError_t set_row_tiles(Graph &g, int slots, int rows, int heavy_degree, cudaStream_t st);

}  // namespace gabp

struct gabp_s {
  gabp::Graph g;
  gabp_options opt;
  cudaStream_t stream = nullptr;
  std::string last_error;
  gabp_stats stats{};
  int64_t user_nnz = 0;            // nnz of the CSR given to gabp_create

  gabp::Buffers buf{};
  bool have64 = false, have32 = false;
  int m64_cur = 0;                 // buffer holding the messages left by gabp_run_rounds
  gabp::Ctl *ctl = nullptr;        // device control block
  gabp::Ctl *ctl_host = nullptr;   // pinned mirror
  gabp::DevScalars *red = nullptr; // device reductions
  double *bbuf = nullptr, *xbuf = nullptr;  // device staging for gabp_solve_host

  // one instantiated solve graph per control mode
  cudaGraphExec_t exec[gabp::CTL_MODES] = {};
  cudaGraph_t graph[gabp::CTL_MODES] = {};
  cudaGraphConditionalHandle cond[gabp::CTL_MODES][2] = {};   // (WHILE, SWITCH) per mode
  // least-squares batches (Section VII augmented systems)
  int32_t *lsq_K = nullptr;            // device: K_s
  int64_t *lsq_aug_off = nullptr;      // device: first augmented row of system s
  int64_t *lsq_y_off = nullptr;        // device: offset of y_s in the concatenated y
  int64_t *lsq_x_off = nullptr;        // device: offset of x^_s in the concatenated x^
  int64_t lsq_ny = 0, lsq_nx = 0;      // total lengths of y and x^
  double *lsq_rhs = nullptr, *lsq_x = nullptr;   // device: augmented rhs and solution
  // systems given psi_s = 0 (the Moore-Penrose solution): iterated around the augmented solve
  std::vector<uint8_t> lsq_pinv_host;  // per system: 1 = psi_s was 0
  uint8_t *lsq_pinv = nullptr;         // device copy
  double *lsq_inv_psi0 = nullptr;      // device: 1 / psi_0 of those systems, 0 for the others
  double *lsq_u = nullptr, *lsq_v = nullptr;     // device: augmented work vectors
  unsigned long long *lsq_gmax = nullptr;        // device: per-system max |S^T r| (bit patterns)
  unsigned long long *diag_ns = nullptr;         // device: duration of the wait-limit check
  int graph_K = 0;                     // K the CTL_MULTI graph was recorded for
  size_t capK = 0;                     // columns the multi buffers hold
  gabp::MultiCols cols{};              // device per-column arrays (capK each)
  gabp::Dense *dense = nullptr;        // Section VII batches in dense bipartite form
  gabp::Grid *grid = nullptr;          // nearest-neighbour operators on a box, grid form
  gabp_tuning tuning{};                // launch shapes (chosen by the autotuner or default)
  gabp::Resident res{};                // small FP64 systems: one cluster launch per solve
  gabp::Win win{};                     // window form of the mean sweep (nwin = 0: not in use)
  double *ring[3] = {};                // Aitken: the last three FP64 tentative means
  // colour schedule (Section III-C serial schedule by colour classes)
  int32_t *perm = nullptr;             // device: caller's row of renumbered row i
  double *bperm = nullptr, *xperm = nullptr;   // device: b and x in the renumbered order
  double *bKperm = nullptr, *xKperm = nullptr; // device: n x K right-hand sides and solutions, renumbered
  size_t capKperm = 0;
  cudaStream_t cap_stream = nullptr;   // private stream used to record graphs

  // profiling (gabp_options.profile): pairs of events around kernels
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
};
