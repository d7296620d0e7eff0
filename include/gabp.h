/*
 * gabp.h -- C ABI of the GB300 (sm_103a) Gaussian belief propagation solver.
 *
 * The library solves A x = b for a square symmetric A by synchronous
 * ("parallel", flooding) Gaussian belief propagation in the broadcast form of
 * Algorithm 2 of Shental, Bickson, Siegel, Wolf and Dolev, "Gaussian Belief
 * Propagation for Solving Systems of Linear Equations: Theory and
 * Application":
 *
 *   node totals     P~_i = A_ii + sum_{k in N(i)} P_ki
 *                   h~_i = b_i  + sum_{k in N(i)} P_ki mu_ki   (h~_i = P~_i mu~_i)
 *   edge messages   P_ij = -A_ij^2 / (P~_i - P_ji)
 *                   mu_ij = (h~_i - P_ji mu_ji) / A_ij
 *   solution        x_i = h~_i / P~_i                          (Alg. 2, steps 2 and 4)
 *
 * where every round reads only the previous round's messages (Section III-C,
 * parallel scheduling) and the graph has one node per row of A and one edge
 * per off-diagonal non-zero (Section II-B).  All messages start at zero
 * (Alg. 2, step 1).
 *
 * Conventions for every entry point:
 *   - Matrices are passed as a full symmetric CSR (diagonal included, column
 *     indices strictly increasing in each row), 0-based.  Explicit zeros
 *     off the diagonal are dropped (they are not edges).  The number of
 *     off-diagonal entries must be below 2^31 - 64.
 *   - Arrays named *_host are host memory; arrays named *_dev are device
 *     memory of the current CUDA device.  Device work is issued on the
 *     handle's stream (gabp_options.stream, NULL = the legacy default stream).
 *   - Functions return a gabp_status and never abort; gabp_last_error()
 *     gives a message for the last failure on a handle.
 *   - A handle runs one operation at a time (no concurrent calls on the same
 *     handle); different handles are independent.
 */
#ifndef GABP_H
#define GABP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gabp_s *gabp_handle;

typedef enum {
  GABP_OK = 0,
  GABP_ERR_INVALID_ARG = 1,    /* null pointer, bad size, malformed CSR */
  GABP_ERR_NOT_SYMMETRIC = 2,  /* pattern or values of A not symmetric, or rev inconsistent */
  GABP_ERR_ZERO_DIAG = 3,      /* a missing or zero diagonal entry (P_ii = A_ii must be != 0) */
  GABP_ERR_BREAKDOWN = 4,      /* some P~_i - P_ji was zero or not finite */
  GABP_ERR_DIVERGED = 5,       /* the residual became non-finite or grew by > 1e30 */
  GABP_ERR_NOT_CONVERGED = 6,  /* stop rule not met within max_iter sweeps */
  GABP_ERR_CUDA = 7,           /* a CUDA runtime call failed */
  GABP_ERR_OOM = 8,            /* device allocation failed */
  GABP_ERR_TIMEOUT = 9         /* a bounded device wait gave up */
} gabp_status;

typedef enum {
  GABP_PREC_FP64 = 0,        /* plain FP64 messages, every sweep updates P and mu */
  GABP_PREC_MIXED_FP32 = 1,  /* FP32 messages inside FP64 residual refinement */
  GABP_PREC_MIXED_BF16 = 2   /* as MIXED_FP32 with BF16 storage of the mean messages, climbing
                                a precision ladder: the first refinement step that fails to
                                shrink the residual by 10 % (BF16 messages hold about three
                                digits, which ill-conditioned systems can need more than)
                                switches the later inner solves to FP32 storage of the mean
                                messages (per system in a dense batch under per-system
                                control); the handle holds both buffers */
} gabp_precision;

typedef enum {
  GABP_RESIDUAL_ABS = 0,     /* stop when ||b - A x||_inf < tol */
  GABP_RESIDUAL_REL = 1      /* stop when ||b - A x||_inf / ||b||_inf < tol */
} gabp_residual_kind;

typedef struct {
  int32_t precision;      /* gabp_precision */
  int32_t residual_kind;  /* gabp_residual_kind */
  int32_t check_every;    /* sweeps between convergence checks; 0 = automatic */
  int32_t group_lanes;    /* lanes per row of the FP64 sweep (2..32, power of 2); 0 = automatic */
  int32_t autotune;       /* 1 = time the candidate launch shapes once at create and keep the
                             fastest (see gabp_get_tuning); dimensions pinned below stay pinned */
  int32_t profile;        /* 1 = bracket every kernel with CUDA events and report the times in gabp_stats */
  int32_t lsq_form;       /* gabp_create_lsq_batched: 0 = dense bipartite kernels when every
                             K_s <= 256 and N_s <= 1024, else the general CSR path;
                             1 = always the general CSR path */
  int32_t tile_slots;     /* CSR form: slots per row tile of the FP32 sweeps (32..1024); 0 = 1024 */
  double inner_tol;       /* mixed modes: relative accuracy asked of an inner FP32 solve (for one
                             system the last refinement step asks only what the stop rule still
                             needs); 0 = automatic: 1e-7, or 1e-6 for batched handles */
  void *stream;           /* cudaStream_t used by every call on the handle; NULL = legacy default */
  double damping;         /* gamma in [0, 1): each new message's information P_ij mu_ij becomes
                             gamma * previous + (1 - gamma) * new (precisions undamped); a fixed
                             point is unchanged.  0 = the plain rule of Alg. 2. */
  int32_t tile_rows;      /* CSR form: rows per row tile (1..256); 0 = 256 */
  int32_t heavy_degree;   /* CSR form: a tile holding a row of higher degree runs slot-parallel
                             instead of thread-per-row (>= 1); 0 = 64 */
  int32_t dense_rows;     /* dense Section VII form: grid rows each warp loads ahead in the FP32
                             sweeps (1, 2 or 4); 0 = 2 */
  int32_t small_form;     /* FP64 solves of systems that fit one thread-block cluster's shared
                             memory (<= 16 x 3584 off-diagonal entries, <= 16 x 1024 rows):
                             0 = the whole solve in one cluster launch, 1 = always a launch
                             per sweep */
  int32_t cluster_ctas;   /* CTAs of that cluster (2, 4, 8 or 16); 0 = automatic */
  int32_t aitken;         /* FP64 solves and gabp_run_rounds: Aitken's Delta^2 (Section IV-A,
                             convergence acceleration) on the tentative means of rounds
                             t - 2s, t - s and t with stride s = aitken (1..64); the stop rule
                             and the returned x use the extrapolated means.  On grid
                             (bipartite) graphs the synchronous schedule's error flips sign
                             every round: s = 2 accelerates there, s = 1 does not.
                             Mixed solves with one right-hand side on CSR and grid handles
                             (any aitken > 0): each inner solve's means d are recorded every
                             2^j sweeps (j = 6..12) and the refinement step uses d
                             extrapolated by Delta^2 from the widest spacing s with 6 s <=
                             the inner solve's sweeps (no extrapolation after an
                             extrapolated step that failed to shrink the residual by 10 %);
                             the next inner solve then restarts GaBP from the extrapolated
                             solution (Steffensen's iteration, Section IV-A, in residual
                             form).  It holds 21 FP32 values per node; on CSR handles one
                             small extra launch follows every mean sweep.
                             0 = off (dense Section VII handles and multi right-hand-side
                             solves: always off) */
  int32_t schedule;       /* 0 = synchronous (the parallel schedule of Section III-C, two message
                             buffers); 1 = colour-serial: rows are coloured greedily in the
                             caller's order (no two neighbours share a colour) and every sweep
                             updates the colour classes one after another in place, each using
                             the latest messages -- the serial schedule of Section III-C with
                             nodes visited by colour, which needs about half the sweeps on grid
                             and other two-colourable graphs.  Small FP64 systems then take the
                             per-sweep path.  gabp_create_batched: not available.
                             gabp_create_lsq_batched: dense form only (lsq_form 0 and every
                             system within its limits); the classes are all x^ nodes, then all
                             z nodes, so a sweep still streams each grid once. */
  int32_t damp_scope;     /* which messages `damping` blends: 0 = every information message;
                             1 = only those the last colour class sends (schedule = 1 only;
                             in the dense Section VII form: the z -> x^ messages, so the
                             x^ -> z ones are never stored).  The fixed point is the same. */
  int32_t pull_lanes;     /* CSR form, FP32 full sweeps (mixed modes): -1 = scatter form (each
                             row sends its messages to the receivers' slots); 2, 4, 8, 16 or 32 =
                             in-place form with that many lanes per row (each slot recomputes the
                             reverse message of the previous round from its own row's totals two
                             rounds back and updates its incoming message; the only random
                             access is a gather of the sender's node totals); 0 = automatic: the
                             autotuner times both forms, else the scatter form.  The in-place
                             form needs the synchronous schedule and no damping. */
  double pinv_shift;      /* gabp_create_lsq_batched, systems given psi_s = 0: their augmented
                             matrix is built with Psi_0 = pinv_shift * (mean squared column norm
                             of S_s) I and the solve iterates to S_s^+ y_s (see there); larger
                             values make each augmented solve easier for GaBP and the iteration
                             slower.  0 = 0.1 */
  int32_t naive;          /* 1 = FP64 sweeps by Algorithm 1, the naive form: every cavity sum
                             P_{i\j} = A_ii + sum_{k != j} P_ki (and its information part) is
                             added up over the other incoming messages directly, O(deg^2) per
                             row, instead of node total minus reverse message (Algorithm 2).
                             The same round without that cancellation, for cross-checks on
                             small systems.  CSR handles, FP64, schedule 0, no damping;
                             0 = Algorithm 2 */
  int32_t mean_window;    /* CSR form, mean-only sweeps (mixed modes): -1 = tile form (each row
                             sends its messages to the receivers' slots, a scattered store per
                             edge); W in 256..65536 = window form with windows of about W
                             slots: the rows are cut into windows of consecutive rows, each
                             window's outgoing messages are kept sorted by destination, and a
                             sweep moves them as contiguous runs through shared memory (no
                             scattered access).  0 = automatic: with autotune the tuner times
                             both forms and several window sizes, else the tile form.  The
                             window form needs the synchronous schedule. */
  int32_t batch_control;  /* gabp_create_lsq_batched in the dense form, mixed and FP64 solves:
                             0 = per system: each system freezes its precisions, ends its
                             inner solves (asking only the accuracy its own stop rule still
                             needs) and takes its refinement step on its own numbers, inside
                             the sweep that ends the inner solve, and drops out of the sweeps
                             once it meets the stop rule -- so a system takes the same sweeps,
                             and its x^ the same bits, in a batch as when it is solved alone;
                             1 = one controller for the whole batch (its maxima decide the
                             freeze and the end of each inner solve, and every system sweeps
                             until the last one is done). */
} gabp_options;

/* Statistics of the last solve on a handle. */
typedef struct {
  int32_t sweeps_total;     /* all message sweeps (full and mean-only) */
  int32_t sweeps_full;      /* sweeps that updated precisions and means */
  int32_t sweeps_mean;      /* mean-only sweeps with frozen precisions */
  int32_t outer_steps;      /* FP64 refinement steps (mixed modes; 1 for FP64) */
  int32_t residual_checks;  /* FP64 residual evaluations */
  int32_t status;           /* gabp_status of the solve */
  double residual;          /* final ||b - A x||_inf (absolute) */
  double rhs_norm;          /* ||b||_inf */
  int64_t n;                /* unknowns */
  int64_t edges;            /* directed edges = off-diagonal non-zeros */
  int64_t kernel_launches;  /* kernels launched by the solve */
  /* With gabp_options.profile: summed device time (ms) of the kernels of
   * each kind, measured with CUDA events on the handle's stream. */
  double ms_full;           /* full sweeps (FP64 or FP32) */
  double ms_mean;           /* mean-only sweeps */
  double ms_residual;       /* FP64 residual evaluations */
  double ms_other;          /* norms, scaling, refinement updates */
  int64_t positions_swept;  /* dense Section VII batches: grid positions (edge pairs) that the
                               solve's sweeps processed, summed over the sweeps (with per-system
                               control a system that is done adds none, and the sweep that ends
                               a system's inner solve skips its grid pass); 0 for the other
                               forms */
  int32_t sweeps_wide;      /* MIXED_BF16: mean-only sweeps that stored FP32 mean messages
                               after the precision ladder climbed (dense batch under
                               per-system control: sweeps in which some system had climbed) */
  int32_t aitken_steps;     /* mixed solves with aitken > 0: refinement steps that used
                               the extrapolated means */
} gabp_stats;

/* Fills *opt with the defaults: FP64, relative residual, automatic check
 * interval and launch shape, no autotuning, automatic inner_tol, NULL stream. */
void gabp_default_options(gabp_options *opt);

/*
 * Builds a solver for the n x n symmetric matrix given as a full CSR in host
 * memory: row_ptr_host[n+1], col_host[nnz], val_host[nnz] (Section II-B: one
 * graph node per row, one edge per off-diagonal non-zero).
 *
 * rev_host (optional, may be NULL): the reverse-edge permutation over the
 * CSR entries, rev[e] = position of entry (j, i) for e = (i, j) (rev of a
 * diagonal entry is itself).  It is validated when given and computed when
 * NULL.
 *
 * Ownership: the library copies what it needs into device memory it owns;
 * the caller may free the inputs on return.  opt may be NULL (defaults).
 * Errors: GABP_ERR_INVALID_ARG (n < 1, malformed CSR, unsorted columns,
 * too many edges), GABP_ERR_NOT_SYMMETRIC (|A_ij - A_ji| > 1e-14 max|A_ij|,
 * asymmetric pattern or a wrong rev), GABP_ERR_ZERO_DIAG, GABP_ERR_OOM,
 * GABP_ERR_CUDA.  On error *out is NULL.
 */
gabp_status gabp_create(gabp_handle *out, int64_t n, int64_t nnz, const int64_t *row_ptr_host,
                        const int32_t *col_host, const double *val_host, const int64_t *rev_host,
                        const gabp_options *opt);

/* Releases the handle and all device memory it owns.  NULL is accepted. */
gabp_status gabp_destroy(gabp_handle h);

/* Replaces the stream used by later calls on the handle. */
gabp_status gabp_set_stream(gabp_handle h, void *stream);

/*
 * Solves A x = b (b_dev[n], x_dev[n], FP64 device arrays, caller-owned) with
 * the handle's precision mode, starting from zero messages (Alg. 2, step 1;
 * the initial content of x_dev is ignored).  Stops when the FP64 residual
 * ||b - A x||_inf (absolute or relative to ||b||_inf, per residual_kind)
 * falls below tol, or after max_iter sweeps.
 *
 * *iters (may be NULL) receives the number of message sweeps executed.
 * The call returns when x_dev holds the result (the stream is synchronised).
 * Errors: GABP_ERR_NOT_CONVERGED (x_dev holds the last iterate),
 * GABP_ERR_BREAKDOWN (a zero or non-finite P~_i - P_ji), GABP_ERR_DIVERGED,
 * GABP_ERR_INVALID_ARG, GABP_ERR_CUDA.
 */
gabp_status gabp_solve(gabp_handle h, const double *b_dev, double *x_dev, double tol,
                       int32_t max_iter, int32_t *iters);

/* As gabp_solve with b and x in host memory: the library copies b to the
 * device, solves, and copies x back, all on the handle's stream. */
gabp_status gabp_solve_host(gabp_handle h, const double *b_host, double *x_host, double tol,
                            int32_t max_iter, int32_t *iters);

/*
 * Solves A X = B for nrhs right-hand sides at once.  B_dev and X_dev are
 * n x nrhs FP64 device arrays, row-major ("column-interleaved": element
 * (i, k) at i * nrhs + k).
 *
 * Mixed modes (nrhs <= 256): the precision messages do not depend on b
 * (Alg. 2: P_ij involves only A and other precisions), so they are iterated
 * once (FP32 sweeps on a zero right-hand side) and frozen; then the FP32
 * mean messages of all columns advance together, stored column-interleaved
 * (message k of slot s at s * nrhs + k), inside FP64 refinement with a
 * residual norm and scale per column.  Stops when every column meets the
 * residual rule (absolute, or relative to that column's ||b_k||_inf).  The
 * mean messages are FP32 in both mixed modes.
 * FP64 mode: the columns are solved one after another with gabp_solve's path.
 *
 * *iters receives the sweeps executed (precision sweeps plus K-column mean
 * sweeps in the mixed modes).  Errors as gabp_solve; GABP_ERR_INVALID_ARG
 * for nrhs < 1, or nrhs > 256 in a mixed mode.
 */
gabp_status gabp_solve_multi(gabp_handle h, const double *B_dev, double *X_dev, int32_t nrhs,
                             double tol, int32_t max_iter, int32_t *iters);

/*
 * Batched independent systems.  The CSR (host arrays, as for gabp_create)
 * holds nsys systems along the diagonal: rows sys_row_off_host[s] ..
 * sys_row_off_host[s+1]-1 belong to system s, and no entry may couple two
 * systems (GABP_ERR_INVALID_ARG otherwise).  GaBP on a block-diagonal matrix
 * is GaBP on every block, so one sweep kernel advances all systems at once
 * (one persistent launch per sweep, one CUDA graph per solve).
 * gabp_solve on such a handle applies the stop rule to every system: with
 * the relative rule, each system's ||b_s - A_s x_s||_inf must fall below
 * tol ||b_s||_inf.  Errors as gabp_create.
 */
gabp_status gabp_create_batched(gabp_handle *out, int32_t nsys, const int64_t *sys_row_off_host,
                                int64_t nnz, const int64_t *row_ptr_host, const int32_t *col_host,
                                const double *val_host, const gabp_options *opt);

/*
 * Batched least squares through the symmetric augmented system of Section
 * VII: for every s, with S_s of shape N_s x K_s (row-major, the matrices
 * concatenated in S_host) and Psi_s = psi_s I,
 *     [ I_K   S_s^T  ] [x^_s]   [ 0  ]
 *     [ S_s  -Psi_s  ] [z_s ] = [ y_s],
 * whose first K_s unknowns are x^_s = (S_s^T S_s + psi_s I)^{-1} S_s^T y_s
 * (the MMSE detector of Section VIII-B when psi_s is the noise variance).
 * The handle is a batched handle over the augmented systems (3 K_s rows
 * when N_s = 2 K_s).  Requires K_s, N_s >= 1 and psi_s >= 0.
 *
 * psi_s = 0 asks for the Moore-Penrose solution x^_s = S_s^+ y_s, the case
 * Section VII singles out.  GaBP cannot run on the augmented matrix with a
 * zero Psi (every z node has a zero diagonal), so such a system is built with
 * Psi_0 = pinv_shift * (mean squared column norm of S_s) I (option
 * pinv_shift, 0 = 0.1), and gabp_solve_lsq_batched iterates
 *     x^ <- x^ + (S^T S + Psi_0)^{-1} S^T (y - S x^),
 * each step one augmented solve with right-hand side [0; y - S x^], until
 * the normal equations hold: ||S_s^T (y_s - S_s x^_s)||_inf <=
 * tol ||S_s^T y_s||_inf.  For S_s of full column rank that is S_s^+ y_s; each
 * step multiplies the error along a singular direction of S_s (singular
 * value sigma) by psi_0 / (sigma^2 + psi_0).
 */
gabp_status gabp_create_lsq_batched(gabp_handle *out, int32_t nsys, const int32_t *K_host,
                                    const int32_t *N_host, const double *S_host,
                                    const double *psi_host, const gabp_options *opt);

/*
 * Solves every augmented system of a gabp_create_lsq_batched handle:
 * y_dev = the y_s concatenated (sum N_s FP64 device values), xhat_dev = the
 * x^_s concatenated (sum K_s values).  The stop rule (per system) is applied
 * to the augmented systems.  *iters as gabp_solve.
 * If some system was given psi_s = 0, the solve runs the iteration described
 * at gabp_create_lsq_batched; tol then also bounds the normal-equation
 * residual of those systems.  *iters and the statistics sum the sweeps of
 * all augmented solves, outer_steps counts them, and residual / rhs_norm
 * are ||S^T (y - S x^)||_inf / ||S^T y||_inf of the system furthest from
 * its rule.  GABP_ERR_NOT_CONVERGED after max_iter sweeps or 500 augmented
 * solves; the status of a failed augmented solve otherwise.
 */
gabp_status gabp_solve_lsq_batched(gabp_handle h, const double *y_dev, double *xhat_dev, double tol,
                                   int32_t max_iter, int32_t *iters);

/*
 * A handle for a matrix that couples only nearest neighbours of a box (the
 * Laplacians of Section IX and any symmetric operator with the same
 * pattern), kept in the grid form: no index arrays.  The nodes of the
 * dims[0] x dims[1] x dims[2] box (ndim = 1, 2 or 3 entries of dims; dims[0]
 * even and >= 2; x fastest) are split into the two colour classes of the
 * box, (x + y + z) mod 2, and every message sits in a per-direction plane of
 * its class, so a sweep reads and writes contiguous runs.
 *
 * Arguments: the CSR of A in host memory, rows in the box's natural order
 * (i = x + dims[0] (y + dims[1] z)), the diagonal stored in every row and
 * column indices strictly increasing; every off-diagonal entry must join
 * nearest neighbours inside the box (a missing or zero entry is an absent
 * edge).  The arrays are copied; the caller keeps ownership.  Options as
 * gabp_create: schedule 0 runs the synchronous sweep of Alg. 2 (one launch
 * per sweep), schedule 1 the serial schedule of Section III-C with the two
 * classes in turn (red-black, one in-place launch per class), damp_scope 1
 * limits damping to the second class.  b and x of gabp_solve stay in the
 * natural order.  gabp_solve, gabp_solve_host, gabp_solve_multi (columns in
 * turn) and gabp_run_rounds work as on a gabp_create handle;
 * gabp_get_messages returns GABP_ERR_INVALID_ARG.
 *
 * Errors: GABP_ERR_INVALID_ARG (bad dims, an entry that is not a nearest
 * neighbour, malformed CSR), GABP_ERR_NOT_SYMMETRIC, GABP_ERR_ZERO_DIAG,
 * GABP_ERR_OOM, GABP_ERR_CUDA; the reason is in gabp_last_error(NULL).
 */
gabp_status gabp_create_grid(gabp_handle *out, int32_t ndim, const int32_t *dims, int64_t nnz,
                             const int64_t *row_ptr_host, const int32_t *col_host,
                             const double *val_host, const gabp_options *opt);

/* Statistics of the last solve on the handle. */
gabp_status gabp_get_stats(gabp_handle h, gabp_stats *stats);

/*
 * Message sweeps each system of a batched handle took part in during its
 * last solve, in the caller's order: sweeps_host[s] for s < nsys, nsys = the
 * handle's number of systems (host memory, caller-owned).  With per-system
 * control (gabp_options.batch_control 0 on a dense Section VII batch) these
 * are the system's own sweeps; otherwise every system took part in every
 * sweep and each entry is the solve's sweeps_total.  After a psi_s = 0
 * (Moore-Penrose) solve they are those of its last augmented solve.
 * GABP_ERR_INVALID_ARG for a handle that is not batched or a wrong nsys.
 */
gabp_status gabp_get_system_sweeps(gabp_handle h, int32_t *sweeps_host, int32_t nsys);

/*
 * Turns per-kernel timing on (1) or off (0) for the handle's later solves,
 * like gabp_options.profile at create.  With timing on, a solve is driven
 * from the host with CUDA events around every kernel (the same kernels and
 * launch shapes as the graph driver) and gabp_stats reports the times.
 */
gabp_status gabp_set_profile(gabp_handle h, int32_t on);

/*
 * Launch shapes of a handle.  (The paper has no counterpart: these choices
 * belong to the GPU mapping of the Alg. 2 sweep.)  With
 * gabp_options.autotune = 1, gabp_create* times the candidates on the
 * handle's own matrix, with zero messages, and keeps the fastest:
 *   CSR form, mixed precisions: the degree above which a row tile runs
 *     slot-parallel ("heavy") instead of thread-per-row (16, 32, 64, 128 or
 *     never), then the tile shape (slots x rows: 1024 x 256, 512 x 256,
 *     512 x 128, 256 x 64), scored by 4 mean sweeps + 1 full sweep;
 *   CSR form, mixed precisions, synchronous schedule: the form of the FP32
 *     full sweep (scatter, or in place with 2 .. 32 lanes per row), then the
 *     form of the mean sweep (tiles, or windows of about E / (SMs x m)
 *     slots, m = 3, 4, 6, 8), scored by mean sweeps alone;
 *   CSR form, FP64: lanes per row of the FP64 sweep (2 .. 32);
 *   dense Section VII form, mixed precisions: grid rows each warp loads
 *     ahead (1, 2 or 4) in the mean sweep and in the full sweep.
 * Without autotune the defaults are reported (tuned = 0).
 */
typedef struct {
  int32_t tuned;            /* 1 = chosen by timing at create */
  int32_t candidates;       /* launch shapes timed */
  int32_t tile_slots;       /* CSR form: slots per row tile (FP32 sweeps, residual) */
  int32_t tile_rows;        /* CSR form: rows per row tile */
  int32_t heavy_degree;     /* CSR form: tiles with a row above this degree run slot-parallel */
  int32_t group_lanes;      /* CSR form: lanes per row of the FP64 sweep */
  int32_t dense_rows_mean;  /* dense form: grid rows loaded ahead per warp, mean sweep */
  int32_t dense_rows_full;  /* dense form: the same, full sweeps */
  int32_t cluster_ctas;     /* small FP64 systems: CTAs of the resident cluster (0 = not used) */
  int32_t pull_lanes;       /* CSR form: lanes per row of the in-place FP32 full sweep (0 = scatter form) */
  int32_t mean_window;      /* CSR form: target slots per window of the window-form mean sweep
                               (0 = tile form) */
  int32_t windows;          /* CSR form: windows of the window form (0 = tile form) */
  double tune_ms;           /* host time spent tuning */
  double reserved[3];
} gabp_tuning;

gabp_status gabp_get_tuning(gabp_handle h, gabp_tuning *tuning);

/*
 * Diagnostics, no counterpart in the paper.  Every wait inside the library's
 * kernels (the shared-memory staging of the sweeps) is bounded in time:
 * 100 ms of the GPU's global timer after its first unsatisfied poll it gives
 * up, the launch raises a flag, and the solve ends with GABP_ERR_TIMEOUT
 * instead of holding the device.  This call exercises that path on h's
 * device and stream: one warp runs the sweeps' own bounded wait on a barrier
 * that nothing ever completes (no copy is issued), for `limit_us`
 * microseconds (1..100000; 0 = the library's limit of 100000), then reports
 * through the same controller.  Returns GABP_ERR_TIMEOUT when the path works
 * (the handle stays usable); GABP_ERR_INVALID_ARG for limit_us outside
 * 0..100000.  *seconds_waited (may be NULL) receives the measured duration
 * of the wait.  On first use it allocates what a first solve would (the
 * control block, the reductions, an n-entry FP64 scratch vector) and 8 bytes
 * more.
 */
gabp_status gabp_check_wait_limit(gabp_handle h, int32_t limit_us, double *seconds_waited);

/*
 * Instrumentation for parity tests.  Runs exactly `rounds` synchronous FP64
 * rounds of Alg. 2 from zero messages on b_dev and writes the tentative
 * means after the last round to x_dev (rounds = 0 gives x_i = b_i / A_ii).
 * The messages of the last round stay in the handle for gabp_get_messages.
 */
gabp_status gabp_run_rounds(gabp_handle h, const double *b_dev, int32_t rounds, double *x_dev);

/*
 * Copies the messages left by gabp_run_rounds into host arrays of length
 * nnz laid out like the CSR given to gabp_create: the message from i to j
 * (precision P_ij and mean mu_ij) at the position of entry (i, j); diagonal
 * positions receive 0.
 */
gabp_status gabp_get_messages(gabp_handle h, double *P_host, double *mu_host);

/*
 * gabp_run_rounds without any device allocation.  (The paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory when they call -- applications that reserve all device memory up
 * front, where a late cudaMalloc fails or is forbidden; code running inside
 * an allocator or memory-pool callback, which cannot re-enter the
 * allocator; loops that must never pay the device-wide synchronisation of
 * cudaMalloc/cudaFree.)
 *
 * Runs exactly `rounds` synchronous FP64 rounds of Alg. 2 from zero messages
 * on a matrix the caller already holds in device memory and writes the
 * tentative means after the last round to x_dev, like gabp_run_rounds:
 *   row_ptr_dev[n+1], col_dev[nnz], val_dev[nnz]: full symmetric CSR with
 *     the diagonal stored (columns in any order within a row; the caller
 *     guarantees symmetry, non-zero diagonal and in-range indices -- nothing
 *     is validated on the device);
 *   rev_dev[nnz]: reverse-entry permutation, rev[e] = position of (j, i) for
 *     e = (i, j) (rev of a diagonal entry is itself);
 *   b_dev[n] in, x_dev[n] out; all FP64 / int device arrays owned by the
 *   caller.
 * Stream: work is issued on `stream` (cudaStream_t); NULL means the calling
 * thread's per-thread default stream (cudaStreamPerThread), not the legacy
 * default stream, which would synchronise implicitly with every blocking
 * stream of the process.  The call ends by reading a status word into host
 * memory and synchronising the stream, so the stream must not be capturing:
 * a capturing stream is rejected with GABP_ERR_INVALID_ARG before any work
 * is issued.
 * Working space: one fixed array of 2 x 2^18 message pairs (8 MiB) in the
 * library's static device memory, present on every GPU that loads the
 * library until the process exits.  nnz above 2^18 = 262144 is rejected
 * with GABP_ERR_INVALID_ARG (message via gabp_last_error(NULL)).  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 * The array's device address is looked up on every call (a lookup
 * allocates nothing); the first call on a device may load the library's
 * module there, so make it before any stream capture on that device.  After
 * a device reset the next call finds the array at its new address.  All
 * calls share the array and it keeps the last call's contents (nothing in
 * it needs to start at zero except a status word the call clears itself);
 * calls that overlap on the GPU -- on different streams or host threads --
 * race on it.
 * Errors: GABP_ERR_INVALID_ARG, GABP_ERR_BREAKDOWN, GABP_ERR_CUDA.
 */
gabp_status gabp_run_rounds_noalloc(int64_t n, int64_t nnz, const int64_t *row_ptr_dev,
                                    const int32_t *col_dev, const double *val_dev,
                                    const int64_t *rev_dev, const double *b_dev, int32_t rounds,
                                    double *x_dev, void *stream);

/* Message of the last failure on the handle (never NULL; "" when none).
 * With h == NULL: the last failure of gabp_create* or of an entry point
 * without a handle on this thread. */
const char *gabp_last_error(gabp_handle h);

/* Name of a status code. */
const char *gabp_status_string(gabp_status s);

/* Library version string. */
const char *gabp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GABP_H */
