/*
 * gabp_oracle.c -- plain FP64 CPU reference for Gaussian belief propagation
 * (GaBP) on Ax = b (Shental, Bickson, Siegel, Wolf, Dolev, "Gaussian Belief
 * Propagation for Solving Systems of Linear Equations: Theory and
 * Application").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct oracle
 * that the CUDA library is checked against.  Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes (Section III of the paper):
 *   - the synchronous ("parallel", two-buffer) schedule, Section III-C;
 *   - the broadcast form of Algorithm 2 (node totals P~_i, mu~_i, then each
 *     directed message obtained by subtracting the reverse message);
 *   - the naive form of Algorithm 1 (each message summed over N(i)\j
 *     directly), used only as a cross-check on tiny inputs;
 *   - the Jacobi reduction (the GaBP/Jacobi proposition of Section VI-C):
 *     precision messages held at zero and the message from j included;
 *   - the marginal means and precisions of Algorithm 1/2, step 4;
 *   - the serial schedule of Section III-C (oracle_gabp_serial): nodes
 *     visited one after another in a given order, each computing its
 *     totals from the latest messages and overwriting its outgoing ones.
 *
 * Storage: A is a full symmetric CSR matrix with the diagonal stored and the
 * column indices of each row strictly increasing.  The message on the
 * directed edge i -> j is kept at the CSR position of entry (i, j), i.e. in
 * the sender's row.  Diagonal positions hold zero.  The messages are the
 * paper's (P_ij, mu_ij) pair: a precision and a mean.
 *
 * Arithmetic follows the paper's notation literally:
 *   P_ii  = A_ii,           mu_ii = b_i / A_ii                 (Alg. 2 step 1)
 *   P~_i  = P_ii + sum_{k in N(i)} P_ki                       (Alg. 2 step 2)
 *   mu~_i = (P_ii mu_ii + sum_{k in N(i)} P_ki mu_ki) / P~_i   (Alg. 2 step 2)
 *   P_ij  = -A_ij^2 / (P~_i - P_ji)                            (Alg. 2 step 2)
 *   mu_ij = (P~_i mu~_i - P_ji mu_ji) / A_ij                   (Alg. 2 step 2)
 *   mu_i  = mu~_i,  P_i = P~_i  computed from the messages of the last round
 *                                                              (Alg. 2 step 4)
 * Sums run over the CSR row in column order; nodes are independent within a
 * round, so an OpenMP loop over nodes does not change any result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Return codes. */
#define OR_OK 0
#define OR_BAD_INPUT 1      /* not square-symmetric CSR, unsorted, missing diagonal */
#define OR_BREAKDOWN 2      /* P~_i - P_ji == 0 or non-finite */
#define OR_NOT_CONVERGED 3  /* stop rule not met within max_rounds */

/* Stop rules. */
#define OR_STOP_FIXED 0     /* run exactly max_rounds rounds */
#define OR_STOP_MSG 1       /* every message changed by less than tol (Section VIII) */
#define OR_STOP_RES_ABS 2   /* ||b - A x||_inf < tol */
#define OR_STOP_RES_REL 3   /* ||b - A x||_inf / ||b||_inf < tol */

/* Variants. */
#define OR_BROADCAST 0      /* Algorithm 2 */
#define OR_NAIVE 1          /* Algorithm 1 */
#define OR_JACOBI 2         /* Section VI-C: P := 0 and k ranges over all of N(i) */

/* Position of entry (r, c) in row r, or -1.  Binary search: columns are sorted. */
static int64_t find_entry(const int64_t *row_ptr, const int32_t *col, int64_t r, int32_t c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == c) return mid;
    if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Checks the CSR and fills:
 *   diag_pos[i] = position of A_ii,
 *   twin[e]     = position of entry (j, i) for e = (i, j), -1 on the diagonal.
 * Returns OR_OK or OR_BAD_INPUT. */
int oracle_check_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                     int64_t *diag_pos, int64_t *twin) {
  if (n < 1 || row_ptr[0] != 0) return OR_BAD_INPUT;
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return OR_BAD_INPUT;
    diag_pos[i] = -1;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (col[e] < 0 || col[e] >= n) return OR_BAD_INPUT;
      if (e > row_ptr[i] && col[e] <= col[e - 1]) return OR_BAD_INPUT;
      if (col[e] == i) diag_pos[i] = e;
    }
    if (diag_pos[i] < 0 || val[diag_pos[i]] == 0.0) return OR_BAD_INPUT;
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (col[e] == i) { twin[e] = -1; continue; }
      int64_t t = find_entry(row_ptr, col, col[e], (int32_t)i);
      if (t < 0 || val[t] != val[e]) return OR_BAD_INPUT;  /* A must be symmetric */
      twin[e] = t;
    }
  }
  return OR_OK;
}

/* r = b - A x, returns ||r||_inf (Section II: the solution satisfies Ax = b). */
double oracle_residual_inf(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                           const double *b, const double *x, double *r_out) {
  double worst = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double ax = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) ax += val[e] * x[col[e]];
    double r = b[i] - ax;
    if (r_out) r_out[i] = r;
    if (fabs(r) > worst || r != r) worst = (r != r) ? INFINITY : fabs(r);
  }
  return worst;
}

/*
 * One synchronous round: new messages (Pn, Mn) from old ones (Po, Mo).
 * Returns OR_OK or OR_BREAKDOWN.
 */
static int one_round(int variant, int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const double *val, const double *b, const int64_t *diag_pos,
                     const int64_t *twin, const double *Po, const double *Mo, double *Pn,
                     double *Mn, double gamma) {
  int status = OR_OK;
#pragma omp parallel for schedule(dynamic, 256) reduction(max : status)
  for (int64_t i = 0; i < n; ++i) {
    const double Pii = val[diag_pos[i]];   /* P_ii = A_ii */
    const double muii = b[i] / Pii;        /* mu_ii = b_i / A_ii */
    if (variant == OR_BROADCAST) {
      /* Broadcast sums over all of N(i): P~_i and mu~_i. */
      double Psum = Pii, hsum = Pii * muii;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (twin[e] < 0) continue;
        Psum += Po[twin[e]];                   /* P_ki, k = col[e] */
        hsum += Po[twin[e]] * Mo[twin[e]];     /* P_ki mu_ki */
      }
      const double Pt = Psum, mut = hsum / Psum;   /* P~_i, mu~_i */
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (twin[e] < 0) { Pn[e] = 0.0; Mn[e] = 0.0; continue; }
        const double Aij = val[e];
        const double Pji = Po[twin[e]], muji = Mo[twin[e]];
        const double denom = Pt - Pji;            /* P_{i\j} */
        if (denom == 0.0 || !isfinite(denom)) { status = OR_BREAKDOWN; }
        Pn[e] = -Aij * Aij / denom;
        Mn[e] = (Pt * mut - Pji * muji) / Aij;
        if (gamma > 0.0) {
          /* Damping (the heuristic Section VI-D cites for belief propagation):
           * the information P_ij mu_ij of the new message is blended with the
           * previous round's, the precision is not; a fixed point of the
           * damped rule is a fixed point of the undamped one. */
          const double eta = gamma * (Po[e] * Mo[e]) + (1.0 - gamma) * (Pn[e] * Mn[e]);
          Mn[e] = eta / Pn[e];
        }
      }
    } else if (variant == OR_NAIVE) {
      /* Algorithm 1: every message sums over N(i)\j directly. */
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (twin[e] < 0) { Pn[e] = 0.0; Mn[e] = 0.0; continue; }
        const int32_t j = col[e];
        double Pex = Pii, hex = Pii * muii;
        for (int64_t f = row_ptr[i]; f < row_ptr[i + 1]; ++f) {
          if (twin[f] < 0 || col[f] == j) continue;   /* k in N(i) \ j */
          Pex += Po[twin[f]];
          hex += Po[twin[f]] * Mo[twin[f]];
        }
        if (Pex == 0.0 || !isfinite(Pex)) { status = OR_BREAKDOWN; }
        Pn[e] = -val[e] * val[e] / Pex;
        Mn[e] = hex / val[e];
      }
    } else {
      /* Section VI-C (GaBP/Jacobi proposition): P_ij := 0 and the sum runs over all of N(i).  With the
       * precision zero the message is carried as P_ij mu_ij = -A_ij mu_{i\j}
       * (Mn holds that product), mu_{i\j} = A_ii^{-1}(b_i + sum_k P_ki mu_ki). */
      double hsum = b[i];
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (twin[e] < 0) continue;
        hsum += Mo[twin[e]];
      }
      const double mu_excl = hsum / Pii;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        Pn[e] = 0.0;
        Mn[e] = (twin[e] < 0) ? 0.0 : -val[e] * mu_excl;
      }
    }
  }
  return status;
}

/* Marginals from the current messages (Algorithm 2, step 4). */
static void infer(int variant, int64_t n, const int64_t *row_ptr, const double *val,
                  const double *b, const int64_t *diag_pos, const int64_t *twin,
                  const double *Pm, const double *Mm, double *x, double *Pi) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double Pii = val[diag_pos[i]];
    const double muii = b[i] / Pii;
    if (variant == OR_JACOBI) {
      double hsum = b[i];
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (twin[e] >= 0) hsum += Mm[twin[e]];
      x[i] = hsum / Pii;
      if (Pi) Pi[i] = Pii;
      continue;
    }
    double Psum = Pii, hsum = Pii * muii;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (twin[e] < 0) continue;
      Psum += Pm[twin[e]];
      hsum += Pm[twin[e]] * Mm[twin[e]];
    }
    x[i] = hsum / Psum;
    if (Pi) Pi[i] = Psum;
  }
}

/*
 * Run GaBP from zero messages (Algorithm 2 step 1: P_ki = mu_ki = 0).
 *
 *   variant    OR_BROADCAST | OR_NAIVE | OR_JACOBI
 *   stop       OR_STOP_FIXED | OR_STOP_MSG | OR_STOP_RES_ABS | OR_STOP_RES_REL
 *   max_rounds upper bound on rounds (exact count for OR_STOP_FIXED)
 *   tol        threshold of the stop rule
 * Outputs (caller-allocated; msgP/msgMu may be NULL):
 *   x[n]       tentative means after the last round (x = b_i/A_ii at round 0)
 *   Pi[n]      marginal precisions P_i after the last round (may be NULL)
 *   msgP[nnz], msgMu[nnz]   messages of the last round, i->j at entry (i,j)
 *   rounds     rounds executed
 *   gamma      damping in [0, 1) of the broadcast variant (0 = the plain rule)
 * Returns OR_OK, OR_BAD_INPUT, OR_BREAKDOWN or OR_NOT_CONVERGED.
 */
int oracle_gabp(int variant, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const double *val, const double *b, int stop, int max_rounds, double tol,
                double *x, double *Pi, double *msgP, double *msgMu, int *rounds, double gamma) {
  const int64_t nnz = row_ptr[n];
  int64_t *diag_pos = malloc(sizeof(int64_t) * (size_t)n);
  int64_t *twin = malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  double *P0 = calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  double *M0 = calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  double *P1 = calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  double *M1 = calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  double *xr = (stop == OR_STOP_RES_ABS || stop == OR_STOP_RES_REL) ? malloc(sizeof(double) * (size_t)n) : NULL;
  int status = oracle_check_csr(n, row_ptr, col, val, diag_pos, twin);
  *rounds = 0;
  if (status != OR_OK) goto done;

  double bnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) bnorm = fmax(bnorm, fabs(b[i]));

  /* Round 0: all messages zero, so x_i = mu_ii = b_i / A_ii. */
  infer(variant, n, row_ptr, val, b, diag_pos, twin, P0, M0, x, Pi);
  status = (stop == OR_STOP_FIXED && max_rounds == 0) ? OR_OK : OR_NOT_CONVERGED;
  for (int t = 1; t <= max_rounds; ++t) {
    int s = one_round(variant, n, row_ptr, col, val, b, diag_pos, twin, P0, M0, P1, M1, gamma);
    double *tp = P0; P0 = P1; P1 = tp;
    double *tm = M0; M0 = M1; M1 = tm;
    *rounds = t;
    if (s != OR_OK) { status = s; break; }
    infer(variant, n, row_ptr, val, b, diag_pos, twin, P0, M0, x, Pi);
    if (stop == OR_STOP_FIXED) { status = (t == max_rounds) ? OR_OK : OR_NOT_CONVERGED; continue; }
    if (stop == OR_STOP_MSG) {
      double change = 0.0;
      for (int64_t e = 0; e < nnz; ++e) {
        change = fmax(change, fabs(P0[e] - P1[e]));
        change = fmax(change, fabs(M0[e] - M1[e]));
      }
      if (change < tol) { status = OR_OK; break; }
    } else {
      double r = oracle_residual_inf(n, row_ptr, col, val, b, x, xr);
      if (stop == OR_STOP_RES_REL) r = (bnorm > 0.0) ? r / bnorm : r;
      if (r < tol) { status = OR_OK; break; }
    }
  }
  if (msgP) memcpy(msgP, P0, sizeof(double) * (size_t)nnz);
  if (msgMu) memcpy(msgMu, M0, sizeof(double) * (size_t)nnz);
done:
  free(diag_pos); free(twin); free(P0); free(M0); free(P1); free(M1); free(xr);
  return status;
}

/*
 * One round of the serial schedule (Section III-C): node i = order[k] for
 * k = 0..n-1 forms P~_i and mu~_i from the current incoming messages (the
 * ones of nodes visited earlier in this round are already new) and
 * overwrites its outgoing messages in place, by the rules of Algorithm 2.
 * `order` NULL means 0, 1, ..., n-1.  Returns OR_OK or OR_BREAKDOWN.
 */
static int serial_round(int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const double *val, const double *b, const int64_t *diag_pos,
                        const int64_t *twin, const int64_t *order, double *P, double *M,
                        double gamma, const unsigned char *damp_from) {
  int status = OR_OK;
  (void)col;
  for (int64_t k = 0; k < n; ++k) {
    const int64_t i = order ? order[k] : k;
    const double g = (damp_from && !damp_from[i]) ? 0.0 : gamma;
    const double Pii = val[diag_pos[i]];
    const double muii = b[i] / Pii;
    double Psum = Pii, hsum = Pii * muii;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (twin[e] < 0) continue;
      Psum += P[twin[e]];
      hsum += P[twin[e]] * M[twin[e]];
    }
    const double Pt = Psum, mut = hsum / Psum;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (twin[e] < 0) { P[e] = 0.0; M[e] = 0.0; continue; }
      const double Aij = val[e];
      const double Pji = P[twin[e]], muji = M[twin[e]];
      const double denom = Pt - Pji;
      if (denom == 0.0 || !isfinite(denom)) status = OR_BREAKDOWN;
      const double Pn = -Aij * Aij / denom;
      double Mn = (Pt * mut - Pji * muji) / Aij;
      if (g > 0.0) Mn = (g * (P[e] * M[e]) + (1.0 - g) * (Pn * Mn)) / Pn;
      P[e] = Pn;
      M[e] = Mn;
    }
  }
  return status;
}

/*
 * GaBP under the serial schedule from zero messages; arguments and outputs
 * as oracle_gabp (broadcast form only), plus the visiting order (NULL = the
 * natural order).  A round is one pass over all nodes.  damp_from (NULL =
 * every node) restricts the damping blend to the messages sent by the nodes
 * i with damp_from[i] != 0; the others send their undamped message.  The
 * fixed point does not depend on it.
 */
int oracle_gabp_serial(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       const double *b, const int64_t *order, int stop, int max_rounds, double tol,
                       double *x, double *Pi, double *msgP, double *msgMu, int *rounds,
                       double gamma, const unsigned char *damp_from) {
  const int64_t nnz = row_ptr[n];
  const size_t m = (size_t)(nnz > 0 ? nnz : 1);
  int64_t *diag_pos = malloc(sizeof(int64_t) * (size_t)n);
  int64_t *twin = malloc(sizeof(int64_t) * m);
  double *P = calloc(m, sizeof(double)), *M = calloc(m, sizeof(double));
  double *Pp = calloc(m, sizeof(double)), *Mp = calloc(m, sizeof(double));
  double *xr = malloc(sizeof(double) * (size_t)n);
  int status = oracle_check_csr(n, row_ptr, col, val, diag_pos, twin);
  *rounds = 0;
  if (status != OR_OK) goto done;
  double bnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) bnorm = fmax(bnorm, fabs(b[i]));
  infer(OR_BROADCAST, n, row_ptr, val, b, diag_pos, twin, P, M, x, Pi);
  status = (stop == OR_STOP_FIXED && max_rounds == 0) ? OR_OK : OR_NOT_CONVERGED;
  for (int t = 1; t <= max_rounds; ++t) {
    memcpy(Pp, P, sizeof(double) * m);
    memcpy(Mp, M, sizeof(double) * m);
    int s = serial_round(n, row_ptr, col, val, b, diag_pos, twin, order, P, M, gamma, damp_from);
    *rounds = t;
    if (s != OR_OK) { status = s; break; }
    infer(OR_BROADCAST, n, row_ptr, val, b, diag_pos, twin, P, M, x, Pi);
    if (stop == OR_STOP_FIXED) { status = (t == max_rounds) ? OR_OK : OR_NOT_CONVERGED; continue; }
    if (stop == OR_STOP_MSG) {
      double change = 0.0;
      for (int64_t e = 0; e < nnz; ++e) {
        change = fmax(change, fabs(P[e] - Pp[e]));
        change = fmax(change, fabs(M[e] - Mp[e]));
      }
      if (change < tol) { status = OR_OK; break; }
    } else {
      double r = oracle_residual_inf(n, row_ptr, col, val, b, x, xr);
      if (stop == OR_STOP_RES_REL) r = (bnorm > 0.0) ? r / bnorm : r;
      if (r < tol) { status = OR_OK; break; }
    }
  }
  if (msgP) memcpy(msgP, P, sizeof(double) * (size_t)nnz);
  if (msgMu) memcpy(msgMu, M, sizeof(double) * (size_t)nnz);
done:
  free(diag_pos); free(twin); free(P); free(M); free(Pp); free(Mp); free(xr);
  return status;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int k) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}
