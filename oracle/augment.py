"""Augmented symmetric system of Section VII (distributed pseudoinverse).

TEST INFRASTRUCTURE ONLY (part of the oracle package).

Section VII turns a rectangular system into a symmetric one of size K + N:

    R~ = [[ I_K ,  S^T ],      x~ = [x^ ; z],     y~ = [0_K ; y]
          [  S  ,  -Psi]]

with S of shape N x K.  Eliminating z from the two block rows gives
x^ = (S^T Psi^{-1} S + I)^{-1} S^T Psi^{-1} y; with Psi = sigma^2 I this is
(S^T S + sigma^2 I)^{-1} S^T y, the MMSE detector of Section VIII-B.

Reading of the garbled passage: the paper writes S in R^{k x n} while its
unknown x^ has k entries, and one line carries Psi where Psi^{-1} belongs;
the block form above is the one whose elimination yields the closed form the
paper states, so it is the one built here.
"""
from __future__ import annotations

import numpy as np


def augment_lsq(S, psi_diag, y):
    """Build (row_ptr, col, val, rhs) of R~ x~ = y~ from dense S (N x K).

    ``psi_diag`` is the diagonal of Psi (length N, or a scalar).  Exact zeros
    of S are not stored (they are not edges of the graph, Section II-B).
    Columns of every row are increasing.
    """
    S = np.asarray(S, dtype=np.float64)
    N, K = S.shape
    psi = np.broadcast_to(np.asarray(psi_diag, dtype=np.float64), (N,))
    y = np.asarray(y, dtype=np.float64)
    n = K + N
    rows, cols, vals = [], [], []
    # Block row 1: x^_k + sum_n S_nk z_n = 0.
    for k in range(K):
        rows.append(k); cols.append(k); vals.append(1.0)
        for m in range(N):
            if S[m, k] != 0.0:
                rows.append(k); cols.append(K + m); vals.append(S[m, k])
    # Block row 2: sum_k S_mk x^_k - psi_m z_m = y_m.
    for m in range(N):
        for k in range(K):
            if S[m, k] != 0.0:
                rows.append(K + m); cols.append(k); vals.append(S[m, k])
        rows.append(K + m); cols.append(K + m); vals.append(-psi[m])
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    vals = np.asarray(vals, dtype=np.float64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    rhs = np.concatenate([np.zeros(K), y])
    return row_ptr, cols, vals, rhs


def pinv_solution(S, y):
    """Section VII with Psi = 0: the Moore-Penrose solution x^ = S^+ y, which
    the section states as the zero-noise case of its closed form.  Written as
    the definition: the minimum-norm minimiser of ||y - S x||_2, through
    LAPACK (numpy.linalg.lstsq)."""
    S = np.asarray(S, dtype=np.float64)
    return np.linalg.lstsq(S, np.asarray(y, dtype=np.float64), rcond=None)[0]


def iterated_tikhonov(S, y, psi0, steps):
    """The route the library takes to Psi = 0, where GaBP cannot run on the
    augmented matrix (its z nodes would have a zero diagonal): from x^ = 0,
    ``steps`` times x^ <- x^ + (S^T S + psi0 I)^{-1} S^T (y - S x^), each step
    the Section VII closed form with Psi = psi0 I and right-hand side
    y - S x^.  Returns the iterates x^_1 .. x^_steps (rows)."""
    S = np.asarray(S, dtype=np.float64)
    K = S.shape[1]
    M = S.T @ S + psi0 * np.eye(K)
    x = np.zeros(K)
    out = []
    for _ in range(steps):
        x = x + np.linalg.solve(M, S.T @ (np.asarray(y, dtype=np.float64) - S @ x))
        out.append(x.copy())
    return np.array(out)
