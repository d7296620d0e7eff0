"""Seeded synthetic inputs for the GaBP solver and its oracle.

This module holds no GaBP arithmetic: it only builds matrices and right-hand
sides (numpy PCG64 generators, explicit seeds), so that the CUDA library and
the CPU oracle can be fed the very same inputs.  Every matrix is returned as a
full symmetric CSR (diagonal included, columns strictly increasing per row).

Workloads (each mirrors a structure the paper uses or a detection system it
describes):
  * ``poisson2d(p)``  -- 5-point Laplacian, Dirichlet boundary, natural
    ordering, diagonal 4 and off-diagonals -1 (Section IX, 2-D Poisson).
  * ``poisson3d(p)``  -- the 7-point analogue (diagonal 6).
  * ``er_sdd(n, d, dom)`` -- Erdos-Renyi pattern of average degree d,
    off-diagonals N(0,1), A_ii = dom * sum_j |A_ij| (strict diagonal
    dominance, the sufficient condition of Section IV).
  * ``random_tree(n)`` -- a random recursive tree (acyclic graph, Section IV:
    exact means and precisions).
  * ``detection_batch(...)`` -- CDMA linear-detection systems
    A = S^T S + sigma^2 I, b = S^T y (Section VIII-B, MMSE detector).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Full symmetric matrix in CSR form (int64 row_ptr, int32 col, f64 val)."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def n_directed_edges(self) -> int:
        """Off-diagonal entries = directed edges of the GaBP graph."""
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        return int(np.count_nonzero(rows != self.col))

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        A[rows, self.col] = self.val
        return A

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        return np.bincount(rows, self.val * x[self.col], minlength=self.n)


def csr_from_coo(n: int, rows, cols, vals) -> CSR:
    """CSR from coordinate triplets without duplicates."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), vals)


def csr_from_dense(A: np.ndarray) -> CSR:
    A = np.asarray(A, dtype=np.float64)
    r, c = np.nonzero(A)
    return csr_from_coo(A.shape[0], r, c, A[r, c])


def reverse_index(m: CSR) -> np.ndarray:
    """rev[e] = position of entry (j, i) for the entry e = (i, j); rev of a
    diagonal entry is itself.  This is the reverse-edge permutation the
    library's ``gabp_create`` accepts (it can also compute it)."""
    rows = np.repeat(np.arange(m.n, dtype=np.int64), np.diff(m.row_ptr))
    key = rows * m.n + m.col
    rkey = m.col.astype(np.int64) * m.n + rows
    # keys are already sorted (CSR order), so a search finds the twin.
    pos = np.searchsorted(key, rkey)
    if np.any(pos >= key.size) or np.any(key[np.minimum(pos, key.size - 1)] != rkey):
        raise ValueError("pattern is not symmetric")
    return pos.astype(np.int64)


def poisson2d(p: int) -> CSR:
    """5-point Laplacian on a p x p interior grid, natural (lexicographic) order."""
    n = p * p
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % p, idx // p
    rows, cols, vals = [idx], [idx], [np.full(n, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (ix + dx >= 0) & (ix + dx < p) & (iy + dy >= 0) & (iy + dy < p)
        rows.append(idx[ok]); cols.append(idx[ok] + dx + dy * p); vals.append(np.full(ok.sum(), -1.0))
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson3d(p: int) -> CSR:
    """7-point Laplacian on a p^3 interior grid, lexicographic order.

    Built directly in CSR order (neighbour offsets -p^2, -p, -1, 0, +1, +p,
    +p^2 are increasing), so p = 256 (n = 16.8M) needs no sort."""
    n = p ** 3
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % p, (idx // p) % p, idx // (p * p)
    offs = [(-p * p, iz > 0), (-p, iy > 0), (-1, ix > 0), (0, None),
            (1, ix < p - 1), (p, iy < p - 1), (p * p, iz < p - 1)]
    mask = np.ones((n, 7), dtype=bool)
    colm = np.empty((n, 7), dtype=np.int64)
    valm = np.full((n, 7), -1.0)
    for k, (o, ok) in enumerate(offs):
        colm[:, k] = idx + o
        if ok is not None:
            mask[:, k] = ok
    valm[:, 3] = 6.0
    deg = mask.sum(1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = colm[mask].astype(np.int32)
    val = valm[mask]
    return CSR(n, row_ptr, col, val)


def er_sdd(n: int, avg_degree: float, dominance: float, seed: int) -> CSR:
    """Symmetric Erdos-Renyi pattern with off-diagonals N(0,1) and
    A_ii = dominance * sum_j |A_ij| (A_ii = 1 for a row with no neighbour).

    Sampling: n*avg_degree/2 ordered pairs (i, j) uniform over [0, n)^2 and
    one N(0,1) value per pair; self pairs are dropped, each unordered pair is
    kept at its first occurrence, then mirrored."""
    rng = np.random.default_rng(seed)
    m = int(round(n * avg_degree / 2))
    i = rng.integers(0, n, m, dtype=np.int64)
    j = rng.integers(0, n, m, dtype=np.int64)
    v = rng.standard_normal(m)
    keep = i != j
    i, j, v = i[keep], j[keep], v[keep]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    _, first = np.unique(lo * n + hi, return_index=True)
    lo, hi, v = lo[first], hi[first], v[first]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    vals = np.concatenate([v, v])
    absrow = np.bincount(rows, np.abs(vals), minlength=n)
    diag = dominance * absrow
    diag[diag == 0.0] = 1.0
    d = np.arange(n, dtype=np.int64)
    return csr_from_coo(n, np.concatenate([rows, d]), np.concatenate([cols, d]),
                        np.concatenate([vals, diag]))


def random_tree(n: int, seed: int, diag_scale: float = 1.0, indefinite: bool = False) -> CSR:
    """Random recursive tree: node k > 0 attaches to a uniform node < k.
    Off-diagonals N(0,1); diagonal diag_scale * (1 + |N(0,1)|), with random
    signs when ``indefinite`` (the tree result of Section IV needs neither
    positive definiteness nor diagonal dominance)."""
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, k) for k in range(1, n)], dtype=np.int64)
    child = np.arange(1, n, dtype=np.int64)
    w = rng.standard_normal(n - 1)
    diag = diag_scale * (1.0 + np.abs(rng.standard_normal(n)))
    if indefinite:
        diag *= rng.choice([-1.0, 1.0], n)
    d = np.arange(n, dtype=np.int64)
    return csr_from_coo(n, np.concatenate([parent, child, d]), np.concatenate([child, parent, d]),
                        np.concatenate([w, w, diag]))


def path_graph(n: int, seed: int) -> CSR:
    """Tridiagonal matrix (a path: the tree of largest diameter)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(n - 1)
    diag = 1.0 + 2.5 * np.abs(rng.standard_normal(n))
    i = np.arange(n - 1, dtype=np.int64)
    d = np.arange(n, dtype=np.int64)
    return csr_from_coo(n, np.concatenate([i, i + 1, d]), np.concatenate([i + 1, i, d]),
                        np.concatenate([w, w, diag]))


def uniform_rhs(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def normal_rhs(n: int, seed: int, k: int | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) if k is None else rng.standard_normal((n, k))


@dataclass
class DetectionSystem:
    S: np.ndarray       # N x K spreading matrix, entries +-1/sqrt(N)
    x: np.ndarray       # K transmitted symbols in {+-1}
    y: np.ndarray       # N received chips, y = S x + noise
    sigma2: float       # noise variance

    @property
    def K(self) -> int:
        return self.S.shape[1]

    def dense_system(self):
        """MMSE detector as a linear system: A = S^T S + sigma^2 I, b = S^T y."""
        A = self.S.T @ self.S + self.sigma2 * np.eye(self.K)
        return A, self.S.T @ self.y


def detection_batch(nsys: int, k_min: int, k_max: int, snr_db: float, seed: int,
                    spread: int = 2) -> list[DetectionSystem]:
    """Independent CDMA detection systems: K ~ U{k_min..k_max}, N = spread*K,
    S entries +-1/sqrt(N) (unit-norm columns), symbols +-1 (unit energy), so
    the noise variance at the given SNR is sigma^2 = 10^(-snr_db/10)."""
    rng = np.random.default_rng(seed)
    sigma2 = 10.0 ** (-snr_db / 10.0)
    out = []
    for _ in range(nsys):
        K = int(rng.integers(k_min, k_max + 1))
        N = spread * K
        S = rng.choice([-1.0, 1.0], size=(N, K)) / np.sqrt(N)
        x = rng.choice([-1.0, 1.0], size=K)
        y = S @ x + np.sqrt(sigma2) * rng.standard_normal(N)
        out.append(DetectionSystem(S, x, y, sigma2))
    return out
