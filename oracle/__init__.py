"""Plain FP64 CPU oracle for Gaussian belief propagation on Ax = b.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's ``smoke()``
check and the benchmark's CPU-baseline leg may import this package.  It
shares no code with the CUDA library (``paper_0810_1119_gb300``) and never
imports it; the CUDA library never imports this package.

Contents
--------
* ``gabp``          -- synchronous GaBP from zero messages in one of three
                       variants: the broadcast form (Algorithm 2), the naive
                       form (Algorithm 1) and the Jacobi reduction (GaBP/Jacobi
                       proposition, Section VI-C).  C code in ``gabp_oracle.c``.
* ``residual_inf``  -- ||b - A x||_inf (Section II, residual definition).
* ``augment_lsq``   -- the symmetric augmented system of Section VII
                       (``augment.py``).
* ``pinv_solution``, ``iterated_tikhonov`` -- Section VII with Psi = 0: the
                       Moore-Penrose solution, and the iteration that reaches
                       it through augmented solves with Psi_0 > 0
                       (``augment.py``).
* ``gabp_serial``   -- the serial schedule of Section III-C over a given node
                       order (``greedy_colouring`` gives colour classes).
* ``aitken``, ``gabp_aitken`` -- Aitken's Delta^2 extrapolation of the
                       tentative means (Section IV-A, convergence acceleration),
                       applied per node to the means of rounds t - 2s, t - s
                       and t.
* ``steffensen_residual`` -- Steffensen's iteration (Section IV-A) in
                       residual form: GaBP on the residual from zero messages,
                       Delta^2 of three of its iterates, the extrapolated
                       correction added to x, repeated.

Every function is pinned by CPU tests (``tests/test_oracle_*.py``) to values
the paper prints, closed forms and brute force -- not to itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .augment import augment_lsq, iterated_tikhonov, pinv_solution  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BROADCAST, NAIVE, JACOBI = 0, 1, 2
STOP_FIXED, STOP_MSG, STOP_RES_ABS, STOP_RES_REL = 0, 1, 2, 3
STATUS = {0: "ok", 1: "bad_input", 2: "breakdown", 3: "not_converged"}


def build(force: bool = False) -> str:
    """Compile ``gabp_oracle.c`` with gcc into ``_build/liboracle.so``.

    IEEE semantics are kept: no fast-math and no FMA contraction, so the
    oracle rounds the same way on every host.
    """
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _bind(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_gabp.restype = ctypes.c_int
    lib.oracle_gabp.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, i32p, f64p, f64p,
                                ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                f64p, f64p, f64p, f64p, ctypes.POINTER(ctypes.c_int),
                                ctypes.c_double]
    lib.oracle_gabp_serial.restype = ctypes.c_int
    lib.oracle_gabp_serial.argtypes = [ctypes.c_int64, i64p, i32p, f64p, f64p, i64p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       f64p, f64p, f64p, f64p, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_uint8)]
    lib.oracle_residual_inf.restype = ctypes.c_double
    lib.oracle_residual_inf.argtypes = [ctypes.c_int64, i64p, i32p, f64p, f64p, f64p, f64p]
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def compile_variant(source: str, out_path: str):
    """Compile an edited copy of the oracle source (used by the tests that
    plant a mistake in the oracle and check that its pins catch it)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", src, "-o", out_path, "-lm"], check=True)
    return _bind(ctypes.CDLL(out_path))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _csr_arrays(row_ptr, col, val):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return row_ptr, col, val


def gabp(row_ptr, col, val, b, *, variant=BROADCAST, stop=STOP_FIXED, max_rounds=1,
         tol=0.0, want_messages=False, lib=None, damping=0.0):
    """Synchronous GaBP from zero messages on the CSR matrix (row_ptr, col, val).

    The CSR holds the full symmetric matrix with its diagonal and sorted
    columns.  Returns a dict with ``x`` (tentative means after the last
    round), ``Pi`` (marginal precisions), ``rounds``, ``status`` and, if
    ``want_messages``, ``P`` and ``mu``: the last round's message i -> j at
    the CSR position of entry (i, j) (zero on the diagonal).  In the Jacobi
    variant ``mu`` holds the product P_ij mu_ij, as the proposition carries it.
    ``damping`` (broadcast variant) blends each new message's P_ij mu_ij
    with the previous round's: gamma old + (1 - gamma) new.
    """
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = row_ptr.shape[0] - 1
    nnz = int(row_ptr[-1])
    x = np.empty(n)
    Pi = np.empty(n)
    P = np.empty(nnz) if want_messages else None
    mu = np.empty(nnz) if want_messages else None
    rounds = ctypes.c_int(0)
    st = (lib or _load()).oracle_gabp(variant, n, _ptr(row_ptr, ctypes.c_int64), _ptr(col, ctypes.c_int32),
                             _ptr(val, ctypes.c_double), _ptr(b, ctypes.c_double), stop,
                             int(max_rounds), float(tol), _ptr(x, ctypes.c_double),
                             _ptr(Pi, ctypes.c_double), _ptr(P, ctypes.c_double),
                             _ptr(mu, ctypes.c_double), ctypes.byref(rounds), float(damping))
    out = {"x": x, "Pi": Pi, "rounds": rounds.value, "status": STATUS[st]}
    if want_messages:
        out["P"], out["mu"] = P, mu
    return out


def gabp_serial(row_ptr, col, val, b, *, order=None, stop=STOP_FIXED, max_rounds=1, tol=0.0,
                want_messages=False, damping=0.0, damp_from=None, lib=None):
    """GaBP under the serial schedule (Section III-C): every round visits the
    nodes in ``order`` (default: natural), each one computing its totals
    from the latest messages and overwriting its outgoing messages.
    ``damp_from`` (boolean per node, default all) limits the damping blend to
    the messages those nodes send.  Output as ``gabp``."""
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = row_ptr.shape[0] - 1
    nnz = int(row_ptr[-1])
    order_a = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    mask = None if damp_from is None else np.ascontiguousarray(damp_from, dtype=np.uint8)
    if mask is not None and mask.shape != (row_ptr.shape[0] - 1,):
        raise ValueError("damp_from needs one flag per node")
    x = np.empty(n)
    Pi = np.empty(n)
    P = np.empty(nnz) if want_messages else None
    mu = np.empty(nnz) if want_messages else None
    rounds = ctypes.c_int(0)
    st = (lib or _load()).oracle_gabp_serial(
        n, _ptr(row_ptr, ctypes.c_int64), _ptr(col, ctypes.c_int32), _ptr(val, ctypes.c_double),
        _ptr(b, ctypes.c_double), _ptr(order_a, ctypes.c_int64), stop, int(max_rounds), float(tol),
        _ptr(x, ctypes.c_double), _ptr(Pi, ctypes.c_double), _ptr(P, ctypes.c_double),
        _ptr(mu, ctypes.c_double), ctypes.byref(rounds), float(damping), _ptr(mask, ctypes.c_uint8))
    out = {"x": x, "Pi": Pi, "rounds": rounds.value, "status": STATUS[st]}
    if want_messages:
        out["P"], out["mu"] = P, mu
    return out


def greedy_colouring(row_ptr, col):
    """Colour classes of the graph of A (no two adjacent nodes share a
    colour), greedy in natural order.  Returns an int array of colours."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col)
    n = row_ptr.shape[0] - 1
    c = -np.ones(n, dtype=np.int64)
    for i in range(n):
        used = {int(c[j]) for j in col[row_ptr[i]:row_ptr[i + 1]] if j != i and c[j] >= 0}
        k = 0
        while k in used:
            k += 1
        c[i] = k
    return c


def residual_inf(row_ptr, col, val, b, x):
    """||b - A x||_inf computed row by row in FP64."""
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = row_ptr.shape[0] - 1
    return float(_load().oracle_residual_inf(n, _ptr(row_ptr, ctypes.c_int64),
                                             _ptr(col, ctypes.c_int32), _ptr(val, ctypes.c_double),
                                             _ptr(b, ctypes.c_double), _ptr(x, ctypes.c_double),
                                             None))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(k: int) -> None:
    _load().oracle_set_num_threads(int(k))


def aitken(x0, x1, x2):
    """Aitken's Delta^2 per node (Section IV-A, convergence acceleration):
    y = x0 - (x1 - x0)^2 / (x2 - 2 x1 + x0) for three iterates of a sequence
    that converges linearly.  Where the second difference is not above the
    rounding level of the iterates (|x2 - 2 x1 + x0| <= 64 eps max|x_k|) the
    formula carries no information and the latest iterate x2 is kept."""
    x0 = np.asarray(x0, dtype=np.float64)
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    d1 = x1 - x0
    den = (x2 - x1) - d1
    scale = np.maximum(np.maximum(np.abs(x0), np.abs(x1)), np.abs(x2))
    ok = np.abs(den) > 64.0 * np.finfo(np.float64).eps * scale
    y = np.where(ok, x0 - d1 * d1 / np.where(ok, den, 1.0), x2)
    return y


def gabp_aitken(row_ptr, col, val, b, rounds: int, stride: int = 2, damping: float = 0.0):
    """Aitken-extrapolated means after `rounds` synchronous rounds: the
    Delta^2 of the tentative means of rounds rounds - 2 stride,
    rounds - stride and rounds (plain means when rounds < 2 stride)."""
    if rounds < 2 * stride:
        return gabp(row_ptr, col, val, b, max_rounds=rounds, damping=damping)["x"]
    xs = [gabp(row_ptr, col, val, b, max_rounds=r, damping=damping)["x"]
          for r in (rounds - 2 * stride, rounds - stride, rounds)]
    return aitken(*xs)


def steffensen_residual(row_ptr, col, val, b, *, inner_rounds: int, spacing: int,
                        outer_steps: int):
    """Steffensen's iteration (Section IV-A) in residual form, FP64.

    Each step takes the residual r = b - A x, runs synchronous GaBP (Alg. 2)
    on A d = r from zero messages, takes its tentative means after
    inner_rounds - 2 spacing, inner_rounds - spacing and inner_rounds rounds,
    forms their Delta^2 value y (``aitken``) and sets x <- x + y: the
    extrapolated value replaces the iterate and GaBP is run again, on the new
    residual.  With spacing = 0 the step adds the last means unchanged (plain
    iterative refinement, the comparison).  A x uses scipy's CSR product.
    Returns x and the infinity norms of the residual before each step and
    after the last."""
    import scipy.sparse as sp
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = row_ptr.size - 1
    A = sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col, dtype=np.int64), row_ptr),
                      shape=(n, n))
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n)
    hist = []
    for _ in range(outer_steps):
        r = b - A @ x
        hist.append(float(np.abs(r).max()))
        if spacing > 0 and inner_rounds >= 2 * spacing:
            ds = [gabp(row_ptr, col, val, r, max_rounds=k)["x"]
                  for k in (inner_rounds - 2 * spacing, inner_rounds - spacing, inner_rounds)]
            y = aitken(*ds)
        else:
            y = gabp(row_ptr, col, val, r, max_rounds=inner_rounds)["x"]
        x = x + y
    hist.append(float(np.abs(b - A @ x).max()))
    return x, hist
