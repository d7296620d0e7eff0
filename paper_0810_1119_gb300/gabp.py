"""ctypes binding of the C ABI declared in ``include/gabp.h``.

Argument marshalling only: every step of the solve runs inside
``libgabp.so``.  The functions keep the C names (``gabp_create``,
``gabp_solve``, ...); device arrays are passed as ``torch.Tensor`` objects on
the current CUDA device and the handle uses the stream that was current when
it was created (or the one given to ``gabp_set_stream``).

Importing this module loads the library and raises ``RuntimeError`` if it has
not been built (``python -m paper_0810_1119_gb300.build_lib``): there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgabp.so")

# gabp_status
GABP_OK = 0
STATUS_NAMES = {0: "GABP_OK", 1: "GABP_ERR_INVALID_ARG", 2: "GABP_ERR_NOT_SYMMETRIC",
                3: "GABP_ERR_ZERO_DIAG", 4: "GABP_ERR_BREAKDOWN", 5: "GABP_ERR_DIVERGED",
                6: "GABP_ERR_NOT_CONVERGED", 7: "GABP_ERR_CUDA", 8: "GABP_ERR_OOM",
                9: "GABP_ERR_TIMEOUT"}
PREC_FP64, PREC_MIXED_FP32, PREC_MIXED_BF16 = 0, 1, 2
RESIDUAL_ABS, RESIDUAL_REL = 0, 1
SCHEDULE_SYNC, SCHEDULE_COLOUR = 0, 1

# Every symbol include/gabp.h declares (checked by the CPU tests).
EXPORTED = ("gabp_default_options", "gabp_create", "gabp_destroy", "gabp_set_stream",
            "gabp_solve", "gabp_solve_host", "gabp_solve_multi", "gabp_get_stats",
            "gabp_run_rounds", "gabp_get_messages", "gabp_last_error", "gabp_status_string",
            "gabp_version", "gabp_create_batched", "gabp_create_lsq_batched",
            "gabp_solve_lsq_batched", "gabp_run_rounds_noalloc", "gabp_get_tuning",
            "gabp_set_profile", "gabp_create_grid", "gabp_check_wait_limit",
            "gabp_get_system_sweeps")


class GabpOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("residual_kind", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("lsq_form", ctypes.c_int32), ("tile_slots", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("damping", ctypes.c_double), ("tile_rows", ctypes.c_int32),
                ("heavy_degree", ctypes.c_int32), ("dense_rows", ctypes.c_int32),
                ("small_form", ctypes.c_int32), ("cluster_ctas", ctypes.c_int32),
                ("aitken", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("damp_scope", ctypes.c_int32), ("pull_lanes", ctypes.c_int32),
                ("pinv_shift", ctypes.c_double), ("naive", ctypes.c_int32),
                ("mean_window", ctypes.c_int32), ("batch_control", ctypes.c_int32)]


class GabpStats(ctypes.Structure):
    _fields_ = [("sweeps_total", ctypes.c_int32), ("sweeps_full", ctypes.c_int32),
                ("sweeps_mean", ctypes.c_int32), ("outer_steps", ctypes.c_int32),
                ("residual_checks", ctypes.c_int32), ("status", ctypes.c_int32),
                ("residual", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("n", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms_full", ctypes.c_double),
                ("ms_mean", ctypes.c_double), ("ms_residual", ctypes.c_double),
                ("ms_other", ctypes.c_double), ("positions_swept", ctypes.c_int64),
                ("sweeps_wide", ctypes.c_int32), ("aitken_steps", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class GabpTuning(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("tile_slots", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("heavy_degree", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("dense_rows_mean", ctypes.c_int32), ("dense_rows_full", ctypes.c_int32),
                ("cluster_ctas", ctypes.c_int32), ("pull_lanes", ctypes.c_int32),
                ("mean_window", ctypes.c_int32), ("windows", ctypes.c_int32),
                ("tune_ms", ctypes.c_double), ("reserved", ctypes.c_double * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class GabpError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libgabp.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_0810_1119_gb300.build_lib` (needs nvcc)")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    i64p, i32p, f64p = (ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                        ctypes.POINTER(ctypes.c_double))
    vp = ctypes.c_void_p
    sig = {
        "gabp_default_options": (None, [ctypes.POINTER(GabpOptions)]),
        "gabp_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int64, ctypes.c_int64, i64p, i32p,
                                       f64p, i64p, ctypes.POINTER(GabpOptions)]),
        "gabp_destroy": (ctypes.c_int, [H]),
        "gabp_set_stream": (ctypes.c_int, [H, vp]),
        "gabp_solve": (ctypes.c_int, [H, vp, vp, ctypes.c_double, ctypes.c_int32, i32p]),
        "gabp_solve_host": (ctypes.c_int, [H, f64p, f64p, ctypes.c_double, ctypes.c_int32, i32p]),
        "gabp_solve_multi": (ctypes.c_int, [H, vp, vp, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_int32, i32p]),
        "gabp_get_stats": (ctypes.c_int, [H, ctypes.POINTER(GabpStats)]),
        "gabp_get_system_sweeps": (ctypes.c_int, [H, i32p, ctypes.c_int32]),
        "gabp_run_rounds": (ctypes.c_int, [H, vp, ctypes.c_int32, vp]),
        "gabp_get_messages": (ctypes.c_int, [H, f64p, f64p]),
        "gabp_last_error": (ctypes.c_char_p, [H]),
        "gabp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "gabp_version": (ctypes.c_char_p, []),
        "gabp_create_batched": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int32, i64p, ctypes.c_int64,
                                               i64p, i32p, f64p, ctypes.POINTER(GabpOptions)]),
        "gabp_create_lsq_batched": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int32, i32p, i32p, f64p,
                                                   f64p, ctypes.POINTER(GabpOptions)]),
        "gabp_solve_lsq_batched": (ctypes.c_int, [H, vp, vp, ctypes.c_double, ctypes.c_int32, i32p]),
        "gabp_create_grid": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int32, i32p, ctypes.c_int64,
                                            i64p, i32p, f64p, ctypes.POINTER(GabpOptions)]),
        "gabp_run_rounds_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp, vp,
                                                   ctypes.c_int32, vp, vp]),
        "gabp_get_tuning": (ctypes.c_int, [H, ctypes.POINTER(GabpTuning)]),
        "gabp_set_profile": (ctypes.c_int, [H, ctypes.c_int32]),
        "gabp_check_wait_limit": (ctypes.c_int, [H, ctypes.c_int32, f64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(h, status):
    if status != GABP_OK:
        msg = load().gabp_last_error(h)
        raise GabpError(status, msg.decode() if msg else "")


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dev_ptr(t, dtype_name, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch.Tensor")
    if str(t.dtype) != dtype_name or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype_name} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def gabp_default_options() -> GabpOptions:
    o = GabpOptions()
    load().gabp_default_options(ctypes.byref(o))
    return o


def current_stream_handle() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def gabp_create(row_ptr, col, val, rev=None, options: GabpOptions | None = None):
    """Create a solver from a full symmetric CSR given as host (numpy) arrays."""
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    n = row_ptr.shape[0] - 1
    nnz = int(row_ptr[-1]) if n >= 0 else 0
    if options is None:
        options = gabp_default_options()
    revp = None
    if rev is not None:
        rev = np.ascontiguousarray(rev, dtype=np.int64)
        revp = _ptr(rev, ctypes.c_int64)
    h = ctypes.c_void_p()
    st = lib.gabp_create(ctypes.byref(h), n, nnz, _ptr(row_ptr, ctypes.c_int64),
                         _ptr(col, ctypes.c_int32), _ptr(val, ctypes.c_double), revp,
                         ctypes.byref(options))
    _check(None, st)
    return h


def gabp_create_batched(sys_row_off, row_ptr, col, val, options: GabpOptions | None = None):
    """Create a handle over independent systems along the diagonal of one CSR
    (host arrays); sys_row_off[s]..sys_row_off[s+1] are the rows of system s."""
    lib = load()
    sys_row_off = np.ascontiguousarray(sys_row_off, dtype=np.int64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    if options is None:
        options = gabp_default_options()
    h = ctypes.c_void_p()
    st = lib.gabp_create_batched(ctypes.byref(h), len(sys_row_off) - 1, _ptr(sys_row_off, ctypes.c_int64),
                                 int(row_ptr[-1]), _ptr(row_ptr, ctypes.c_int64),
                                 _ptr(col, ctypes.c_int32), _ptr(val, ctypes.c_double),
                                 ctypes.byref(options))
    _check(None, st)
    return h


def gabp_create_grid(dims, row_ptr, col, val, options: GabpOptions | None = None):
    """Create a grid-form handle for a CSR (host arrays, natural order of the
    box ``dims``, x fastest) that couples only nearest neighbours."""
    lib = load()
    d = np.ascontiguousarray(dims, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    if options is None:
        options = gabp_default_options()
    h = ctypes.c_void_p()
    st = lib.gabp_create_grid(ctypes.byref(h), len(d), _ptr(d, ctypes.c_int32), int(row_ptr[-1]),
                              _ptr(row_ptr, ctypes.c_int64), _ptr(col, ctypes.c_int32),
                              _ptr(val, ctypes.c_double), ctypes.byref(options))
    _check(None, st)
    return h


def gabp_create_lsq_batched(S_list, psi, options: GabpOptions | None = None):
    """Create a least-squares batch (Section VII augmented systems) from a list
    of dense S_s (N_s x K_s) and noise variances psi_s (scalar or list); psi_s
    = 0 asks for the Moore-Penrose solution S_s^+ y_s."""
    lib = load()
    K = np.ascontiguousarray([S.shape[1] for S in S_list], dtype=np.int32)
    N = np.ascontiguousarray([S.shape[0] for S in S_list], dtype=np.int32)
    Scat = np.ascontiguousarray(np.concatenate([np.asarray(S, dtype=np.float64).ravel() for S in S_list]))
    psi = np.ascontiguousarray(np.broadcast_to(np.asarray(psi, dtype=np.float64), (len(S_list),)))
    if options is None:
        options = gabp_default_options()
    h = ctypes.c_void_p()
    st = lib.gabp_create_lsq_batched(ctypes.byref(h), len(S_list), _ptr(K, ctypes.c_int32),
                                     _ptr(N, ctypes.c_int32), _ptr(Scat, ctypes.c_double),
                                     _ptr(psi, ctypes.c_double), ctypes.byref(options))
    _check(None, st)
    return h


def gabp_solve_lsq_batched(h, y, xhat, tol: float, max_iter: int) -> int:
    """y: concatenated y_s (device float64), xhat: concatenated x^_s (output)."""
    it = ctypes.c_int32(0)
    st = load().gabp_solve_lsq_batched(h, _dev_ptr(y, "torch.float64"), _dev_ptr(xhat, "torch.float64"),
                                       float(tol), int(max_iter), ctypes.byref(it))
    _check(h, st)
    return it.value


def gabp_destroy(h):
    _check(None, load().gabp_destroy(h))


def gabp_set_stream(h, stream: int):
    _check(h, load().gabp_set_stream(h, ctypes.c_void_p(stream)))


def gabp_solve(h, b, x, tol: float, max_iter: int) -> int:
    """Solve on device tensors b, x (float64, length n).  Returns sweeps."""
    it = ctypes.c_int32(0)
    st = load().gabp_solve(h, _dev_ptr(b, "torch.float64"), _dev_ptr(x, "torch.float64"),
                           float(tol), int(max_iter), ctypes.byref(it))
    _check(h, st)
    return it.value


def gabp_solve_host(h, b: np.ndarray, tol: float, max_iter: int, x: np.ndarray | None = None):
    """Solve with host arrays (copies inside the library).  Returns (x, sweeps)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    if x is None:
        x = np.empty_like(b)
    it = ctypes.c_int32(0)
    st = load().gabp_solve_host(h, _ptr(b, ctypes.c_double), _ptr(x, ctypes.c_double), float(tol),
                                int(max_iter), ctypes.byref(it))
    _check(h, st)
    return x, it.value


def gabp_solve_multi(h, B, X, tol: float, max_iter: int) -> int:
    """B, X: device float64 tensors of shape (n, nrhs), row-major."""
    if B.dim() != 2 or X.shape != B.shape:
        raise ValueError("B and X must be (n, nrhs)")
    it = ctypes.c_int32(0)
    st = load().gabp_solve_multi(h, _dev_ptr(B, "torch.float64"), _dev_ptr(X, "torch.float64"),
                                 int(B.shape[1]), float(tol), int(max_iter), ctypes.byref(it))
    _check(h, st)
    return it.value


def gabp_get_stats(h) -> dict:
    s = GabpStats()
    _check(h, load().gabp_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def gabp_get_system_sweeps(h, nsys: int) -> np.ndarray:
    """Message sweeps each system of a batched handle took part in during the
    last solve (caller's order)."""
    out = np.zeros(nsys, dtype=np.int32)
    _check(h, load().gabp_get_system_sweeps(h, _ptr(out, ctypes.c_int32), int(nsys)))
    return out


def gabp_set_profile(h, on: bool):
    _check(h, load().gabp_set_profile(h, 1 if on else 0))


def gabp_get_tuning(h) -> dict:
    t = GabpTuning()
    _check(h, load().gabp_get_tuning(h, ctypes.byref(t)))
    return t.as_dict()


def gabp_run_rounds(h, b, rounds: int, x):
    _check(h, load().gabp_run_rounds(h, _dev_ptr(b, "torch.float64"), int(rounds),
                                     _dev_ptr(x, "torch.float64")))


def gabp_get_messages(h, nnz: int):
    P = np.empty(nnz)
    mu = np.empty(nnz)
    _check(h, load().gabp_get_messages(h, _ptr(P, ctypes.c_double), _ptr(mu, ctypes.c_double)))
    return P, mu


def gabp_run_rounds_noalloc(row_ptr, col, val, rev, b, rounds: int, x, stream: int | None = None):
    """FP64 rounds without any device allocation by the library (for callers
    that cannot allocate): every argument is a device tensor the caller owns
    (row_ptr int64, col int32, val float64, rev int64, b / x float64)."""
    n, nnz = b.numel(), val.numel()
    st = load().gabp_run_rounds_noalloc(
        n, nnz, _dev_ptr(row_ptr, "torch.int64", n + 1), _dev_ptr(col, "torch.int32", nnz),
        _dev_ptr(val, "torch.float64"), _dev_ptr(rev, "torch.int64", nnz),
        _dev_ptr(b, "torch.float64"), int(rounds), _dev_ptr(x, "torch.float64", n),
        ctypes.c_void_p(current_stream_handle() if stream is None else stream))
    _check(None, st)


def gabp_check_wait_limit(h, limit_us: int = 0):
    """Make the sweeps' bounded device wait run out on purpose (see
    include/gabp.h): `limit_us` microseconds, 0 = the library's own limit.
    Returns (status name, seconds waited); the expected status is
    GABP_ERR_TIMEOUT, and the handle stays usable."""
    sec = ctypes.c_double(0.0)
    st = load().gabp_check_wait_limit(h, int(limit_us), ctypes.byref(sec))
    return STATUS_NAMES.get(st, str(st)), sec.value


def gabp_version() -> str:
    return load().gabp_version().decode()


def _options(*, precision=PREC_FP64, residual_kind=RESIDUAL_REL, check_every=0, group_lanes=0,
             inner_tol=0.0, profile=False, damping=0.0, stream: int | None = None, autotune=False,
             tile_slots=0, tile_rows=0, heavy_degree=0, small_form=0, cluster_ctas=0, aitken=0,
             schedule=0, damp_scope=0, pull_lanes=0, naive=0, mean_window=0) -> GabpOptions:
    o = gabp_default_options()
    o.precision = precision
    o.residual_kind = residual_kind
    o.check_every = check_every
    o.group_lanes = group_lanes
    o.inner_tol = inner_tol
    o.profile = 1 if profile else 0
    o.damping = damping
    o.stream = current_stream_handle() if stream is None else stream
    o.autotune = 1 if autotune else 0
    o.tile_slots = tile_slots
    o.tile_rows = tile_rows
    o.heavy_degree = heavy_degree
    o.small_form = small_form
    o.cluster_ctas = cluster_ctas
    o.aitken = aitken
    o.schedule = schedule
    o.damp_scope = damp_scope
    o.pull_lanes = pull_lanes
    o.naive = naive
    o.mean_window = mean_window
    return o


@dataclass
class Solver:
    """Owning wrapper: ``Solver(csr, precision=...)`` then ``solve(b)``."""
    handle: ctypes.c_void_p
    n: int
    nnz: int

    @classmethod
    def from_csr(cls, row_ptr, col, val, rev=None, *, precision=PREC_FP64,
                 residual_kind=RESIDUAL_REL, check_every=0, group_lanes=0, inner_tol=0.0,
                 profile=False, damping=0.0, stream: int | None = None, autotune=False,
                 tile_slots=0, tile_rows=0, heavy_degree=0, small_form=0, cluster_ctas=0,
                 aitken=0, schedule=0, damp_scope=0, pull_lanes=0, naive=0, mean_window=0):
        o = _options(precision=precision, residual_kind=residual_kind, check_every=check_every,
                     group_lanes=group_lanes, inner_tol=inner_tol, profile=profile, damping=damping,
                     stream=stream, autotune=autotune, tile_slots=tile_slots, tile_rows=tile_rows,
                     heavy_degree=heavy_degree, small_form=small_form, cluster_ctas=cluster_ctas,
                     aitken=aitken, schedule=schedule, damp_scope=damp_scope, pull_lanes=pull_lanes,
                     naive=naive, mean_window=mean_window)
        h = gabp_create(row_ptr, col, val, rev, o)
        return cls(h, len(row_ptr) - 1, int(row_ptr[-1]))

    @classmethod
    def from_grid(cls, dims, row_ptr, col, val, *, precision=PREC_FP64, residual_kind=RESIDUAL_REL,
                  check_every=0, inner_tol=0.0, profile=False, damping=0.0,
                  stream: int | None = None, aitken=0, schedule=0, damp_scope=0):
        """Grid form (gabp_create_grid): ``dims`` of the box, CSR in its natural order."""
        o = _options(precision=precision, residual_kind=residual_kind, check_every=check_every,
                     inner_tol=inner_tol, profile=profile, damping=damping, stream=stream,
                     aitken=aitken, schedule=schedule, damp_scope=damp_scope)
        h = gabp_create_grid(dims, row_ptr, col, val, o)
        return cls(h, len(row_ptr) - 1, int(row_ptr[-1]))

    def solve(self, b, x=None, tol=1e-10, max_iter=10000):
        import torch
        if x is None:
            x = torch.empty_like(b)
        iters = gabp_solve(self.handle, b, x, tol, max_iter)
        return x, iters

    def tuning(self) -> dict:
        return gabp_get_tuning(self.handle)

    def stats(self) -> dict:
        return gabp_get_stats(self.handle)

    def close(self):
        if self.handle:
            gabp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
