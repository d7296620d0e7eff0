"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/gabp.h declares, and its host-side validation rejects bad
matrices before any device work (no GPU needed for any of this)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_0810_1119_gb300 import build_lib
from paper_0810_1119_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gabp.h")


@pytest.fixture(scope="module")
def lib():
    path = build_lib.build()
    from paper_0810_1119_gb300 import gabp
    return gabp.load(path)


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gabp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    from paper_0810_1119_gb300 import gabp
    assert _declared_functions() == sorted(gabp.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gabp_\w+)", out))
    for name in _declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_default_options_and_strings(lib):
    from paper_0810_1119_gb300 import gabp
    o = gabp.gabp_default_options()
    assert o.precision == gabp.PREC_FP64 and o.residual_kind == gabp.RESIDUAL_REL
    assert o.inner_tol == 0.0   # automatic
    assert lib.gabp_status_string(4) == b"GABP_ERR_BREAKDOWN"
    assert b"sm_103a" in lib.gabp_version()


def _create_status(m, rev=None):
    from paper_0810_1119_gb300 import gabp
    try:
        gabp.gabp_create(m.row_ptr, m.col, m.val, rev)
    except gabp.GabpError as e:
        return e.name, str(e)
    return "GABP_OK", ""


@pytest.mark.parametrize("A,expect", [
    (np.array([[2.0, 1.0], [0.5, 2.0]]), "GABP_ERR_NOT_SYMMETRIC"),
    (np.array([[2.0, 1.0], [0.0, 2.0]]), "GABP_ERR_NOT_SYMMETRIC"),
    (np.array([[0.0, 1.0], [1.0, 2.0]]), "GABP_ERR_ZERO_DIAG"),
])
def test_create_rejects_bad_matrices_on_the_host(lib, A, expect):
    status, msg = _create_status(W.csr_from_dense(A))
    assert status == expect, msg


def test_create_rejects_malformed_csr(lib):
    m = W.poisson2d(3)
    bad = W.CSR(m.n, m.row_ptr.copy(), m.col.copy(), m.val.copy())
    bad.col[1], bad.col[2] = bad.col[2], bad.col[1]     # unsorted row
    assert _create_status(bad)[0] == "GABP_ERR_INVALID_ARG"
    bad = W.CSR(m.n, m.row_ptr.copy(), m.col.copy(), m.val.copy())
    bad.col[0] = m.n + 5                                # out of range
    assert _create_status(bad)[0] == "GABP_ERR_INVALID_ARG"


def test_create_rejects_wrong_rev(lib):
    m = W.poisson2d(4)
    rev = W.reverse_index(m)
    off = np.flatnonzero(np.repeat(np.arange(m.n), np.diff(m.row_ptr)) != m.col)
    rev[off[0]], rev[off[1]] = rev[off[1]], rev[off[0]]
    assert _create_status(m, rev)[0] == "GABP_ERR_NOT_SYMMETRIC"


def test_reverse_index_is_an_involution():
    m = W.er_sdd(500, 6, 1.1, 3)
    rev = W.reverse_index(m)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    assert np.array_equal(rev[rev], np.arange(m.nnz))
    assert np.array_equal(m.col[rev], rows)


def test_create_batched_rejects_coupled_systems(lib):
    from paper_0810_1119_gb300 import gabp
    A = np.array([[4.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.0, 1.0, 4.0]])
    m = W.csr_from_dense(A)
    with pytest.raises(gabp.GabpError) as ei:
        gabp.gabp_create_batched([0, 1, 3], m.row_ptr, m.col, m.val)   # (0,1) couples the systems
    assert ei.value.name == "GABP_ERR_INVALID_ARG"


def test_create_lsq_batched_rejects_bad_noise(lib):
    """psi_s must be finite and >= 0 (0 asks for the Moore-Penrose solution),
    pinv_shift finite and >= 0; refused on the host before any device work."""
    from paper_0810_1119_gb300 import gabp
    S = np.ones((4, 2)) / 2.0
    for psi in (-0.1, float("nan"), float("inf")):
        with pytest.raises(gabp.GabpError) as ei:
            gabp.gabp_create_lsq_batched([S], psi)
        assert ei.value.name == "GABP_ERR_INVALID_ARG"
        assert "psi_s >= 0" in str(ei.value)
    for shift in (-1.0, float("nan")):
        o = gabp.gabp_default_options()
        o.pinv_shift = shift
        with pytest.raises(gabp.GabpError) as ei:
            gabp.gabp_create_lsq_batched([S], 0.0, o)
        assert "pinv_shift" in str(ei.value)


def test_launch_shape_options_are_validated():
    """Out-of-range launch shapes are refused on the host, before any device
    work (no GPU needed)."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for field, value in (("tile_slots", 16), ("tile_slots", 2048), ("tile_rows", 300),
                         ("heavy_degree", -1), ("dense_rows", 3), ("cluster_ctas", 3), ("aitken", -1),
                         ("schedule", 2), ("schedule", -1)):
        o = G.gabp_default_options()
        setattr(o, field, value)
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert ei.value.name == "GABP_ERR_INVALID_ARG"
        assert "launch shape" in str(ei.value)


def test_colour_schedule_refusals_are_host_checks(lib):
    """The colour schedule is refused for block-diagonal batches and for
    Section VII batches outside the dense form, before any device work."""
    from paper_0810_1119_gb300 import gabp as G
    o = G.gabp_default_options()
    o.schedule = 1
    m = W.poisson2d(4)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_batched([0, m.n], m.row_ptr, m.col, m.val, o)
    assert ei.value.name == "GABP_ERR_INVALID_ARG"
    S = np.ones((4, 2)) / 2.0
    o.lsq_form = 1                                   # general CSR form
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_lsq_batched([S], 0.1, o)
    assert "dense form" in str(ei.value)
    o.lsq_form = 0                                   # K = 300 is beyond the dense kernels
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_lsq_batched([S, np.ones((300, 300)) / 300.0], 0.1, o)
    assert "dense form" in str(ei.value)


def test_damp_scope_is_validated(lib):
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for schedule, scope in ((0, 1), (1, 2), (1, -1)):
        o = G.gabp_default_options()
        o.schedule, o.damp_scope = schedule, scope
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert "damp_scope" in str(ei.value)


def test_pull_lanes_is_validated(lib):
    """The in-place FP32 full sweep takes 2..32 lanes per row (powers of two)
    and needs the synchronous schedule without damping; refused on the host."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for lanes, damping, schedule in ((3, 0.0, 0), (64, 0.0, 0), (-2, 0.0, 0), (1, 0.0, 0),
                                     (8, 0.2, 0), (8, 0.0, 1)):
        o = G.gabp_default_options()
        o.precision = G.PREC_MIXED_FP32
        o.pull_lanes, o.damping, o.schedule = lanes, damping, schedule
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert ei.value.name == "GABP_ERR_INVALID_ARG"
        assert "pull_lanes" in str(ei.value)


def test_mean_window_is_validated(lib):
    """The window form of the mean sweep takes windows of 256..65536 slots
    (-1 = tile form, 0 = automatic) and needs the synchronous schedule;
    refused on the host."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for mw, schedule in ((-2, 0), (1, 0), (255, 0), (65537, 0), (1024, 1)):
        o = G.gabp_default_options()
        o.precision = G.PREC_MIXED_FP32
        o.mean_window, o.schedule = mw, schedule
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert ei.value.name == "GABP_ERR_INVALID_ARG"
        assert "mean_window" in str(ei.value)


def test_batch_control_is_validated(lib):
    """batch_control is 0 (per system) or 1 (whole batch); refused on the host,
    and gabp_get_system_sweeps refuses a handle that is not batched."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for bc in (-1, 2):
        o = G.gabp_default_options()
        o.batch_control = bc
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert ei.value.name == "GABP_ERR_INVALID_ARG"
        assert "batch_control" in str(ei.value)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_get_system_sweeps(None, 1)
    assert ei.value.name == "GABP_ERR_INVALID_ARG"


def test_naive_is_validated(lib):
    """Algorithm 1 (naive = 1) needs FP64, the synchronous schedule and no
    damping; refused on the host."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(4)
    for naive, prec, schedule, damping in ((2, 0, 0, 0.0), (-1, 0, 0, 0.0), (1, 1, 0, 0.0),
                                          (1, 0, 1, 0.0), (1, 0, 0, 0.2)):
        o = G.gabp_default_options()
        o.naive, o.precision, o.schedule, o.damping = naive, prec, schedule, damping
        with pytest.raises(G.GabpError) as ei:
            G.gabp_create(m.row_ptr, m.col, m.val, None, o)
        assert "naive" in str(ei.value)


def test_grid_create_validates_on_the_host(lib):
    """gabp_create_grid accepts only a nearest-neighbour operator on the box
    given, in natural order, with an even first dimension; every refusal is
    a host check (no GPU needed)."""
    from paper_0810_1119_gb300 import gabp as G
    m = W.poisson2d(6)                                   # 6 x 6, natural order
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_grid([5, 6], m.row_ptr, m.col, m.val)   # odd first dimension (and 30 != 36 rows)
    assert ei.value.name == "GABP_ERR_INVALID_ARG"
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_grid([4, 9], m.row_ptr, m.col, m.val)   # +-6 is no neighbour offset of a 4 x 9 box
    assert "nearest neighbour" in str(ei.value)
    A = np.zeros((8, 8))                                 # 4 x 2 box with a coupling that wraps a row
    for i in range(8):
        A[i, i] = 4.0
    A[3, 4] = A[4, 3] = -1.0                             # (x=3, y=0) - (x=0, y=1): not adjacent
    w = W.csr_from_dense(A)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_grid([4, 2], w.row_ptr, w.col, w.val)
    assert "nearest neighbour" in str(ei.value)
    A[3, 4] = A[4, 3] = 0.0
    A[0, 1], A[1, 0] = -1.0, -0.5                        # neighbours, but not symmetric
    w = W.csr_from_dense(A)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_grid([4, 2], w.row_ptr, w.col, w.val)
    assert ei.value.name == "GABP_ERR_NOT_SYMMETRIC"
    with pytest.raises(G.GabpError) as ei:
        G.gabp_create_grid([6, 4], m.row_ptr, m.col, m.val)   # 24 rows expected, 36 given
    assert ei.value.name == "GABP_ERR_INVALID_ARG"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    of the C structures in include/gabp.h (compiled here with the host C
    compiler), so options, statistics and tuning cross the ABI intact."""
    import shutil
    from paper_0810_1119_gb300 import gabp as G
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"gabp_options": G.GabpOptions, "gabp_stats": G.GabpStats, "gabp_tuning": G.GabpTuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gabp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
