"""GPU tests of the launch-shape autotuner and of every shape it can choose.

The tuner picks, per handle, the row-binning threshold and the row-tile shape
of the FP32 sweeps (CSR form), the lanes per row of the FP64 sweep, and the
rows each warp loads ahead in the dense Section VII kernels.  Each candidate
is pinned here through gabp_options and checked against the CPU oracle (or
the closed form), so whichever one the tuner keeps is a tested one.
Tolerances as in test_gpu_parity: 1e-12 per FP64 round, 1e-10 relative
residual and 1e-8 relative error for solves.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1119_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("CUDA device required", allow_module_level=True)


@pytest.fixture(scope="module")
def G():
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    gabp.load()
    return gabp


def _rel(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def _hub_graph(n=30000, seed=4):
    """ER base of degree 4, 40 hubs of degree ~300 and one of degree ~2500
    (longer than any tile): light, heavy and long rows in one matrix."""
    rng = np.random.default_rng(seed)
    base = W.er_sdd(n, 4, 1.1, seed)
    rows = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = rows != base.col
    pairs = {}
    for r, c, v in zip(rows[keep], base.col[keep], base.val[keep]):
        pairs[(int(r), int(c))] = float(v)
    for hb, deg in [(int(h), 300) for h in rng.choice(n, 40, replace=False)] + [(7, 2500)]:
        for j in rng.choice(n, deg, replace=False):
            j = int(j)
            if j != hb and (hb, j) not in pairs:
                w = 0.05 * rng.standard_normal()
                pairs[(hb, j)] = w
                pairs[(j, hb)] = w
    r = np.array([k[0] for k in pairs]); c = np.array([k[1] for k in pairs])
    v = np.array(list(pairs.values()))
    diag = 1.2 * np.bincount(r, np.abs(v), minlength=n) + 0.1
    return W.csr_from_coo(n, np.concatenate([r, np.arange(n)]), np.concatenate([c, np.arange(n)]),
                          np.concatenate([v, diag]))


@pytest.fixture(scope="module")
def hub():
    m = _hub_graph()
    b = W.normal_rhs(m.n, 3)
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=20000, tol=1e-13)
    assert ref["status"] == "ok"
    return m, b, ref["x"]


# every (tile slots, tile rows, heavy degree) the tuner can choose
SHAPES = [(1024, 256, 16), (1024, 256, 32), (1024, 256, 64), (1024, 256, 128), (1024, 256, 1 << 30),
          (512, 256, 64), (512, 128, 64), (256, 64, 64), (256, 64, 1 << 30)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_h{s[2]}")
@pytest.mark.parametrize("precision", [0, 1])
def test_every_tile_shape_solves(G, hub, shape, precision):
    m, b, xref = hub
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, tile_slots=shape[0],
                          tile_rows=shape[1], heavy_degree=shape[2])
    t = s.tuning()
    assert (t["tile_slots"], t["tile_rows"], t["heavy_degree"], t["tuned"]) == (*shape, 0)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert _rel(x, xref) < 1e-8
    s.close()


def test_autotune_mixed_records_its_choice(G, hub):
    m, b, xref = hub
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=1, autotune=True)
    t = s.tuning()
    # 5 heavy-row thresholds + 3 tile shapes + 5 lane counts of the in-place
    # full sweep + 1 to 4 distinct window sizes of the window-form mean sweep
    assert t["tuned"] == 1 and 14 <= t["candidates"] <= 17 and t["tune_ms"] > 0
    assert t["mean_window"] == 0 or 256 <= t["mean_window"] <= 24000
    assert (t["tile_slots"], t["tile_rows"]) in {(1024, 256), (512, 256), (512, 128), (256, 64)}
    assert t["heavy_degree"] in {16, 32, 64, 128, 1 << 30}
    assert t["pull_lanes"] in {0, 2, 4, 8, 16, 32}
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    assert _rel(xt.cpu().numpy(), xref) < 1e-8
    # a repeated solve on the tuned handle meets the same bar (heavy tiles add
    # row sums with shared-memory atomics, so the bits may differ run to run)
    xt2, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    assert _rel(xt2.cpu().numpy(), xref) < 1e-8
    s.close()


def test_autotune_fp64_lanes_keep_round_parity(G):
    m = W.er_sdd(5000, 8, 1.1, 9)
    b = W.normal_rhs(m.n, 4)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, autotune=True)
    t = s.tuning()
    # 5 lane counts, plus the cluster sizes that fit (one-launch solves)
    assert t["tuned"] == 1 and t["candidates"] >= 5 and t["group_lanes"] in {2, 4, 8, 16, 32}
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    for r in (1, 4, 11):
        G.gabp_run_rounds(s.handle, bt, r, xt)
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r)
        assert _rel(xt.cpu().numpy(), ref["x"]) <= 1e-12
    s.close()


@pytest.mark.parametrize("rows", [1, 2, 4, 0])
def test_dense_rows_ahead_solve(G, rows):
    """rows = 0 with autotune: the tuner's pick; 1, 2, 4 pinned."""
    systems = W.detection_batch(30, 16, 200, 10.0, seed=5)
    o = G.gabp_default_options()
    o.precision = 1
    o.dense_rows = rows
    o.autotune = 1 if rows == 0 else 0
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    t = G.gabp_get_tuning(h)
    if rows:
        assert t["dense_rows_mean"] == rows and t["dense_rows_full"] == rows and t["tuned"] == 0
    else:
        assert t["tuned"] == 1 and t["candidates"] == 6
        assert t["dense_rows_mean"] in {1, 2, 4} and t["dense_rows_full"] in {1, 2, 4}
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
    got = xh.cpu().numpy()
    off = 0
    for d in systems:
        A, bb = d.dense_system()
        assert _rel(got[off:off + d.K], np.linalg.solve(A, bb)) < 1e-8
        off += d.K
    G.gabp_destroy(h)
