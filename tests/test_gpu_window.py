"""Window form of the mean-only sweep (option mean_window), through the C ABI.

The window form computes the same round of Alg. 2 with frozen precisions as
the tile form -- eta_ij = c_ij (h~_i - eta_ji), h~_i = rhs_i + sum_k eta_ki --
and changes only where the messages live between sweeps (sorted by
destination, moved as contiguous runs through shared memory) instead of
scattering each one to its receiver's slot.

Tolerances (written here, derived from the arithmetic):
  * a row of degree <= 64 is summed by one thread in slot order in both
    forms, and every message is c * (h~ - eta) in FP32, so those sweeps agree
    bit for bit; a row of degree > 64 is summed by a warp in a fixed
    butterfly order in the window form and by segmented sums and shared
    atomics in the tile form: the same FP32 terms in another order, a few
    ulps (6e-8) per node total per sweep.  The sweeps contract, so the x of a
    mixed solve stopped after k <= 40 sweeps agrees to 1e-5 relative --
    compared whenever the two solves stopped in the same controller state
    (same full, mean and outer counts; a decision taken one sweep apart on
    rounding noise is not a difference in the sweep).
  * the window form is deterministic: the same solve twice gives the same
    bits and the same sweep counts.
  * solves: the FP64 residual, recomputed by the oracle, below 1e-10
    relative, and the error against the oracle's converged solution below
    1e-8 relative, as for the other forms.
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


def _hub_with_ring(n_leaves, seed):
    """A hub joined to every other node plus a ring: one row of degree
    n_leaves next to rows of degree 3."""
    rng = np.random.default_rng(seed)
    n = n_leaves + 1
    A = np.zeros((n, n))
    for k in range(1, n):
        A[0, k] = A[k, 0] = rng.standard_normal() * 0.1
        nxt = 1 + (k % n_leaves)
        if nxt != k:
            w = rng.standard_normal() * 0.3
            A[k, nxt] += w / 2
            A[nxt, k] += w / 2
    np.fill_diagonal(A, 1.5 * np.abs(A).sum(1) + 0.5)
    return W.csr_from_dense(A)


def _x_after(G, s, bt, k):
    """x of a mixed solve stopped by max_iter = k: ||r|| times the FP32 means
    of the last sweep (the solve ends NOT_CONVERGED), and the controller state
    it stopped in."""
    xt = torch.zeros_like(bt)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve(s.handle, bt, xt, 1e-30, k)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    st = s.stats()
    return xt.cpu().numpy(), (st["sweeps_full"], st["sweeps_mean"], st["outer_steps"])


def _compare_sweeps(G, tile, win, bt, ks, tol):
    compared = 0
    for k in ks:
        xa, sa = _x_after(G, tile, bt, k)
        xb, sb = _x_after(G, win, bt, k)
        if sa != sb:
            continue
        assert _rel(xb, xa) <= tol, (k, _rel(xb, xa))
        compared += 1
    assert compared >= len(ks) - 3, compared
    return compared


# (graph, window target, has a row of degree > 64 -- summed by a warp)
SWEEP_CASES = {
    "er_3000_w256": (W.er_sdd(3000, 8, 1.1, 5), 256, False),
    "er_3000_w2048": (W.er_sdd(3000, 8, 1.1, 5), 2048, False),
    "er_ragged_isolated_w300": (W.er_sdd(3001, 3, 1.05, 2), 300, False),
    "poisson2d_p20_w512": (W.poisson2d(20), 512, False),
    "tree_400_w256": (W.random_tree(400, 5, diag_scale=3.0), 256, False),
    "one_window": (W.er_sdd(2000, 6, 1.2, 8), 65536, False),
    "hub_300_w256": (_hub_with_ring(300, 3), 256, True),
}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name", sorted(SWEEP_CASES))
def test_window_sweeps_match_tile_sweeps(G, name, prec):
    m, target, _ = SWEEP_CASES[name]
    precision = G.PREC_MIXED_FP32 if prec == "fp32" else G.PREC_MIXED_BF16
    b = W.normal_rhs(m.n, 31)
    bt = torch.tensor(b, device="cuda")
    # the tile form with every row thread-per-row (no slot-parallel tiles)
    tile = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, mean_window=-1,
                             pull_lanes=-1, heavy_degree=1 << 20)
    win = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, mean_window=target,
                            pull_lanes=-1, heavy_degree=1 << 20)
    t = win.tuning()
    assert t["mean_window"] == target and t["windows"] >= 1
    assert tile.tuning()["mean_window"] == 0
    _compare_sweeps(G, tile, win, bt, list(range(1, 16)) + [20, 27, 40], 1e-5)
    assert win.stats()["sweeps_mean"] > 1
    tile.close()
    win.close()


def _oracle_solution(m, b):
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=100000,
                      tol=1e-13)
    assert ref["status"] == "ok"
    return ref["x"]


SOLVE_CASES = {
    "er_20000": (W.er_sdd(20000, 8, 1.1, 11), 1024),
    "er_dom105_deg10": (W.er_sdd(20000, 10, 1.05, 12), 4096),
    "poisson3d_p16": (W.poisson3d(16), 2048),
    "hub_300": (_hub_with_ring(300, 4), 256),
    "tree_indefinite_300": (W.random_tree(300, 2, diag_scale=2.0), 256),
}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name", sorted(SOLVE_CASES))
def test_window_solve_matches_oracle(G, name, prec):
    m, target = SOLVE_CASES[name]
    if prec == "bf16" and name in ("poisson3d_p16", "tree_indefinite_300"):
        pytest.skip("BF16 mean storage does not reach 1e-10 on this system (either form)")
    precision = G.PREC_MIXED_FP32 if prec == "fp32" else G.PREC_MIXED_BF16
    b = W.normal_rhs(m.n, 41)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, mean_window=target)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=50000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert _rel(x, _oracle_solution(m, b)) < 1e-8
    st = s.stats()
    assert st["status"] == 0 and st["sweeps_mean"] > 0
    s.close()


def test_window_damped_sweeps_match_tile_sweeps(G):
    """Damping blends each message with its previous value, which the window
    form reads at the same send-order position (and, right after a freeze,
    from the slot layout)."""
    m = W.er_sdd(2500, 7, 1.05, 21)
    b = W.normal_rhs(m.n, 22)
    bt = torch.tensor(b, device="cuda")
    tile = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, damping=0.3,
                             mean_window=-1, heavy_degree=1 << 20)
    win = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, damping=0.3,
                            mean_window=512, heavy_degree=1 << 20)
    _compare_sweeps(G, tile, win, bt, list(range(1, 14)) + [18, 25], 1e-5)
    xt, _ = win.solve(bt, tol=1e-10, max_iter=50000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert _rel(x, _oracle_solution(m, b)) < 1e-8
    tile.close()
    win.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_window_solves_are_deterministic(G, prec):
    """The same solve twice on one handle: the same x bit for bit and the
    same sweep counts (every sum in the window form has a fixed order)."""
    m = W.er_sdd(30000, 8, 1.1, 17)
    precision = G.PREC_MIXED_FP32 if prec == "fp32" else G.PREC_MIXED_BF16
    bt = torch.tensor(W.normal_rhs(m.n, 18), device="cuda")
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, mean_window=2048,
                          pull_lanes=-1)
    runs = []
    for _ in range(2):
        xt, it = s.solve(bt, tol=1e-10, max_iter=50000)
        st = s.stats()
        runs.append((xt.cpu().numpy(), it, st["sweeps_full"], st["sweeps_mean"], st["outer_steps"]))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1:] == runs[1][1:]
    s.close()


def test_window_batched_systems(G):
    """Independent systems in one block-diagonal handle: windows span system
    boundaries; every system meets its own relative rule."""
    mats = [W.er_sdd(800, 8, 1.1, 1), W.poisson2d(12), W.random_tree(300, 2, diag_scale=2.0),
            W.er_sdd(1500, 5, 1.2, 3)]
    n = sum(m.n for m in mats)
    rows, cols, vals, off = [], [], [], [0]
    for m in mats:
        r = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
        rows.append(r + off[-1]); cols.append(m.col + off[-1]); vals.append(m.val)
        off.append(off[-1] + m.n)
    big = W.csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    scales = [1.0, 1e-6, 1e3, 1.0]
    b = np.concatenate([sc * W.normal_rhs(m.n, 10 + k) for k, (m, sc) in enumerate(zip(mats, scales))])
    o = G.gabp_default_options()
    o.precision = G.PREC_MIXED_FP32
    o.mean_window = 700
    o.stream = G.current_stream_handle()
    h = G.gabp_create_batched(np.array(off, dtype=np.int64), big.row_ptr, big.col, big.val, o)
    s = G.Solver(h, big.n, big.nnz)
    assert s.tuning()["windows"] > 1
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    for k, m in enumerate(mats):
        bs, xs = b[off[k]:off[k + 1]], x[off[k]:off[k + 1]]
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, bs, xs) < 1e-10 * np.abs(bs).max(), k
    s.close()


def test_window_handle_repeats_solves_and_multi_rhs(G):
    """A second solve on the same handle freezes again and rebuilds the
    send-ordered coefficients; the multi-RHS path keeps the slot layout."""
    m = W.er_sdd(6000, 8, 1.1, 16)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, mean_window=1024)
    for seed in (1, 2):
        b = W.normal_rhs(m.n, seed)
        xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    B = W.normal_rhs(m.n, 7, k=5)
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    G.gabp_solve_multi(s.handle, Bt, Xt, 1e-10, 10000)
    X = Xt.cpu().numpy()
    for k in range(B.shape[1]):
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, B[:, k], X[:, k]) < 1e-10 * np.abs(B[:, k]).max()
    b = W.normal_rhs(m.n, 3)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    s.close()


def test_autotuner_times_the_window_form(G):
    m = W.er_sdd(200000, 8, 1.1, 14)
    b = W.normal_rhs(m.n, 43)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, autotune=True)
    t = s.tuning()
    assert t["mean_window"] == 0 or 256 <= t["mean_window"] <= 24000
    print(f"autotuned mean form: window target {t['mean_window']}, {t['windows']} windows")
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    s.close()
    # colour-scheduled handles keep the tile form
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, autotune=True, schedule=1)
    assert s.tuning()["mean_window"] == 0
    s.close()
