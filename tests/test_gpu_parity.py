"""GPU parity of the CUDA library against the FP64 CPU oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * FP64 sweeps, per round: 1e-12 relative (infinity norm over each array of
    P_ij, mu_ij and x).  Both sides compute the same IEEE operations except
    for summation order and the eta = P mu storage form, i.e. a few ulps per
    round; 1e-12 leaves room for the growth of that over tens of rounds.
  * Solves: the FP64 residual ||b - A x||_inf, recomputed by the oracle, below
    tol (1e-10 relative, or absolute where the workload says so), and the
    error against the oracle's converged solution within the residual times
    the conditioning of the small test systems (1e-8 relative).
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


def _star_with_ring(n_leaves, seed):
    """A hub joined to every other node plus a ring: one row of degree
    n_leaves (runs warp-per-row) next to rows of degree 3."""
    rng = np.random.default_rng(seed)
    n = n_leaves + 1
    rows, cols, vals = [], [], []
    for k in range(1, n):
        w = rng.standard_normal() * 0.1
        rows += [0, k]; cols += [k, 0]; vals += [w, w]
        nxt = 1 + (k % n_leaves)
        if nxt != k:
            w2 = rng.standard_normal() * 0.3
            rows += [k, nxt]; cols += [nxt, k]; vals += [w2, w2]
    A = np.zeros((n, n))
    for r, c, v in zip(rows, cols, vals):
        A[r, c] += v
    A = (A + A.T) / 2
    np.fill_diagonal(A, 1.5 * np.abs(A).sum(1) + 0.5)
    return W.csr_from_dense(A)


PARITY_CASES = {
    "single_node": W.csr_from_dense(np.array([[3.0]])),
    "toy_tree": W.csr_from_dense(np.array([[1.0, -2.0, 3.0], [-2.0, 1.0, 0.0], [3.0, 0.0, 1.0]])),
    "poisson2d_p9": W.poisson2d(9),
    "poisson2d_p33": W.poisson2d(33),
    "poisson3d_p12": W.poisson3d(12),
    "er_4000": W.er_sdd(4000, 8, 1.1, 1),
    "er_ragged_isolated": W.er_sdd(3001, 3, 1.05, 2),
    "tree_400": W.random_tree(400, 5, diag_scale=1.0),
    "star_300_long_row": _star_with_ring(300, 3),
}


def _solver(G, m, **kw):
    return G.Solver.from_csr(m.row_ptr, m.col, m.val, **kw)


def _round_parity(G, m, b, rounds, **kw):
    s = _solver(G, m, **kw)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    worst = {}
    for r in rounds:
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r, want_messages=True)
        assert ref["status"] == "ok"
        G.gabp_run_rounds(s.handle, bt, r, xt)
        P, mu = G.gabp_get_messages(s.handle, m.nnz)
        for key, got, want in (("x", xt.cpu().numpy(), ref["x"]), ("P", P, ref["P"]),
                               ("mu", mu, ref["mu"])):
            e = _rel(got, want) if np.abs(want).max() > 0 else float(np.abs(got).max())
            worst[(key, r)] = e
    s.close()
    return worst


@pytest.mark.parametrize("name", sorted(PARITY_CASES))
def test_fp64_messages_match_oracle_every_round(G, name):
    m = PARITY_CASES[name]
    b = W.normal_rhs(m.n, 17)
    worst = _round_parity(G, m, b, (0, 1, 2, 3, 7, 15))
    bad = {k: v for k, v in worst.items() if v > 1e-12}
    assert not bad, bad


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_fp64_parity_for_every_group_width(G, lanes):
    m = W.er_sdd(2500, 9, 1.1, 4)
    b = W.uniform_rhs(m.n, 5)
    worst = _round_parity(G, m, b, (1, 4, 9), group_lanes=lanes)
    bad = {k: v for k, v in worst.items() if v > 1e-12}
    assert not bad, bad


def test_rev_given_equals_rev_computed(G):
    m = W.er_sdd(3000, 7, 1.1, 8)
    b = W.normal_rhs(m.n, 1)
    rev = W.reverse_index(m)
    s1 = _solver(G, m)
    s2 = G.Solver(G.gabp_create(m.row_ptr, m.col, m.val, rev), m.n, m.nnz)
    bt = torch.tensor(b, device="cuda")
    x1, x2 = torch.empty_like(bt), torch.empty_like(bt)
    G.gabp_run_rounds(s1.handle, bt, 6, x1)
    G.gabp_run_rounds(s2.handle, bt, 6, x2)
    assert torch.equal(x1, x2)


def _oracle_solution(m, b):
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=100000,
                      tol=1e-13)
    assert ref["status"] == "ok"
    return ref["x"]


SOLVE_CASES = {
    "er_20000": (W.er_sdd(20000, 8, 1.1, 11), "normal"),
    "poisson3d_p16": (W.poisson3d(16), "uniform"),
    "er_dom105_deg10": (W.er_sdd(20000, 10, 1.05, 12), "normal"),
}


def _rhs(m, kind, seed):
    return W.normal_rhs(m.n, seed) if kind == "normal" else W.uniform_rhs(m.n, seed)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(SOLVE_CASES))
def test_solve_reaches_relative_residual(G, name, precision):
    m, kind = SOLVE_CASES[name]
    b = _rhs(m, kind, 21)
    s = _solver(G, m, precision=precision)
    bt = torch.tensor(b, device="cuda")
    xt, iters = s.solve(bt, tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    res = oracle.residual_inf(m.row_ptr, m.col, m.val, b, x)
    assert res < 1e-10 * np.abs(b).max()
    assert _rel(x, _oracle_solution(m, b)) < 1e-8
    st = s.stats()
    assert st["sweeps_total"] == iters and st["status"] == 0
    if precision == 1:
        assert st["sweeps_mean"] > 0 and st["outer_steps"] >= 2
    s.close()


def test_config1_poisson2d_p32_absolute_residual(G):
    """2-D Poisson 32x32, b ~ U[-1,1], plain FP64 sweeps until
    ||Ax - b||_inf < 1e-10 (absolute)."""
    m = W.poisson2d(32)
    b = W.uniform_rhs(m.n, 0)
    s = _solver(G, m, precision=0, residual_kind=0)
    xt, iters = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_ABS, max_rounds=20000, tol=1e-10)
    # The GPU checks every few sweeps, so it stops at most check_every - 1
    # rounds after the oracle's first round that meets the rule.
    assert ref["rounds"] <= iters <= ref["rounds"] + 8
    s.close()


def test_mixed_precision_matches_fp64_oracle_poisson2d(G):
    m = W.poisson2d(32)
    b = W.uniform_rhs(m.n, 0)
    s = _solver(G, m, precision=1, residual_kind=0)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=50000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10
    assert _rel(x, _oracle_solution(m, b)) < 1e-8
    s.close()


def test_solve_host_matches_device(G):
    m = W.er_sdd(5000, 8, 1.1, 3)
    b = W.normal_rhs(m.n, 4)
    s = _solver(G, m, precision=1)
    xd, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10)
    xh, _ = G.gabp_solve_host(s.handle, b, 1e-10, 10000)
    assert np.array_equal(xd.cpu().numpy(), xh)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_rhs_matches_single_solves(G, precision):
    m = W.er_sdd(4000, 10, 1.05, 6)
    B = W.normal_rhs(m.n, 7, k=5)
    s = _solver(G, m, precision=precision)
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    G.gabp_solve_multi(s.handle, Bt, Xt, 1e-10, 10000)
    X = Xt.cpu().numpy()
    for k in range(B.shape[1]):
        res = oracle.residual_inf(m.row_ptr, m.col, m.val, B[:, k], X[:, k])
        assert res < 1e-10 * np.abs(B[:, k]).max()
    s.close()


def test_breakdown_is_reported(G):
    m = W.csr_from_dense(np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0]]))
    s = _solver(G, m, precision=0, check_every=1)
    with pytest.raises(G.GabpError) as ei:
        s.solve(torch.ones(3, dtype=torch.float64, device="cuda"), tol=1e-12, max_iter=50)
    assert ei.value.name == "GABP_ERR_BREAKDOWN"
    s.close()


def test_not_converged_keeps_last_iterate(G):
    m = W.poisson2d(20)
    b = W.uniform_rhs(m.n, 1)
    s = _solver(G, m, precision=0, check_every=1)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve(s.handle, bt, xt, 1e-10, 5)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=4)   # x of round 4 after 5 sweeps
    assert _rel(xt.cpu().numpy(), ref["x"]) < 1e-12
    s.close()


def test_dense_detection_system_diverges(G):
    """Dense A = S^T S + sigma^2 I of the detection workload: plain GaBP
    diverges (rho(|I - D^-1 A|) > 1); the solver says so instead of
    returning garbage."""
    sysd = W.detection_batch(1, 48, 48, 10.0, seed=3)[0]
    A, bb = sysd.dense_system()
    m = W.csr_from_dense(A)
    s = _solver(G, m, precision=0, check_every=1)
    with pytest.raises(G.GabpError) as ei:
        s.solve(torch.tensor(bb, device="cuda"), tol=1e-10, max_iter=2000)
    assert ei.value.name in ("GABP_ERR_DIVERGED", "GABP_ERR_BREAKDOWN")
    s.close()


def test_nondefault_stream(G):
    m = W.er_sdd(3000, 8, 1.1, 9)
    b = W.normal_rhs(m.n, 2)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s = _solver(G, m, precision=1)
        bt = torch.tensor(b, device="cuda")
        xt, _ = s.solve(bt, tol=1e-10)
    side.synchronize()
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    s.close()


# ---------------------------------------------------------------------------
# The benchmark's workload at full size: Erdos-Renyi n = 1,000,000, average
# degree 8, dominance 1.1, b ~ N(0,1), with the launch configuration the
# benchmark uses (automatic group width, mixed FP32 + FP64 refinement).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def er_full():
    m = W.er_sdd(1_000_000, 8, 1.1, 0)
    b = W.normal_rhs(m.n, 1)
    return m, b


def test_full_size_rounds_match_oracle(G, er_full):
    m, b = er_full
    worst = _round_parity(G, m, b, (3,))
    assert max(worst.values()) <= 1e-12, worst


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_solve(G, er_full, precision):
    m, b = er_full
    s = _solver(G, m, precision=precision)
    xt, iters = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=2000)
    x = xt.cpu().numpy()
    res = oracle.residual_inf(m.row_ptr, m.col, m.val, b, x)
    assert res < 1e-10 * np.abs(b).max()
    assert _rel(x, _oracle_solution(m, b)) < 1e-9
    s.close()


# ---------------------------------------------------------------------------
# Drivers and storage modes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_and_host_drivers_agree(G, precision):
    """The graph driver (one CUDA graph per solve) and the host driver
    (profile mode) run the same kernels and the same device-side decisions,
    so they give bit-identical solutions and sweep counts."""
    m = W.er_sdd(6000, 8, 1.1, 14)
    b = W.normal_rhs(m.n, 15)
    bt = torch.tensor(b, device="cuda")
    out = []
    for profile in (False, True):
        # small_form=1: the per-sweep path in both (the one-launch cluster
        # solve of small FP64 systems has no host-driven twin)
        s = _solver(G, m, precision=precision, profile=profile, small_form=1)
        xt, it = s.solve(bt, tol=1e-10, max_iter=5000)
        st = s.stats()
        out.append((xt.cpu().numpy(), it, st))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert out[1][2]["ms_full"] > 0 and out[1][2]["ms_residual"] > 0


def test_bf16_mean_storage_reaches_tolerance(G):
    """BF16 storage of the mean messages (FP32 arithmetic) inside FP64
    refinement still reaches 1e-10; it needs more refinement steps."""
    m = W.er_sdd(20000, 8, 1.1, 16)
    b = W.normal_rhs(m.n, 17)
    s32 = _solver(G, m, precision=1)
    s16 = _solver(G, m, precision=2)
    bt = torch.tensor(b, device="cuda")
    x32, _ = s32.solve(bt, tol=1e-10, max_iter=5000)
    x16, _ = s16.solve(bt, tol=1e-10, max_iter=5000)
    for xt in (x32, x16):
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert s16.stats()["outer_steps"] >= s32.stats()["outer_steps"]
    s32.close()
    s16.close()


def test_repeated_solves_reuse_the_graph(G):
    m = W.er_sdd(5000, 8, 1.1, 18)
    s = _solver(G, m, precision=1)
    for seed in range(3):
        b = W.normal_rhs(m.n, 30 + seed)
        xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10)
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    s.close()


# ---------------------------------------------------------------------------
# Multi right-hand sides: precisions once, all columns in one mean sweep
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 5, 40, 64, 100, 256])
def test_multi_rhs_widths(G, K):
    """K columns at once for every columns-per-lane width (1, 2, 4, 8 per lane);
    every column meets its own relative residual and matches the oracle."""
    m = W.er_sdd(3000, 10, 1.05, 40 + K)
    B = W.normal_rhs(m.n, 41, k=K)
    B[:, 0] *= 1e-3                      # columns of very different scale
    s = _solver(G, m, precision=1)
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    G.gabp_solve_multi(s.handle, Bt, Xt, 1e-10, 10000)
    X = Xt.cpu().numpy()
    st = s.stats()
    assert st["sweeps_full"] > 0 and st["sweeps_mean"] > 0
    for k in sorted({0, K // 2, K - 1}):
        res = oracle.residual_inf(m.row_ptr, m.col, m.val, B[:, k], X[:, k])
        assert res < 1e-10 * np.abs(B[:, k]).max(), (k, res)
        assert _rel(X[:, k], _oracle_solution(m, B[:, k])) < 1e-8
    s.close()


def test_multi_rhs_64_columns_dominance_105(G):
    """The multi right-hand-side workload's structure at reduced size: random
    SDD matrix, average degree 10, dominance 1.05, 64 columns b ~ N(0,1)."""
    m = W.er_sdd(50000, 10, 1.05, 3)
    B = W.normal_rhs(m.n, 4, k=64)
    s = _solver(G, m, precision=1)
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    G.gabp_solve_multi(s.handle, Bt, Xt, 1e-10, 10000)
    X = Xt.cpu().numpy()
    worst = max(oracle.residual_inf(m.row_ptr, m.col, m.val, B[:, k], X[:, k]) / np.abs(B[:, k]).max()
                for k in range(64))
    assert worst < 1e-10
    s.close()


# ---------------------------------------------------------------------------
# Batched independent systems and Section VII least-squares batches
# ---------------------------------------------------------------------------
def _block_diag(mats):
    rows, cols, vals, off = [], [], [], [0]
    for m in mats:
        r = np.repeat(np.arange(m.n), np.diff(m.row_ptr)) + off[-1]
        rows.append(r); cols.append(m.col.astype(np.int64) + off[-1]); vals.append(m.val)
        off.append(off[-1] + m.n)
    big = W.csr_from_coo(off[-1], np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return big, np.array(off)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_systems_each_meet_their_rule(G, precision):
    mats = [W.er_sdd(800, 8, 1.1, 1), W.poisson2d(12), W.random_tree(300, 2, diag_scale=2.0),
            W.er_sdd(1500, 5, 1.2, 3), W.poisson3d(6)]
    big, off = _block_diag(mats)
    scales = [1.0, 1e-6, 1e3, 1.0, 1e-2]    # very different magnitudes per system
    b = np.concatenate([sc * W.normal_rhs(m.n, 10 + k) for k, (m, sc) in enumerate(zip(mats, scales))])
    o = G.gabp_default_options()
    o.precision = precision
    o.stream = G.current_stream_handle()
    h = G.gabp_create_batched(off, big.row_ptr, big.col, big.val, o)
    s = G.Solver(h, big.n, big.nnz)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    for k, m in enumerate(mats):
        bs, xs = b[off[k]:off[k + 1]], x[off[k]:off[k + 1]]
        res = oracle.residual_inf(m.row_ptr, m.col, m.val, bs, xs)
        assert res < 1e-10 * np.abs(bs).max(), (k, res)
    s.close()


def test_lsq_batch_matches_closed_form_and_oracle(G):
    systems = W.detection_batch(24, 16, 64, 10.0, seed=7)
    o = G.gabp_default_options()
    o.precision = 1
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    it = G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
    got = xh.cpu().numpy()
    off = 0
    for d in systems:
        A, bb = d.dense_system()
        closed = np.linalg.solve(A, bb)
        assert _rel(got[off:off + d.K], closed) < 1e-8
        # the oracle's own augmentation and GaBP agree with the library
        rp, cl, vl, rhs = oracle.augment_lsq(d.S, d.sigma2, d.y)
        ref = oracle.gabp(rp, cl, vl, rhs, stop=oracle.STOP_RES_REL, max_rounds=20000, tol=1e-12)
        assert ref["status"] == "ok"
        assert _rel(got[off:off + d.K], ref["x"][:d.K]) < 1e-8
        off += d.K
    assert it > 0
    G.gabp_destroy(h)


def test_lsq_batch_many_tiles_per_cta(G):
    """Enough systems that every CTA walks many tiles of both kinds (rows of
    degree 2K > 64 make heavy tiles next to light ones): each system still
    matches its closed form.  Two systems of this batch make plain GaBP
    diverge (the oracle shows it), so the batch runs damped."""
    systems = W.detection_batch(300, 16, 80, 10.0, seed=11)
    o = G.gabp_default_options()
    o.precision = 1
    o.damping = 0.3
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
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


@pytest.mark.parametrize("precision", [0, 1])
def test_heavy_and_light_tiles_mixed(G, precision):
    """A graph with hub rows (degree 300) scattered among low-degree rows:
    heavy and light tiles interleave across every CTA's tile sequence."""
    rng = np.random.default_rng(5)
    n = 40000
    base = W.er_sdd(n, 4, 1.1, 6)
    rows = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = rows != base.col
    r, c, v = list(rows[keep]), list(base.col[keep].astype(np.int64)), list(base.val[keep])
    hubs = rng.choice(n, 60, replace=False)
    existing = set(zip(r, c))
    for hbi in hubs:
        for j in rng.choice(n, 300, replace=False):
            if j != hbi and (hbi, j) not in existing:
                w = 0.05 * rng.standard_normal()
                r += [hbi, j]; c += [j, hbi]; v += [w, w]
                existing.add((hbi, j)); existing.add((j, hbi))
    r, c, v = np.array(r), np.array(c), np.array(v)
    diag = 1.2 * np.bincount(r, np.abs(v), minlength=n) + 0.1
    m = W.csr_from_coo(n, np.concatenate([r, np.arange(n)]), np.concatenate([c, np.arange(n)]),
                       np.concatenate([v, diag]))
    b = W.normal_rhs(n, 7)
    s = _solver(G, m, precision=precision)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert _rel(x, _oracle_solution(m, b)) < 1e-8
    s.close()


@pytest.mark.parametrize("name", ["er_4000", "poisson2d_p33", "star_300_long_row"])
def test_fp64_damped_rounds_match_damped_oracle(G, name):
    m = PARITY_CASES[name]
    b = W.normal_rhs(m.n, 23)
    s = _solver(G, m, damping=0.4)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    for r in (1, 2, 6, 13):
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r, want_messages=True, damping=0.4)
        G.gabp_run_rounds(s.handle, bt, r, xt)
        P, mu = G.gabp_get_messages(s.handle, m.nnz)
        assert _rel(xt.cpu().numpy(), ref["x"]) <= 1e-12
        assert _rel(P, ref["P"]) <= 1e-12
        assert _rel(mu, ref["mu"]) <= 1e-12
    s.close()


def test_damped_solve_rescues_diverging_system(G):
    """Plain GaBP diverges on this augmented detection system; with damping
    the mixed solve reaches 1e-10 and the closed form."""
    sysd = W.detection_batch(300, 16, 80, 10.0, seed=11)[270]
    rp, cl, vl, rhs = oracle.augment_lsq(sysd.S, sysd.sigma2, sysd.y)
    m = W.CSR(len(rp) - 1, rp, cl, vl)
    plain = _solver(G, m, precision=1)
    with pytest.raises(G.GabpError):
        plain.solve(torch.tensor(rhs, device="cuda"), tol=1e-10, max_iter=3000)
    plain.close()
    for precision in (0, 1):
        s = _solver(G, m, precision=precision, damping=0.3)
        xt, _ = s.solve(torch.tensor(rhs, device="cuda"), tol=1e-10, max_iter=20000)
        A, bb = sysd.dense_system()
        assert _rel(xt.cpu().numpy()[:sysd.K], np.linalg.solve(A, bb)) < 1e-8
        s.close()
