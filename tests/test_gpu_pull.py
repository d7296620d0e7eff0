"""In-place form of the FP32 full sweep (option pull_lanes > 0), through the C ABI.

The message j -> i of round t depends only on the totals of j at round t - 1
and on the reverse message i -> j of round t - 1, which in turn depends only
on the totals of i at round t - 2 and on the message j -> i of round t - 2
(Alg. 2, Section III-C).  The in-place form therefore recomputes the reverse
message in every slot and overwrites the slot with the new round, so its
launch t yields the round-t tentative means, where the scatter form's launch t
yields round t - 1.

Tolerances (written here, derived from the arithmetic):
  * round means after k <= 4 FP32 full sweeps against the FP64 oracle's:
    1e-5 relative (infinity norm).  Each message carries a few FP32 ulps
    (6e-8) of rounding per round and a mean is a ratio of sums of a row's
    messages, so k rounds stay near 1e-6; consecutive rounds differ by far
    more than 1e-4 on these systems in rounds 1..4 (checked), so a wrong
    round fails.  (A float32 replay of the rounds on the CPU stays within
    1e-6 of the oracle on every case here.)
  * solves: the FP64 residual, recomputed by the oracle, below 1e-10
    relative, and the error against the oracle's converged solution below
    1e-8 relative, as for the scatter form.
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


ROUND_CASES = {
    "poisson2d_p20": W.poisson2d(20),
    "er_3000": W.er_sdd(3000, 8, 1.1, 5),
    "er_ragged_isolated": W.er_sdd(3001, 3, 1.05, 2),
    "tree_400": W.random_tree(400, 5, diag_scale=3.0),    # well conditioned: FP32 rounds within 2e-7
    "hub_300": _hub_with_ring(300, 3),
}


def _means_after(G, s, bt, k):
    """x after a mixed solve stopped by max_iter = k during the first inner
    solve: ||b||_inf times the FP32 tentative means of the last sweep."""
    xt = torch.zeros_like(bt)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve(s.handle, bt, xt, 1e-14, k)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    return xt.cpu().numpy()


@pytest.mark.parametrize("lanes", [-1, 2, 8, 32])
@pytest.mark.parametrize("name", sorted(ROUND_CASES))
def test_full_sweep_rounds_match_oracle_means(G, name, lanes):
    m = ROUND_CASES[name]
    b = W.normal_rhs(m.n, 31)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, pull_lanes=lanes)
    assert s.tuning()["pull_lanes"] == max(lanes, 0)
    bt = torch.tensor(b, device="cuda")
    lag = 1 if lanes < 0 else 0          # the scatter form reports the previous round
    for k in (1, 2, 3, 4):
        got = _means_after(G, s, bt, k)
        want = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED,
                           max_rounds=k - lag)["x"]
        other = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED,
                            max_rounds=k + 1 - lag)["x"]
        err = _rel(got, want)
        assert err <= 1e-5, (k, err)
        if k <= 3:                           # the check tells neighbouring rounds apart
            assert _rel(other, want) > 1e-4, k
    s.close()


def test_rounds_stay_on_the_oracle_on_an_indefinite_tree(G):
    """A tree whose matrix is indefinite (smallest eigenvalue -0.67) and not
    walk-summable: some edges have A_ij^2 > P_{i\\j} P_{j\\i}.  Each message of
    the in-place form is computed by its receiver and recomputed by its
    sender; unless the two copies agree bit for bit, their difference grows
    along such an edge by that ratio squared every two rounds.  A float32
    replay on the CPU of the kernel's arithmetic stays within 1.5e-5 of the
    oracle for 40 rounds; with the recomputed product left unrounded (a fused
    multiply-add) it leaves 1e-4 at round 7 and reaches 1e2 by round 11."""
    m = W.random_tree(300, 2, diag_scale=2.0)
    b = 1e3 * W.normal_rhs(m.n, 12)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, pull_lanes=8)
    bt = torch.tensor(b, device="cuda")
    for k in range(1, 13):
        want = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED, max_rounds=k)["x"]
        err = _rel(_means_after(G, s, bt, k), want)
        assert err <= 1e-4, (k, err)
    s.close()


def _oracle_solution(m, b):
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=100000,
                      tol=1e-13)
    assert ref["status"] == "ok"
    return ref["x"]


SOLVE_CASES = {
    "er_20000": W.er_sdd(20000, 8, 1.1, 11),
    "er_dom105_deg10": W.er_sdd(20000, 10, 1.05, 12),
    "poisson3d_p16": W.poisson3d(16),
    "hub_300": _hub_with_ring(300, 4),
    "tree_indefinite_300": W.random_tree(300, 2, diag_scale=2.0),
}


@pytest.mark.parametrize("lanes", [4, 8, 32])
@pytest.mark.parametrize("name", sorted(SOLVE_CASES))
def test_mixed_solve_in_place_form(G, name, lanes):
    m = SOLVE_CASES[name]
    b = W.normal_rhs(m.n, 41)
    bt = torch.tensor(b, device="cuda")
    sweeps = {}
    for form in (-1, lanes):
        s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, pull_lanes=form)
        xt, iters = s.solve(bt, tol=1e-10, max_iter=50000)
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
        assert _rel(x, _oracle_solution(m, b)) < 1e-8
        st = s.stats()
        assert st["status"] == 0 and st["sweeps_mean"] > 0
        sweeps[form] = iters
        s.close()
    # same rounds, one launch ahead: the counts differ by the rounding of the stop rules only
    assert abs(sweeps[lanes] - sweeps[-1]) <= max(3, sweeps[-1] // 5), sweeps


def test_bf16_mean_storage_in_place_form(G):
    m = W.er_sdd(20000, 8, 1.1, 13)
    b = W.normal_rhs(m.n, 42)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_BF16, pull_lanes=8)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=50000)
    x = xt.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    s.close()


def test_batched_systems_in_place_form(G):
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
    o.pull_lanes = 8
    o.stream = G.current_stream_handle()
    h = G.gabp_create_batched(np.array(off, dtype=np.int64), big.row_ptr, big.col, big.val, o)
    s = G.Solver(h, big.n, big.nnz)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    x = xt.cpu().numpy()
    for k, m in enumerate(mats):
        bs, xs = b[off[k]:off[k + 1]], x[off[k]:off[k + 1]]
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, bs, xs) < 1e-10 * np.abs(bs).max(), k
    s.close()


def test_multi_rhs_precisions_in_place_form(G):
    """The multi-RHS solve converges the precisions with the FP32 full sweep
    (zero right-hand side), then runs the K-column mean sweeps."""
    m = W.er_sdd(4000, 10, 1.05, 6)
    B = W.normal_rhs(m.n, 7, k=5)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, pull_lanes=8)
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    G.gabp_solve_multi(s.handle, Bt, Xt, 1e-10, 10000)
    X = Xt.cpu().numpy()
    for k in range(B.shape[1]):
        res = oracle.residual_inf(m.row_ptr, m.col, m.val, B[:, k], X[:, k])
        assert res < 1e-10 * np.abs(B[:, k]).max(), k
    s.close()


def test_autotuner_picks_a_form_and_solves(G):
    m = W.er_sdd(200000, 8, 1.1, 14)
    b = W.normal_rhs(m.n, 43)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, autotune=True)
    assert s.tuning()["pull_lanes"] in (0, 2, 4, 8, 16, 32)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=20000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    s.close()
    # damped and colour-scheduled handles keep the scatter form
    for kw in ({"damping": 0.2}, {"schedule": 1}):
        s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_MIXED_FP32, autotune=True, **kw)
        assert s.tuning()["pull_lanes"] == 0, kw
        s.close()
