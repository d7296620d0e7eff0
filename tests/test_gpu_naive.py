"""Algorithm 1 (the naive form) on the GPU, option naive = 1, through the C ABI.

Every cavity sum P_{i\\j} = A_ii + sum_{k != j} P_ki and its information part is
added up over the other incoming messages directly, instead of node total
minus reverse message (Algorithm 2).  It is the same round computed without
that cancellation, so it cross-checks the broadcast kernels.

Tolerances (written here, derived from the arithmetic): per round 1e-12
relative (infinity norm over each array of P_ij, mu_ij and x) against the
oracle's Algorithm 1 and against the GPU's Algorithm 2, as for the FP64
parity tests: both sides compute the same IEEE operations up to the
summation order and the eta = P mu storage form, a few ulps per round.
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


CASES = {
    "toy_tree": W.csr_from_dense(np.array([[1.0, -2.0, 3.0], [-2.0, 1.0, 0.0], [3.0, 0.0, 1.0]])),
    "poisson2d_p9": W.poisson2d(9),
    "er_4000": W.er_sdd(4000, 8, 1.1, 1),
    "er_ragged_isolated": W.er_sdd(3001, 3, 1.05, 2),
    "tree_indefinite_300": W.random_tree(300, 2, diag_scale=2.0),
    "hub_300": _hub_with_ring(300, 3),
}


def _rounds(G, m, b, rounds, naive):
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_FP64, naive=naive)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    out = {}
    for r in rounds:
        G.gabp_run_rounds(s.handle, bt, r, xt)
        P, mu = G.gabp_get_messages(s.handle, m.nnz)
        out[r] = (xt.cpu().numpy(), P, mu)
    s.close()
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_naive_rounds_match_the_oracle_and_the_broadcast_form(G, name):
    m = CASES[name]
    b = W.normal_rhs(m.n, 7)
    rounds = (1, 2, 5, 9)
    naive = _rounds(G, m, b, rounds, 1)
    bcast = _rounds(G, m, b, rounds, 0)
    for r in rounds:
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b, variant=oracle.NAIVE, max_rounds=r,
                          want_messages=True)
        assert ref["status"] == "ok"
        for k, want in enumerate((ref["x"], ref["P"], ref["mu"])):
            assert _rel(naive[r][k], want) <= 1e-12, (r, k)
            assert _rel(naive[r][k], bcast[r][k]) <= 1e-12, (r, k)


def test_naive_fp64_solve(G):
    m = W.er_sdd(20000, 8, 1.1, 11)
    b = W.normal_rhs(m.n, 3)
    bt = torch.tensor(b, device="cuda")
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_FP64, naive=1)
    assert s.tuning()["cluster_ctas"] == 0          # never the one-launch cluster solve
    x, iters = s.solve(bt, tol=1e-10, max_iter=5000)
    s.close()
    t = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=G.PREC_FP64)
    xb, iters_b = t.solve(bt, tol=1e-10, max_iter=5000)
    t.close()
    x, xb = x.cpu().numpy(), xb.cpu().numpy()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    assert iters == iters_b
    assert _rel(x, xb) < 1e-12
