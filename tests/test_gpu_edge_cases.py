"""GPU edge cases of the solve paths, each checked against the oracle or an
exact answer: a 1 x 1 system, empty rows (isolated nodes), a zero right-hand
side, a non-finite right-hand side, a budget of one sweep, and batches that
hold a single system."""
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


PATHS = [dict(precision=0), dict(precision=0, small_form=1), dict(precision=1), dict(precision=2)]


@pytest.mark.parametrize("kw", PATHS, ids=["fp64_cluster", "fp64_sweeps", "mixed", "bf16"])
def test_one_by_one_system(G, kw):
    m = W.csr_from_dense(np.array([[4.0]]))
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, **kw)
    xt, _ = s.solve(torch.tensor([2.0], dtype=torch.float64, device="cuda"), tol=1e-12, max_iter=100)
    assert abs(float(xt.cpu()[0]) - 0.5) < 1e-15
    s.close()


@pytest.mark.parametrize("kw", PATHS, ids=["fp64_cluster", "fp64_sweeps", "mixed", "bf16"])
def test_isolated_nodes(G, kw):
    """Rows with no off-diagonal entry (degree 0) next to connected ones."""
    A = np.diag([2.0, 3.0, 5.0, 7.0, 11.0])
    A[1, 3] = A[3, 1] = 0.5
    m = W.csr_from_dense(A)
    b = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, **kw)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-12, max_iter=1000)
    assert _rel(xt.cpu().numpy(), np.linalg.solve(A, b)) < 1e-12
    s.close()


@pytest.mark.parametrize("kw", PATHS, ids=["fp64_cluster", "fp64_sweeps", "mixed", "bf16"])
def test_zero_rhs_gives_zero(G, kw):
    m = W.poisson2d(9)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, residual_kind=G.RESIDUAL_ABS, **kw)
    xt, _ = s.solve(torch.zeros(m.n, dtype=torch.float64, device="cuda"), tol=1e-12, max_iter=100)
    assert float(xt.abs().max()) == 0.0
    s.close()


@pytest.mark.parametrize("kw", PATHS, ids=["fp64_cluster", "fp64_sweeps", "mixed", "bf16"])
def test_non_finite_rhs_is_reported(G, kw):
    m = W.poisson2d(6)
    b = np.ones(m.n)
    b[7] = np.nan
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, **kw)
    with pytest.raises(G.GabpError) as ei:
        s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=100)
    assert ei.value.name in ("GABP_ERR_INVALID_ARG", "GABP_ERR_DIVERGED", "GABP_ERR_BREAKDOWN")
    s.close()


@pytest.mark.parametrize("kw", PATHS[:2], ids=["fp64_cluster", "fp64_sweeps"])
def test_one_sweep_budget_returns_the_first_round(G, kw):
    """max_iter = 1: one round from zero messages, x_i = b_i / A_ii, and the
    status says the rule was not met."""
    m = W.er_sdd(500, 6, 1.2, 2)
    b = W.normal_rhs(m.n, 3)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, **kw)
    xt = torch.empty(m.n, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve(s.handle, torch.tensor(b, device="cuda"), xt, 1e-10, 1)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    assert s.stats()["sweeps_total"] == 1
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=0)["x"]
    assert _rel(xt.cpu().numpy(), ref) <= 1e-15
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batches_of_one_system(G, precision):
    m = W.er_sdd(3000, 8, 1.1, 5)
    b = W.normal_rhs(m.n, 6)
    o = G.gabp_default_options()
    o.precision = precision
    o.stream = G.current_stream_handle()
    h = G.gabp_create_batched(np.array([0, m.n]), m.row_ptr, m.col, m.val, o)
    s = G.Solver(h, m.n, m.nnz)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=5000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    s.close()
    d = W.detection_batch(1, 40, 40, 10.0, seed=3)[0]
    o2 = G.gabp_default_options()
    o2.precision = precision
    o2.stream = G.current_stream_handle()
    h2 = G.gabp_create_lsq_batched([d.S], [d.sigma2], o2)
    xh = torch.empty(d.K, dtype=torch.float64, device="cuda")
    G.gabp_solve_lsq_batched(h2, torch.tensor(d.y, device="cuda"), xh, 1e-10, 20000)
    A, bb = d.dense_system()
    assert _rel(xh.cpu().numpy(), np.linalg.solve(A, bb)) < 1e-8
    G.gabp_destroy(h2)
