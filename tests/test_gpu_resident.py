"""GPU parity of the one-launch FP64 solve of small systems.

Systems whose messages fit the shared memory of one thread-block cluster are
solved by a single kernel: the rows are split over 2..16 CTAs, messages go
straight into the owning CTA's shared memory, and the residual check and the
stop decision happen inside the cluster.  Its arithmetic per message is that
of the per-sweep FP64 kernels, so the solves are checked against the CPU
oracle (1e-10 residual, 1e-8 error against the converged oracle solution,
the tolerances of test_gpu_parity) and against the per-sweep path
(small_form = 1), whose sweep count they match.
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


CASES = {
    "poisson2d_32": (lambda: W.poisson2d(32), "abs"),
    "er_2000": (lambda: W.er_sdd(2000, 8, 1.1, 3), "rel"),
    "tree_3000": (lambda: W.random_tree(3000, 5, diag_scale=1.5), "rel"),
    "ragged_er_777": (lambda: W.er_sdd(777, 3, 1.05, 8), "rel"),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ctas", [2, 4, 8, 16])
def test_resident_solve_matches_oracle_and_sweep_path(G, name, ctas):
    make, kind = CASES[name]
    m = make()
    b = W.uniform_rhs(m.n, 1)
    rk = G.RESIDUAL_ABS if kind == "abs" else G.RESIDUAL_REL
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b,
                      stop=oracle.STOP_RES_ABS if kind == "abs" else oracle.STOP_RES_REL,
                      max_rounds=100000, tol=1e-12)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=rk, cluster_ctas=ctas)
    t = s.tuning()
    if t["cluster_ctas"] == 0:
        pytest.skip("system does not fit a cluster of this size")
    assert t["cluster_ctas"] == ctas
    bt = torch.tensor(b, device="cuda")
    xt, it = s.solve(bt, tol=1e-10, max_iter=100000)
    st = s.stats()
    assert st["kernel_launches"] == 1
    x = xt.cpu().numpy()
    res = oracle.residual_inf(m.row_ptr, m.col, m.val, b, x)
    assert res < (1e-10 if kind == "abs" else 1e-10 * np.abs(b).max())
    assert _rel(x, ref["x"]) < 1e-8
    # the per-sweep path: same sweeps, same x to rounding
    p = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=rk, small_form=1)
    assert p.tuning()["cluster_ctas"] == 0
    xp, itp = p.solve(bt, tol=1e-10, max_iter=100000)
    assert it == itp
    assert _rel(x, xp.cpu().numpy()) < 1e-12
    s.close()
    p.close()


def test_resident_not_converged_and_damped(G):
    m = W.poisson2d(20)
    b = W.uniform_rhs(m.n, 2)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=G.RESIDUAL_ABS)
    assert s.tuning()["cluster_ctas"] > 0
    with pytest.raises(G.GabpError) as ei:
        s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=10)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    assert s.stats()["sweeps_total"] == 10
    s.close()
    d = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=G.RESIDUAL_ABS,
                          damping=0.3)
    xt, _ = d.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=100000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10
    d.close()


def test_resident_autotune_picks_a_cluster(G):
    m = W.poisson2d(32)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=G.RESIDUAL_ABS,
                          autotune=True)
    t = s.tuning()
    assert t["tuned"] == 1 and t["cluster_ctas"] in {2, 4, 8, 16}
    b = W.uniform_rhs(m.n, 0)
    xt, _ = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=100000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10
    s.close()
