"""GPU parity of the colour-serial schedule (option schedule = 1).

The library colours the graph greedily in the caller's row order and runs
every sweep as one in-place pass per colour class.  Nodes of a class are not
adjacent, so this is the serial schedule of Section III-C with the nodes
visited class by class: the oracle's gabp_serial with the order that sorts
nodes by colour (the same greedy rule: oracle.greedy_colouring).  FP64
rounds are compared with it per round (messages and means, 1e-12 relative,
the synchronous tolerance); solves are compared with the oracle's converged
solution and must need fewer sweeps than the synchronous schedule.
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


def _order(m):
    return np.argsort(oracle.greedy_colouring(m.row_ptr, m.col), kind="stable")


def _star(n_leaves, seed):
    rng = np.random.default_rng(seed)
    n = n_leaves + 1
    A = np.zeros((n, n))
    for k in range(1, n):
        A[0, k] = A[k, 0] = 0.1 * rng.standard_normal()
        nxt = 1 + (k % n_leaves)
        if nxt != k:
            A[k, nxt] = A[nxt, k] = 0.3 * rng.standard_normal()
    np.fill_diagonal(A, 1.5 * np.abs(A).sum(1) + 0.5)
    return W.csr_from_dense(A)


CASES = {
    "er_4000": lambda: W.er_sdd(4000, 8, 1.1, 1),
    "er_ragged_isolated": lambda: W.er_sdd(3001, 3, 1.05, 2),
    "poisson2d_33": lambda: W.poisson2d(33),
    "poisson3d_9": lambda: W.poisson3d(9),
    # diag_scale 3: at 1.5 a one-ulp change of A already moves round 2 of the
    # serial schedule by 8e-12 (an intermediate precision near 6e-4), so the
    # 1e-12 bound would test the case's conditioning, not the kernels
    "tree_700": lambda: W.random_tree(700, 3, diag_scale=3.0),
    "star_1500_long_row": lambda: _star(1500, 4),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("damping", [0.0, 0.4])
def test_colour_rounds_match_serial_oracle(G, name, damping):
    m = CASES[name]()
    b = W.normal_rhs(m.n, 5)
    order = _order(m)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, schedule=1, damping=damping)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    for r in (0, 1, 2, 5, 9):
        G.gabp_run_rounds(s.handle, bt, r, xt)
        ref = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, order=order, max_rounds=r,
                                 want_messages=True, damping=damping)
        P, mu = G.gabp_get_messages(s.handle, m.nnz)
        assert _rel(xt.cpu().numpy(), ref["x"]) <= 1e-12, ("x", r)
        if r > 0:
            assert _rel(P, ref["P"]) <= 1e-12, ("P", r)
            assert _rel(mu, ref["mu"]) <= 1e-12, ("mu", r)
    s.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("name,make", [("poisson2d_48", lambda: W.poisson2d(48)),
                                       ("poisson3d_16", lambda: W.poisson3d(16)),
                                       ("er_20000", lambda: W.er_sdd(20000, 8, 1.1, 16))])
def test_colour_solves_need_fewer_sweeps(G, precision, name, make):
    m = make()
    b = W.uniform_rhs(m.n, 4)
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=200000,
                      tol=1e-13)
    bt = torch.tensor(b, device="cuda")
    sweeps = {}
    for sched in (0, 1):
        s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, schedule=sched,
                              small_form=1)
        xt, it = s.solve(bt, tol=1e-10, max_iter=200000)
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
        assert _rel(x, ref["x"]) < 1e-8
        sweeps[sched] = it
        s.close()
    if precision != 2:   # BF16 storage: the refinement, not the schedule, sets the count
        assert sweeps[1] < sweeps[0], sweeps


def test_colour_schedule_is_refused_for_batches(G):
    m = W.poisson2d(5)
    o = G.gabp_default_options()
    o.schedule = 1
    with pytest.raises(G.GabpError):
        G.gabp_create_batched(np.array([0, m.n]), m.row_ptr, m.col, m.val, o)
    d = W.detection_batch(1, 8, 8, 10.0, seed=1)[0]
    with pytest.raises(G.GabpError):
        G.gabp_create_lsq_batched([d.S], [d.sigma2], o)
