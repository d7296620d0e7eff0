"""GPU parity of Aitken's Delta^2 on the tentative means (Section IV-A,
convergence acceleration), option `aitken` = stride s.

* gabp_run_rounds with aitken = s returns the Delta^2 of the means of rounds
  R - 2s, R - s and R: compared with oracle.gabp_aitken.  The FP64 means of
  each round agree to the 1e-12 per-round tolerance; the formula amplifies a
  perturbation delta of its inputs to at most delta (1 + 4 r + 4 r^2) with
  r = max |x1 - x0| / |x2 - 2 x1 + x0|, so that is the tolerance here, with r
  taken from the oracle's iterates.
* Solves with aitken = 2 (one-launch cluster path and per-sweep path) reach
  the residual rule, match the oracle's converged solution, and stop in
  fewer sweeps than without.
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
    "poisson2d_20": lambda: W.poisson2d(20),
    "er_3000": lambda: W.er_sdd(3000, 8, 1.1, 5),
    "poisson3d_9": lambda: W.poisson3d(9),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("stride", [1, 2, 3])
def test_rounds_with_aitken_match_oracle(G, name, stride):
    m = CASES[name]()
    b = W.uniform_rhs(m.n, 7)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, aitken=stride)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    for R in (2 * stride, 2 * stride + 1, 9, 16):
        G.gabp_run_rounds(s.handle, bt, R, xt)
        ref = oracle.gabp_aitken(m.row_ptr, m.col, m.val, b, R, stride)
        xs = [oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r)["x"]
              for r in (R - 2 * stride, R - stride, R)]
        d1, den = xs[1] - xs[0], (xs[2] - xs[1]) - (xs[1] - xs[0])
        scale = np.maximum(np.maximum(np.abs(xs[0]), np.abs(xs[1])), np.abs(xs[2]))
        ok = np.abs(den) > 64 * np.finfo(float).eps * scale
        r = float(np.max(np.abs(d1[ok]) / np.abs(den[ok]))) if ok.any() else 0.0
        tol = 1e-12 * (1 + 4 * r + 4 * r * r)
        assert _rel(xt.cpu().numpy(), ref) <= tol, (R, r)
    s.close()


@pytest.mark.parametrize("small_form", [0, 1])
def test_aitken_solve_converges_in_fewer_sweeps(G, small_form):
    m = W.poisson2d(32)
    b = W.uniform_rhs(m.n, 0)
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_ABS, max_rounds=100000,
                      tol=1e-12)
    bt = torch.tensor(b, device="cuda")
    out = {}
    for ait in (0, 2):
        s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, residual_kind=G.RESIDUAL_ABS,
                              small_form=small_form, aitken=ait)
        assert (s.tuning()["cluster_ctas"] > 0) == (small_form == 0)
        xt, it = s.solve(bt, tol=1e-10, max_iter=100000)
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10
        assert _rel(x, ref["x"]) < 1e-8
        out[ait] = it
        s.close()
    assert out[2] <= 0.6 * out[0], out


def test_aitken_solve_3d_relative_rule(G):
    m = W.poisson3d(14)
    b = W.uniform_rhs(m.n, 2)
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=100000,
                      tol=1e-13)
    for small_form in (0, 1):
        s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=0, small_form=small_form, aitken=2)
        xt, it = s.solve(torch.tensor(b, device="cuda"), tol=1e-10, max_iter=100000)
        x = xt.cpu().numpy()
        assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
        assert _rel(x, ref["x"]) < 1e-8
        s.close()
