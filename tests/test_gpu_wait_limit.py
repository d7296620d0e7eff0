"""Bounded device waits, through the C ABI: a wait that can never be satisfied
ends, surfaces as GABP_ERR_TIMEOUT through the controller the sweeps use, and
leaves the context usable -- no fault and no hang.

gabp_check_wait_limit runs the sweeps' own time-bounded wait on a barrier
that nothing completes (no copy is in flight), for a given time up to the
library's limit of 100 ms, then reports as a sweep whose staging wait gave
up.  The test then solves on the same handle.
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


@pytest.mark.parametrize("precision", [0, 1])
def test_unsatisfied_wait_reports_timeout_and_the_handle_still_solves(G, precision):
    m = W.er_sdd(3000, 8, 1.1, 4)
    b = W.normal_rhs(m.n, 5)
    bt = torch.tensor(b, device="cuda")
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision)
    for limit_us, lo, hi in ((10, 10e-6, 5e-3), (2000, 2e-3, 20e-3), (0, 0.1, 0.2)):
        status, waited = G.gabp_check_wait_limit(s.handle, limit_us)
        assert status == "GABP_ERR_TIMEOUT", status
        # the wait ends once its limit has passed, and not long after
        assert lo <= waited < hi, (limit_us, waited)
    # the context and the handle are still usable
    xt, _ = s.solve(bt, tol=1e-10, max_iter=20000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    assert s.stats()["status"] == 0
    s.close()


def test_wait_limit_check_validates_its_argument(G):
    m = W.poisson2d(4)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val)
    for bad in (-1, 100001, 2**31 - 1):
        status, _ = G.gabp_check_wait_limit(s.handle, bad)
        assert status == "GABP_ERR_INVALID_ARG", bad
    s.close()
