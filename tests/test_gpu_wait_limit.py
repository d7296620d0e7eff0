"""Bounded device waits, through the C ABI: a wait that can never be satisfied
ends, surfaces as GABP_ERR_TIMEOUT through the controller the sweeps use, and
leaves the context usable -- no fault and no hang.

gabp_check_wait_limit polls a barrier that nothing completes (no copy is in
flight) for a given number of polls, then reports as a sweep whose staging
wait gave up.  The test then solves on the same handle.
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
    for polls in (1, 4096):
        status, per_poll = G.gabp_check_wait_limit(s.handle, polls)
        assert status == "GABP_ERR_TIMEOUT", status
        assert 0.0 <= per_poll < 1e-3, per_poll
    # the library's own limit (2^22 polls) in time on this device
    print(f"unsatisfied try_wait poll: {per_poll * 1e9:.0f} ns; 2^22 polls = {per_poll * 2**22:.2f} s")
    # the context and the handle are still usable
    xt, _ = s.solve(bt, tol=1e-10, max_iter=20000)
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, xt.cpu().numpy()) < 1e-10 * np.abs(b).max()
    assert s.stats()["status"] == 0
    s.close()


def test_wait_limit_check_validates_its_argument(G):
    m = W.poisson2d(4)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val)
    status, _ = G.gabp_check_wait_limit(s.handle, 0)
    assert status == "GABP_ERR_INVALID_ARG"
    s.close()
