"""Run-to-run determinism of the solves, through the C ABI.

Every sum in the sweeps has a fixed order -- segmented warp sums within a
32-slot chunk and the partials of rows that continue across chunks added in
chunk order (CSR heavy tiles), warp sums and per-warp column sums added in
warp order (dense Section VII kernels) -- so the same solve on the same
handle gives the same bits and the same sweep counts.  Each case runs the
solve twice and compares x with np.array_equal, and checks the result
against the oracle's converged solution (or the closed form) as the other
tests do: FP64 residual below 1e-10 relative, error below 1e-8 relative.
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
    n_leaves (it spans many 32-slot chunks of its tile) next to rows of
    degree 3."""
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


def _twice(G, s, bt):
    out = []
    for _ in range(2):
        xt, it = s.solve(bt, tol=1e-10, max_iter=50000)
        st = s.stats()
        out.append((xt.cpu().numpy(), it, st["sweeps_full"], st["sweeps_mean"], st["outer_steps"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:], (out[0][1:], out[1][1:])
    return out[0][0]


CSR_CASES = {
    # heavy_degree 4 turns every tile of a degree-8 graph into a slot-parallel tile
    "er_heavy_tiles": (W.er_sdd(20000, 8, 1.1, 31), 4),
    "hub_900": (_hub_with_ring(900, 7), 64),
}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name", sorted(CSR_CASES))
def test_csr_tile_solves_are_deterministic(G, name, prec):
    m, heavy = CSR_CASES[name]
    precision = G.PREC_MIXED_FP32 if prec == "fp32" else G.PREC_MIXED_BF16
    b = W.normal_rhs(m.n, 32)
    s = G.Solver.from_csr(m.row_ptr, m.col, m.val, precision=precision, heavy_degree=heavy,
                          mean_window=-1, pull_lanes=-1)
    x = _twice(G, s, torch.tensor(b, device="cuda"))
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10 * np.abs(b).max()
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=100000,
                      tol=1e-13)["x"]
    assert _rel(x, ref) < 1e-8
    s.close()


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_dense_lsq_solves_are_deterministic(G, precision, schedule):
    """Section VII batches in the dense bipartite form, K from 16 to 256 (one
    to eight column chunks per lane), FP64 and FP32 messages."""
    systems = W.detection_batch(24, 16, 256, 10.0, seed=9)
    o = G.gabp_default_options()
    o.precision = precision
    o.schedule = schedule
    o.damping = 0.3 if schedule == 0 else 0.2
    o.damp_scope = 1 if schedule == 1 else 0
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(2):
        it = G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 50000)
        st = G.gabp_get_stats(h)
        runs.append((xh.cpu().numpy(), it, st["sweeps_full"], st["sweeps_mean"], st["outer_steps"]))
    G.gabp_destroy(h)
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1:] == runs[1][1:]
    got, off = runs[0][0], 0
    for d in systems:
        A, bb = d.dense_system()
        closed = np.linalg.solve(A, bb)
        assert _rel(got[off:off + d.K], closed) < 1e-8
        off += d.K
