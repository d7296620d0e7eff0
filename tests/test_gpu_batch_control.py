"""Per-system control of dense Section VII batches, through the C ABI.

With gabp_options.batch_control = 0 every rule of the solve -- the precision
freeze, the end of each inner solve, the scale of the refinement, the stop
rule -- reads only the numbers of one system, and a system that meets the
stop rule leaves the sweeps.  So each system must

* meet its own stop rule and match its closed form (S^T S + psi I)^-1 S^T y,
* take exactly the sweeps it takes when solved alone (a batch of one), with
  the same bits of x^,

and the batch must sweep fewer grid positions than with one controller for
the whole batch (batch_control = 1), whose count is sweeps x positions.
"""
import numpy as np
import pytest

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


def _mixed_batch():
    """Systems of unequal difficulty: high and low SNR, spread 2 and the
    harder square case (N = K), K from 8 to 200."""
    return (W.detection_batch(6, 8, 200, 20.0, seed=41) + W.detection_batch(6, 8, 200, 0.0, seed=42)
            + W.detection_batch(4, 16, 96, 10.0, seed=43, spread=1)
            + W.detection_batch(4, 100, 200, 3.0, seed=44))


def _opts(G, precision, schedule, batch_control):
    o = G.gabp_default_options()
    o.precision = precision
    o.schedule = schedule
    if schedule == 1:
        o.damping, o.damp_scope = 0.2, 1
    o.batch_control = batch_control
    o.stream = G.current_stream_handle()
    return o


def _solve(G, systems, o, tol=1e-10, max_iter=50000):
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    G.gabp_solve_lsq_batched(h, y, xh, tol, max_iter)
    st = G.gabp_get_stats(h)
    sw = G.gabp_get_system_sweeps(h, len(systems))
    G.gabp_destroy(h)
    return xh.cpu().numpy(), st, sw


def _split(x, systems):
    out, off = [], 0
    for d in systems:
        out.append(x[off:off + d.K])
        off += d.K
    return out


CASES = [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)]   # (precision, schedule)


@pytest.mark.parametrize("precision,schedule", CASES)
def test_each_system_meets_its_rule_and_its_closed_form(G, precision, schedule):
    systems = _mixed_batch()
    x, st, sw = _solve(G, systems, _opts(G, precision, schedule, 0))
    assert st["status"] == 0
    for d, xs, k in zip(systems, _split(x, systems), sw):
        A, b = d.dense_system()
        closed = np.linalg.solve(A, b)
        assert np.abs(xs - closed).max() <= 1e-8 * np.abs(closed).max()
        assert 0 < k <= st["sweeps_total"]
    # systems leave at different sweeps
    assert len(set(sw.tolist())) > 1


@pytest.mark.parametrize("precision,schedule", CASES)
def test_a_system_sweeps_as_it_does_alone(G, precision, schedule):
    systems = _mixed_batch()
    o = _opts(G, precision, schedule, 0)
    x, _, sw = _solve(G, systems, o)
    xs = _split(x, systems)
    for s in (0, 3, 7, 11, 13, 19):   # both SNRs, both spreads, small and large K
        xa, sta, swa = _solve(G, [systems[s]], o)
        assert swa[0] == sta["sweeps_total"]
        assert sw[s] == sta["sweeps_total"], (s, sw[s], sta["sweeps_total"])
        assert np.array_equal(xs[s], xa), s


@pytest.mark.parametrize("precision,schedule", [(0, 0), (1, 0), (2, 1)])
def test_per_system_control_sweeps_fewer_positions(G, precision, schedule):
    systems = _mixed_batch()
    pairs = sum(d.S.size for d in systems)
    x0, st0, sw0 = _solve(G, systems, _opts(G, precision, schedule, 0))
    x1, st1, sw1 = _solve(G, systems, _opts(G, precision, schedule, 1))
    assert st1["positions_swept"] == st1["sweeps_total"] * pairs
    assert np.all(sw1 == st1["sweeps_total"])
    # per system: the positions are each system's own sweeps, less the grid
    # passes skipped when an inner solve ends
    own = sum(int(k) * d.S.size for k, d in zip(sw0, systems))
    assert st0["positions_swept"] <= own
    assert st0["positions_swept"] < st1["positions_swept"]
    for d, a, b in zip(systems, _split(x0, systems), _split(x1, systems)):
        A, bb = d.dense_system()
        closed = np.linalg.solve(A, bb)
        scale = np.abs(closed).max()
        assert np.abs(a - closed).max() <= 1e-8 * scale
        assert np.abs(b - closed).max() <= 1e-8 * scale


def test_repeated_solves_reset_the_per_system_state(G):
    """Two solves on one handle give the same bits and the same sweeps."""
    systems = _mixed_batch()
    o = _opts(G, 1, 0, 0)
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(2):
        G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 50000)
        runs.append((xh.cpu().numpy(), G.gabp_get_system_sweeps(h, len(systems)),
                     G.gabp_get_stats(h)["positions_swept"]))
    with pytest.raises(G.GabpError):
        G.gabp_get_system_sweeps(h, len(systems) + 1)
    G.gabp_destroy(h)
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]


def test_host_driven_solve_matches_the_graph(G):
    """The host driver (profile mode) runs the same per-system rules."""
    systems = _mixed_batch()
    o = _opts(G, 1, 0, 0)
    xg, stg, swg = _solve(G, systems, o)
    o.profile = 1
    xp, stp, swp = _solve(G, systems, o)
    assert np.array_equal(xg, xp)
    assert np.array_equal(swg, swp)
    assert stg["positions_swept"] == stp["positions_swept"]


@pytest.mark.parametrize("precision", [0, 1])
def test_max_iter_ends_the_batch_cleanly(G, precision):
    """A sweep budget below what the slowest systems need: the solve ends
    GABP_ERR_NOT_CONVERGED at max_iter sweeps, the handle stays usable, and
    a full solve on it afterwards meets every closed form."""
    systems = _mixed_batch()
    o = _opts(G, precision, 0, 0)
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 12)
    assert ei.value.name == "GABP_ERR_NOT_CONVERGED"
    st = G.gabp_get_stats(h)
    assert st["sweeps_total"] == 12
    assert np.all(G.gabp_get_system_sweeps(h, len(systems)) <= 12)
    G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 50000)
    for d, xs in zip(systems, _split(xh.cpu().numpy(), systems)):
        A, b = d.dense_system()
        closed = np.linalg.solve(A, b)
        assert np.abs(xs - closed).max() <= 1e-8 * np.abs(closed).max()
    G.gabp_destroy(h)
