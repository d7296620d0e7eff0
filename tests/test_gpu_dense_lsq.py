"""GPU parity of the dense bipartite form of Section VII batches.

gabp_create_lsq_batched keeps every augmented system
[[I_K, S^T], [S, -psi I]] as an N x K grid of message pairs when K_s <= 256
and N_s <= 1024 (options.lsq_form = 0).  The FP64 rounds are compared with the
CPU oracle run on the same augmented systems written out as CSR
(oracle.augment_lsq, block-diagonal), to the 1e-12 per-round tolerance of the
CSR kernels; the solves with the closed form (S^T S + psi I)^{-1} S^T y and
with the general CSR path of the library.
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


def _systems(shapes, seed, zero_frac=0.0):
    """S_s of the given (N, K) with +-1/sqrt(N) entries (a fraction set to 0),
    psi_s, y_s."""
    rng = np.random.default_rng(seed)
    out = []
    for N, K in shapes:
        S = rng.choice([-1.0, 1.0], size=(N, K)) / np.sqrt(N)
        if zero_frac > 0:
            S[rng.random((N, K)) < zero_frac] = 0.0
        psi = float(rng.uniform(0.05, 0.5))
        y = rng.standard_normal(N)
        out.append((S, psi, y))
    return out


def _augmented_block_diag(systems):
    rows, cols, vals, rhs, off = [], [], [], [], [0]
    for S, psi, y in systems:
        rp, cl, vl, b = oracle.augment_lsq(S, psi, y)
        n = len(rp) - 1
        rows.append(np.repeat(np.arange(n), np.diff(rp)) + off[-1])
        cols.append(cl.astype(np.int64) + off[-1])
        vals.append(vl)
        rhs.append(b)
        off.append(off[-1] + n)
    m = W.csr_from_coo(off[-1], np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return m, np.concatenate(rhs), np.array(off)


def _handle(G, systems, precision, damping=0.0, lsq_form=0):
    o = G.gabp_default_options()
    o.precision = precision
    o.damping = damping
    o.lsq_form = lsq_form
    o.stream = G.current_stream_handle()
    return G.gabp_create_lsq_batched([s[0] for s in systems], [s[1] for s in systems], o)


# ragged K and N: one column chunk, several chunks, K not a multiple of 32,
# the largest K and N the dense kernels take, N = 1
SHAPES = [(10, 1), (1, 5), (62, 31), (66, 33), (128, 64), (200, 100), (1024, 256), (512, 256),
          (70, 130), (3, 97)]


@pytest.mark.parametrize("damping", [0.0, 0.4])
def test_dense_fp64_rounds_match_oracle(G, damping):
    systems = _systems(SHAPES, seed=3, zero_frac=0.1)
    m, _, _ = _augmented_block_diag(systems)
    b = W.normal_rhs(m.n, 5)
    h = _handle(G, systems, precision=0, damping=damping)
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    for r in (0, 1, 2, 5, 9):
        G.gabp_run_rounds(h, bt, r, xt)
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r, damping=damping)
        assert _rel(xt.cpu().numpy(), ref["x"]) <= 1e-12, r
    G.gabp_destroy(h)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_dense_solve_matches_closed_form(G, precision):
    # BF16 mean messages (precision 2) keep about three digits; at 10 dB the
    # augmented systems amplify that past what refinement recovers, at 0 dB
    # (sigma^2 = 1) they do not
    systems = W.detection_batch(40, 16, 130, 0.0 if precision == 2 else 10.0, seed=2)
    h = _handle(G, [(d.S, d.sigma2, d.y) for d in systems], precision=precision)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    it = G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
    got = xh.cpu().numpy()
    off = 0
    for d in systems:
        A, bb = d.dense_system()
        assert _rel(got[off:off + d.K], np.linalg.solve(A, bb)) < 1e-8
        off += d.K
    assert it > 0
    stats = G.gabp_get_stats(h)
    assert stats["status"] == 0
    assert stats["edges"] == 2 * sum(d.S.size for d in systems)
    G.gabp_destroy(h)


def test_dense_and_csr_forms_agree(G):
    """The same damped batch through the dense kernels and through the
    general CSR path reaches the same x^ (both to 1e-10)."""
    systems = W.detection_batch(120, 16, 80, 10.0, seed=11)
    trip = [(d.S, d.sigma2, d.y) for d in systems]
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    out = []
    for form in (0, 1):
        h = _handle(G, trip, precision=1, damping=0.3, lsq_form=form)
        xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
        G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
        out.append(xh.cpu().numpy())
        G.gabp_destroy(h)
    assert _rel(out[0], out[1]) < 1e-8
    off = 0
    for d in systems:
        A, bb = d.dense_system()
        assert _rel(out[0][off:off + d.K], np.linalg.solve(A, bb)) < 1e-8
        off += d.K


def test_dense_handle_rejects_message_export(G):
    systems = _systems([(8, 4)], seed=1)
    h = _handle(G, systems, precision=0)
    with pytest.raises(G.GabpError):
        G.gabp_get_messages(h, 8)
    G.gabp_destroy(h)


def test_oversized_system_takes_the_csr_path(G):
    """K = 300 is beyond the dense kernels: the batch runs on the CSR path and
    still meets the closed form."""
    systems = _systems([(600, 300), (40, 20)], seed=9)
    h = _handle(G, systems, precision=1)
    y = torch.tensor(np.concatenate([s[2] for s in systems]), device="cuda")
    xh = torch.empty(320, dtype=torch.float64, device="cuda")
    G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
    got = xh.cpu().numpy()
    off = 0
    for S, psi, yy in systems:
        K = S.shape[1]
        closed = np.linalg.solve(S.T @ S + psi * np.eye(K), S.T @ yy)
        assert _rel(got[off:off + K], closed) < 1e-8
        off += K
    G.gabp_destroy(h)


@pytest.mark.parametrize("batch_control", [0, 1])
def test_bf16_refinement_converges_on_the_10db_batch(G, batch_control):
    """BF16 mean messages on the 10 dB batch: every system meets 1e-10 and
    its closed form to 1e-8 (per system, and under one controller for the
    whole batch).  Where a refinement step fails to shrink a residual by
    10 %, the precision ladder switches the later inner solves to FP32
    storage; the count of such sweeps stays below the mean sweeps.  Damped
    (gamma 0.3): undamped, one system of this batch does not converge."""
    systems = W.detection_batch(40, 16, 130, 10.0, seed=2)
    o = G.gabp_default_options()
    o.precision = 2
    o.damping = 0.3
    o.batch_control = batch_control
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([d.S for d in systems], [d.sigma2 for d in systems], o)
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 20000)
    st = G.gabp_get_stats(h)
    G.gabp_destroy(h)
    assert st["status"] == 0
    got, off = xh.cpu().numpy(), 0
    for d in systems:
        A, bb = d.dense_system()
        closed = np.linalg.solve(A, bb)
        assert np.abs(got[off:off + d.K] - closed).max() <= 1e-8 * np.abs(closed).max()
        off += d.K
    assert st["sweeps_wide"] <= st["sweeps_mean"], st


@pytest.mark.parametrize("precision,schedule", [(0, 1), (1, 1), (2, 1), (1, 0)])
def test_dense_breakdown_is_reported(G, precision, schedule):
    """S = I with psi = 1e-40: in the first round the z node's cavity
    precision P~_j - P_{x_r -> z_j} = (-psi - 1) - (-1) is zero in FP64 and
    FP32 (the serial kernels see it as a non-finite row or column sum), and
    the solve ends with GABP_ERR_BREAKDOWN instead of returning garbage.  The
    synchronous FP32 round meets -psi as a subnormal instead; its infinite
    message ends the solve too (breakdown or divergence)."""
    o = G.gabp_default_options()
    o.precision = precision
    o.schedule = schedule
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([np.eye(4)], [1e-40], o)
    y = torch.ones(4, dtype=torch.float64, device="cuda")
    xh = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GabpError) as ei:
        G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 1000)
    G.gabp_destroy(h)
    if schedule == 1:
        assert ei.value.name == "GABP_ERR_BREAKDOWN"
    else:
        assert ei.value.name in ("GABP_ERR_BREAKDOWN", "GABP_ERR_DIVERGED")
