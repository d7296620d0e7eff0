"""Section VII with Psi = 0 through the C ABI: gabp_create_lsq_batched given
psi_s = 0 returns the Moore-Penrose solution x^ = S^+ y.

GaBP cannot run on the augmented matrix with a zero Psi (its z nodes would
have a zero diagonal), so the library solves augmented systems with
Psi_0 = 0.1 (mean squared column norm) I and iterates
x^ <- x^ + (S^T S + Psi_0)^{-1} S^T (y - S x^) to the normal equations.
The reference is the oracle's pinv_solution (the least-squares definition,
LAPACK), pinned on the CPU.

Tolerances: the solve stops when ||S^T (y - S x^)||_inf <= 1e-10
||S^T y||_inf for every psi_s = 0 system; that is checked again here in
FP64 (bound 2e-10, the GPU's FP64 products and the check's own sum in a
different order).  The error against S^+ y is then bounded by the
condition number of S^T S times that residual: at most 9 (N = 4K, entries
+-1/sqrt(N)) and 2 (the square case) here, so 1e-8 relative leaves margin.
Systems given psi_s > 0 in the same batch must still return their own
closed form (S^T S + psi_s I)^{-1} S^T y, to 1e-8.
"""
import numpy as np
import pytest

import oracle

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


def _tall(N, K, seed):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], size=(N, K)) / np.sqrt(N), rng.standard_normal(N)


def _batch(nsys, seed0):
    return [_tall(4 * (8 + 4 * (s % 8)), 8 + 4 * (s % 8), seed0 + s) for s in range(nsys)]


def _solve(G, systems, psi, precision, lsq_form, damping=0.0):
    o = G.gabp_default_options()
    o.precision = precision
    o.lsq_form = lsq_form
    o.damping = damping
    o.stream = G.current_stream_handle()
    h = G.gabp_create_lsq_batched([S for S, _ in systems], psi, o)
    y = torch.tensor(np.concatenate([yy for _, yy in systems]), device="cuda")
    xh = torch.full((sum(S.shape[1] for S, _ in systems),), float("nan"), dtype=torch.float64,
                    device="cuda")
    iters = G.gabp_solve_lsq_batched(h, y, xh, 1e-10, 200000)
    st = G.gabp_get_stats(h)
    G.gabp_destroy(h)
    out, off = [], 0
    for S, _ in systems:
        out.append(xh.cpu().numpy()[off:off + S.shape[1]])
        off += S.shape[1]
    return out, iters, st


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lsq_form", [0, 1])
def test_psi_zero_gives_the_moore_penrose_solution(G, precision, lsq_form):
    systems = _batch(12, 100)
    xs, iters, st = _solve(G, systems, 0.0, precision, lsq_form)
    for (S, y), x in zip(systems, xs):
        g = S.T @ (y - S @ x)
        assert np.abs(g).max() <= 2e-10 * np.abs(S.T @ y).max()
        assert _rel(x, oracle.pinv_solution(S, y)) < 1e-8
    # each augmented solve gains a factor psi_0 / (sigma_min^2 + psi_0) <= 0.31
    # here, so 1e-10 takes about 20 of them
    assert 5 <= st["outer_steps"] <= 60, st
    assert st["sweeps_total"] == iters and st["status"] == 0


def test_mixed_batch_keeps_the_regularised_systems(G):
    """psi_s > 0 systems of the same batch return their Section VII closed
    form; only the psi_s = 0 ones are iterated to S^+ y."""
    systems = _batch(8, 300)
    psi = [0.0 if s % 2 == 0 else 0.1 for s in range(8)]
    for lsq_form in (0, 1):
        xs, _, _ = _solve(G, systems, psi, 0, lsq_form)
        for (S, y), x, p in zip(systems, xs, psi):
            if p == 0.0:
                want = oracle.pinv_solution(S, y)
            else:
                want = np.linalg.solve(S.T @ S + p * np.eye(S.shape[1]), S.T @ y)
            assert _rel(x, want) < 1e-8, (lsq_form, p)


def test_square_nonsymmetric_system_gives_its_inverse(G):
    """Section VII extends the solver to square nonsymmetric matrices: with
    Psi = 0 the answer is S^{-1} y."""
    rng = np.random.default_rng(7)
    S = np.eye(16) + 0.3 * rng.standard_normal((16, 16)) / 4
    y = rng.standard_normal(16)
    for precision in (0, 1):
        xs, _, _ = _solve(G, [(S, y)], 0.0, precision, 0)
        assert _rel(xs[0], np.linalg.solve(S, y)) < 1e-8, precision


def test_damped_psi_zero_solve(G):
    systems = _batch(6, 500)
    xs, _, st = _solve(G, systems, 0.0, 0, 0, damping=0.3)
    for (S, y), x in zip(systems, xs):
        assert _rel(x, oracle.pinv_solution(S, y)) < 1e-8
    assert st["residual"] <= 2e-10 * st["rhs_norm"]
