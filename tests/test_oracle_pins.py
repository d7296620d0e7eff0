"""CPU pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value is either
printed in the paper (tests/golden/), a closed form, a textbook method written
out in the test, or a LAPACK solve of a small dense system.
"""
from collections import deque

import numpy as np
import pytest

import oracle
from paper_0810_1119_gb300 import workloads as W
from golden_io import paper_systems, toy_tree

TOY_NAMES = {"x": 0, "y": 1, "z": 2}


def _csr(A):
    return W.csr_from_dense(np.asarray(A, dtype=float))


def _pos(m, i, j):
    for e in range(m.row_ptr[i], m.row_ptr[i + 1]):
        if m.col[e] == j:
            return e
    raise KeyError((i, j))


def _run(m, b, rounds, **kw):
    return oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=rounds, want_messages=True, **kw)


def _diameter(m):
    """Graph diameter of a tree by two breadth-first searches."""
    def bfs(src):
        dist = {src: 0}
        q = deque([src])
        while q:
            u = q.popleft()
            for e in range(m.row_ptr[u], m.row_ptr[u + 1]):
                v = int(m.col[e])
                if v != u and v not in dist:
                    dist[v] = dist[u] + 1
                    q.append(v)
        far = max(dist, key=dist.get)
        return far, dist[far]
    far, _ = bfs(0)
    return bfs(far)[1]


# --------------------------------------------------------------------------
# Section VIII-A: the toy 3x3 tree, every printed message and mean.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_toy_tree_message_table(t):
    g = toy_tree()
    m = _csr([[float(v) for v in row] for row in g["A"]])
    b = np.array([float(v) for v in g["rhs"]])
    r = _run(m, b, t)
    assert r["status"] == "ok"
    for key, series in g.items():
        kind, _, pair = key.partition("_")
        if kind in ("P", "mu") and len(pair) == 2:
            i, j = TOY_NAMES[pair[0]], TOY_NAMES[pair[1]]
            got = r["P" if kind == "P" else "mu"][_pos(m, i, j)]
            assert got == pytest.approx(float(series[t]), abs=1e-14), (key, t)


@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_toy_tree_tentative_means(t):
    g = toy_tree()
    m = _csr([[float(v) for v in row] for row in g["A"]])
    b = np.array([float(v) for v in g["rhs"]])
    x = _run(m, b, t)["x"]
    for name, idx in TOY_NAMES.items():
        assert x[idx] == pytest.approx(float(g["mu_" + name][t]), abs=1e-14)


def test_toy_tree_precisions_equal_inverse_diagonal():
    g = toy_tree()
    A = np.array([[float(v) for v in row] for row in g["A"]])
    m = _csr(A)
    r = _run(m, np.array([float(v) for v in g["rhs"]]), 3)
    for name, idx in TOY_NAMES.items():
        assert r["Pi"][idx] == pytest.approx(float(g["Pfinal_" + name][0]), abs=1e-14)
    np.testing.assert_allclose(1.0 / r["Pi"], np.diag(np.linalg.inv(A)), rtol=1e-14)
    np.testing.assert_allclose(r["x"], [float(v) for v in g["solution"]], atol=1e-14)


# --------------------------------------------------------------------------
# Section IV: on a tree GaBP is exact, and it gets there in diameter rounds.
# --------------------------------------------------------------------------
TREES = [("path", W.path_graph(13, 1)),
         ("recursive", W.random_tree(40, 2, diag_scale=1.0)),
         ("recursive_indefinite", W.random_tree(25, 3, diag_scale=1.0, indefinite=True)),
         ("recursive_big", W.random_tree(200, 4, diag_scale=0.7))]


@pytest.mark.parametrize("name,m", TREES, ids=[t[0] for t in TREES])
def test_tree_exact_within_diameter_rounds(name, m):
    A = m.to_dense()
    b = W.normal_rhs(m.n, 7)
    D = _diameter(m)
    x_true = np.linalg.solve(A, b)
    var_true = np.diag(np.linalg.inv(A))
    r = _run(m, b, D)
    assert r["status"] == "ok"
    scale = np.abs(x_true).max()
    err = np.abs(r["x"] - x_true).max()
    assert err <= 1e-10 * scale
    np.testing.assert_allclose(1.0 / r["Pi"], var_true, rtol=1e-9)
    # One round short of the diameter an endpoint of a longest path is not
    # yet exact: its error is well above rounding level.
    early = _run(m, b, D - 1)
    early_err = np.abs(early["x"] - x_true).max()
    assert early_err > 1e-11 * scale and early_err > 100 * err
    # Further rounds do not move a converged tree.
    later = _run(m, b, D + 3)
    assert np.abs(later["x"] - r["x"]).max() <= 1e-12 * scale


# --------------------------------------------------------------------------
# Section III, Proposition (solution = marginal means): a converged GaBP mean
# equals A^{-1} b on loopy graphs too.
# --------------------------------------------------------------------------
LOOPY = [("poisson2d_p6", W.poisson2d(6)),
         ("er_n60", W.er_sdd(60, 6, 1.1, 5)),
         ("er_n200", W.er_sdd(200, 8, 1.05, 6))]


@pytest.mark.parametrize("name,m", LOOPY, ids=[t[0] for t in LOOPY])
def test_converged_mean_equals_dense_solve(name, m):
    A = m.to_dense()
    b = W.uniform_rhs(m.n, 11)
    r = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=5000,
                    tol=1e-13)
    assert r["status"] == "ok"
    x_true = np.linalg.solve(A, b)
    assert np.abs(r["x"] - x_true).max() <= 1e-10 * np.abs(x_true).max()


# --------------------------------------------------------------------------
# Section VI-C: zero precisions + "k in N(i)" instead of "N(i)\j" is Jacobi.
# --------------------------------------------------------------------------
def _textbook_jacobi(m, b, rounds):
    """x^{t+1}_i = (b_i - sum_{k != i} A_ik x^t_k) / A_ii, x^0 = D^{-1} b."""
    n = m.n
    diag = np.array([m.val[_pos(m, i, i)] for i in range(n)])
    x = b / diag
    for _ in range(rounds):
        new = np.empty(n)
        for i in range(n):
            s = b[i]
            for e in range(m.row_ptr[i], m.row_ptr[i + 1]):
                k = int(m.col[e])
                if k != i:
                    s -= m.val[e] * x[k]
            new[i] = s / diag[i]
        x = new
    return x


@pytest.mark.parametrize("m", [W.poisson2d(5), W.er_sdd(40, 5, 1.2, 9)])
def test_jacobi_variant_is_textbook_jacobi(m):
    b = W.uniform_rhs(m.n, 3)
    for t in (0, 1, 2, 7, 20):
        got = oracle.gabp(m.row_ptr, m.col, m.val, b, variant=oracle.JACOBI, max_rounds=t)["x"]
        assert np.array_equal(got, _textbook_jacobi(m, b, t)), t


# --------------------------------------------------------------------------
# Algorithm 1 (naive) and Algorithm 2 (broadcast) send the same messages.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [W.poisson2d(4), W.er_sdd(50, 7, 1.1, 12), W.random_tree(30, 8)])
def test_naive_equals_broadcast(m):
    b = W.normal_rhs(m.n, 4)
    for t in (1, 2, 5, 12):
        a = _run(m, b, t, variant=oracle.BROADCAST)
        c = _run(m, b, t, variant=oracle.NAIVE)
        for key in ("P", "mu", "x", "Pi"):
            ref = np.abs(c[key]).max()
            assert np.abs(a[key] - c[key]).max() <= 1e-12 * max(ref, 1e-300), (key, t)


# --------------------------------------------------------------------------
# Section VIII-B/C and IX: the paper's small systems.
# --------------------------------------------------------------------------
def _spectral_radius_abs_jacobi(A):
    D = np.diag(np.diag(A))
    M = np.abs(np.eye(A.shape[0]) - np.linalg.solve(D, A))
    return float(np.max(np.abs(np.linalg.eigvals(M))))


@pytest.mark.parametrize("name", ["R3", "R4"])
def test_cdma_spectral_radius_matches_paper(name):
    s = paper_systems()[name]
    assert _spectral_radius_abs_jacobi(s["A"]) == pytest.approx(s["spectral_radius"], abs=1e-4)


@pytest.mark.parametrize("name", ["R3", "R4", "nonPSD", "poisson_p3"])
def test_paper_systems_converge_to_solution(name):
    s = paper_systems()[name]
    m = _csr(s["A"])
    r = oracle.gabp(m.row_ptr, m.col, m.val, s["b"], stop=oracle.STOP_RES_ABS, max_rounds=2000,
                    tol=1e-14)
    assert r["status"] == "ok"
    x_true = np.linalg.solve(s["A"], s["b"])
    np.testing.assert_allclose(r["x"], x_true, rtol=1e-12, atol=1e-13)
    if "solution" in s:
        np.testing.assert_allclose(r["x"], [float(v) for v in s["solution"]], rtol=1e-12)


@pytest.mark.parametrize("name", ["R3", "R4", "nonPSD"])
def test_paper_iteration_counts_same_order(name):
    """Soft pin: message-change rule, threshold 1e-6 (Section VIII)."""
    s = paper_systems()[name]
    m = _csr(s["A"])
    r = oracle.gabp(m.row_ptr, m.col, m.val, s["b"], stop=oracle.STOP_MSG, max_rounds=2000,
                    tol=1e-6)
    assert r["status"] == "ok"
    paper = s["parallel_gabp_iterations"]
    assert paper / 2 <= r["rounds"] <= paper * 2, (r["rounds"], paper)


def test_poisson_iteration_count_same_order():
    """The Poisson table (134 parallel rounds) is captioned p = 3 but the text
    evaluates p = 10; at p = 10 with f = -1 the count is of that order."""
    p = 10
    m = W.poisson2d(p)
    b = np.full(m.n, 1.0 / (p + 1) ** 2)
    r = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_MSG, max_rounds=5000, tol=1e-6)
    assert r["status"] == "ok"
    paper = paper_systems()["poisson_p3"]["parallel_gabp_iterations"]
    assert paper / 3 <= r["rounds"] <= paper * 3, r["rounds"]


# --------------------------------------------------------------------------
# Section VII: the augmented system yields (S^T S + sigma^2 I)^{-1} S^T y.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("K", [4, 9, 16])
def test_augmented_system_closed_form(K):
    sysd = W.detection_batch(1, K, K, 10.0, seed=K)[0]
    row_ptr, col, val, rhs = oracle.augment_lsq(sysd.S, sysd.sigma2, sysd.y)
    n = row_ptr.shape[0] - 1
    m = W.CSR(n, row_ptr, col, val)
    A_dense, b_dense = sysd.dense_system()
    closed = np.linalg.solve(A_dense, b_dense)
    # The augmented matrix itself, solved directly, gives the closed form ...
    full = np.linalg.solve(m.to_dense(), rhs)
    np.testing.assert_allclose(full[:K], closed, rtol=1e-11, atol=1e-12)
    # ... and GaBP on it converges to the same vector.
    r = oracle.gabp(row_ptr, col, val, rhs, stop=oracle.STOP_RES_ABS, max_rounds=3000, tol=1e-13)
    assert r["status"] == "ok"
    np.testing.assert_allclose(r["x"][:K], closed, rtol=1e-9, atol=1e-10)


# --------------------------------------------------------------------------
# Section VII with Psi = 0: the Moore-Penrose solution, and the iteration
# that reaches it through augmented solves with Psi_0 > 0.
# --------------------------------------------------------------------------
def _rect(N, K, seed):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], size=(N, K)) / np.sqrt(N), rng.standard_normal(N)


@pytest.mark.parametrize("N,K", [(8, 3), (40, 16), (64, 16)])
def test_pinv_solution_meets_the_normal_equations(N, K):
    S, y = _rect(N, K, N + K)
    x = oracle.pinv_solution(S, y)
    g = S.T @ (y - S @ x)                    # normal equations S^T (y - S x) = 0
    assert np.abs(g).max() <= 1e-12 * np.abs(S.T @ y).max()
    # full column rank: (S^T S)^{-1} S^T y, the formula the section prints
    np.testing.assert_allclose(x, np.linalg.solve(S.T @ S, S.T @ y), rtol=1e-10, atol=1e-12)
    # the zero-noise limit of the closed form (S^T S + psi I)^{-1} S^T y
    for psi, tol in ((1e-6, 1e-4), (1e-9, 1e-7)):
        closed = np.linalg.solve(S.T @ S + psi * np.eye(K), S.T @ y)
        assert np.abs(closed - x).max() <= tol * np.abs(x).max()


def test_pinv_solution_of_a_square_system_is_the_inverse():
    """Section VII covers square nonsymmetric matrices too: S^+ = S^{-1}."""
    rng = np.random.default_rng(5)
    S = np.eye(6) + 0.3 * rng.standard_normal((6, 6))
    y = rng.standard_normal(6)
    np.testing.assert_allclose(oracle.pinv_solution(S, y), np.linalg.solve(S, y), rtol=1e-11)


def test_pinv_solution_of_a_rank_deficient_system_has_minimum_norm():
    """Two equal columns: every x with x_0 + x_1 fixed fits equally well; the
    pseudoinverse takes the one of minimum norm, x_0 = x_1."""
    rng = np.random.default_rng(6)
    c, d = rng.standard_normal(7), rng.standard_normal(7)
    S = np.stack([c, c, d], axis=1)
    y = rng.standard_normal(7)
    x = oracle.pinv_solution(S, y)
    assert abs(x[0] - x[1]) <= 1e-12 * np.abs(x).max()
    np.testing.assert_allclose(np.abs(S.T @ (y - S @ x)).max(), 0.0, atol=1e-12)


@pytest.mark.parametrize("psi0", [0.02, 0.1, 0.5])
def test_iterated_tikhonov_reaches_the_pinv_at_the_predicted_rate(psi0):
    """x^_k - S^+ y = (psi0 (S^T S + psi0 I)^{-1})^k (0 - S^+ y): the error
    along each right singular vector shrinks by psi0 / (sigma^2 + psi0) per
    step, so after k steps it is at most rho^k |S^+ y| with rho the largest
    such factor, and the first step is the Section VII closed form."""
    S, y = _rect(48, 16, 3)
    xs = oracle.pinv_solution(S, y)
    sig2 = np.linalg.svd(S, compute_uv=False) ** 2
    rho = (psi0 / (sig2 + psi0)).max()
    it = oracle.iterated_tikhonov(S, y, psi0, 30)
    np.testing.assert_allclose(it[0], np.linalg.solve(S.T @ S + psi0 * np.eye(16), S.T @ y), rtol=1e-12)
    for k in (1, 5, 10, 30):
        err = np.linalg.norm(it[k - 1] - xs)
        assert err <= rho ** k * np.linalg.norm(xs) * (1 + 1e-9) + 1e-13, (k, err)
    # the bound is attained in the slowest direction, not just an upper bound
    assert np.linalg.norm(it[9] - xs) >= 0.1 * rho ** 10 * np.abs(np.linalg.svd(S)[2][-1] @ xs)


# --------------------------------------------------------------------------
# Residual helper, input validation and breakdown.
# --------------------------------------------------------------------------
def test_residual_inf_matches_dense():
    m = W.er_sdd(80, 6, 1.1, 2)
    b = W.normal_rhs(80, 1)
    x = W.normal_rhs(80, 2)
    ref = np.abs(b - m.to_dense() @ x).max()
    assert oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) == pytest.approx(ref, rel=1e-13)


def test_bad_inputs_rejected():
    b = np.ones(2)
    asym = W.csr_from_dense(np.array([[2.0, 1.0], [0.5, 2.0]]))
    assert oracle.gabp(asym.row_ptr, asym.col, asym.val, b)["status"] == "bad_input"
    nodiag = W.csr_from_dense(np.array([[0.0, 1.0], [1.0, 2.0]]))
    assert oracle.gabp(nodiag.row_ptr, nodiag.col, nodiag.val, b)["status"] == "bad_input"


def test_breakdown_reported():
    # Round 1 sends P_21 = P_31 = -1 into node 1, so at round 2 the message
    # 1 -> 2 divides by P~_1 - P_21 = 1 - 1 - 1 + 1 = 0.
    m = W.csr_from_dense(np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0]]))
    b = np.ones(3)
    assert _run(m, b, 1)["status"] == "ok"
    assert _run(m, b, 2)["status"] == "breakdown"


# --------------------------------------------------------------------------
# Damping (the heuristic Section VI-D cites): same fixed point, and it
# rescues a Section VII detection system on which plain GaBP diverges.
# --------------------------------------------------------------------------
def test_zero_damping_is_the_plain_rule():
    m = W.er_sdd(120, 6, 1.1, 3)
    b = W.normal_rhs(m.n, 4)
    a = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=9, want_messages=True)
    c = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=9, want_messages=True, damping=0.0)
    for key in ("x", "P", "mu"):
        assert np.array_equal(a[key], c[key])


def test_damped_toy_tree_rounds_match_the_hand_derivation():
    """Rounds 1 and 2 of the synchronous damped rule on the Section VIII-A
    tree, gamma = 1/4, against exact rationals worked out by hand
    (tests/golden/toy_tree_damped.txt gives the derivation).  Round 1 fixes
    which weight the new message gets; round 2, where P_xy changes from -4 to
    1/2, fixes that the blend acts on P mu and not on mu."""
    g = toy_tree("toy_tree_damped.txt")
    gamma = float(g["gamma"][0])
    m = _csr([[float(v) for v in row] for row in g["A"]])
    b = np.array([float(v) for v in g["rhs"]])
    for t in (1, 2):
        r = _run(m, b, t, damping=gamma)
        for key, series in g.items():
            kind, _, pair = key.partition("_")
            if kind in ("P", "mu") and len(pair) == 2:
                e = _pos(m, TOY_NAMES[pair[0]], TOY_NAMES[pair[1]])
                got = r["P" if kind == "P" else "mu"][e]
                assert got == pytest.approx(float(series[t - 1]), rel=1e-14, abs=1e-14), (key, t)
            elif kind == "mu" and len(pair) == 1:
                got = r["x"][TOY_NAMES[pair]]
                assert got == pytest.approx(float(series[t - 1]), rel=1e-14, abs=1e-14), (key, t)


def test_damping_keeps_the_solution_and_rescues_divergence():
    # System 270 of this batch: plain synchronous GaBP diverges on its
    # augmented form (checked below), damped GaBP reaches the closed form.
    sysd = W.detection_batch(300, 16, 80, 10.0, seed=11)[270]
    rp, cl, vl, rhs = oracle.augment_lsq(sysd.S, sysd.sigma2, sysd.y)
    plain = oracle.gabp(rp, cl, vl, rhs, stop=oracle.STOP_RES_REL, max_rounds=600, tol=1e-10)
    assert plain["status"] == "not_converged"
    assert oracle.residual_inf(rp, cl, vl, rhs, plain["x"]) > 1.0
    damped = oracle.gabp(rp, cl, vl, rhs, stop=oracle.STOP_RES_REL, max_rounds=3000, tol=1e-12,
                         damping=0.3)
    assert damped["status"] == "ok"
    A, bb = sysd.dense_system()
    np.testing.assert_allclose(damped["x"][:sysd.K], np.linalg.solve(A, bb), rtol=1e-9, atol=1e-11)
    # precisions are not damped: identical to the plain run's
    np.testing.assert_allclose(damped["Pi"], oracle.gabp(rp, cl, vl, rhs, max_rounds=damped["rounds"])["Pi"],
                               rtol=1e-13)


# ---------------------------------------------------------------------------
# Aitken's Delta^2 (Section IV-A, convergence acceleration)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [0.5, -0.9, 0.99, -0.3])
def test_aitken_is_exact_on_one_geometric_mode(a):
    """For x_n = L + c a^n (any |a| < 1, either sign) the Delta^2 formula
    returns L exactly: the defining property the paper states.  In floating
    point the second difference is c a^n (1 - a)^2, formed from iterates of
    size |L|, so the result carries ~eps / (1 - a)^2 of relative rounding."""
    rng = np.random.default_rng(3)
    L = rng.standard_normal(50)
    c = rng.standard_normal(50)
    n = 7
    xs = [L + c * a ** k for k in (n, n + 1, n + 2)]
    y = oracle.aitken(*xs)
    tol = 100 * np.finfo(float).eps / (1 - a) ** 2
    assert np.abs(y - L).max() <= tol * np.abs(L).max()


def test_aitken_keeps_the_latest_iterate_without_curvature():
    x = np.array([1.0, -2.0, 3.0])
    assert np.array_equal(oracle.aitken(x, x, x), x)             # converged: Delta = 0
    lin0, lin1, lin2 = x, x + 1e-3, x + 2e-3                      # second difference 0
    assert np.array_equal(oracle.aitken(lin0, lin1, lin2), lin2)


def test_aitken_on_gabp_means_solves_poisson_in_fewer_rounds():
    """Synchronous GaBP on the 2D Poisson grid (a bipartite graph): the
    tentative means' error carries a component that flips sign every round,
    so Delta^2 over rounds two apart (stride 2) is what accelerates: the
    extrapolated means meet 1e-10 in well under 60 % of the plain rounds
    (the paper's Table for 2D Poisson: 134 plain vs 25 Aitken rounds)."""
    m = W.poisson2d(10)
    b = W.uniform_rhs(m.n, 0)

    def first_round(extrapolate):
        for r in range(8, 600, 4):
            x = oracle.gabp_aitken(m.row_ptr, m.col, m.val, b, r, 2) if extrapolate else \
                oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=r)["x"]
            if oracle.residual_inf(m.row_ptr, m.col, m.val, b, x) < 1e-10:
                return r
        return None

    plain, acc = first_round(False), first_round(True)
    assert plain is not None and acc is not None
    assert acc <= 0.6 * plain, (plain, acc)


def test_steffensen_residual_reaches_the_solution_faster_than_plain_refinement():
    """Steffensen's iteration (Section IV-A) in residual form on the 2D
    Poisson grid: six steps of 32 GaBP rounds each, Delta^2 over rounds two
    apart, reach the dense solve's solution to 1e-11, while plain
    refinement with the same rounds stays at least 1000 x further off."""
    m = W.poisson2d(10)
    b = W.uniform_rhs(m.n, 0)
    A = np.zeros((m.n, m.n))
    for i in range(m.n):
        A[i, m.col[m.row_ptr[i]:m.row_ptr[i + 1]]] = m.val[m.row_ptr[i]:m.row_ptr[i + 1]]
    ref = np.linalg.solve(A, b)
    xs, hs = oracle.steffensen_residual(m.row_ptr, m.col, m.val, b, inner_rounds=32, spacing=2,
                                        outer_steps=6)
    xp, hp = oracle.steffensen_residual(m.row_ptr, m.col, m.val, b, inner_rounds=32, spacing=0,
                                        outer_steps=6)
    assert np.abs(xs - ref).max() <= 1e-11 * np.abs(ref).max()
    assert hs[-1] <= 1e-3 * hp[-1], (hs, hp)
    assert np.abs(xp - ref).max() > 1e-9 * np.abs(ref).max()


def test_steffensen_residual_is_exact_in_one_step_on_a_chain():
    """On a chain (a tree) GaBP's means are exact once the rounds exceed the
    diameter, so the two later iterates agree; Delta^2 of (x0, x1, x1)
    returns x1 and one step of the iteration gives A^-1 b to rounding."""
    rng = np.random.default_rng(9)
    n = 12
    off = -(0.2 + rng.random(n - 1))
    A = np.diag(2.5 + rng.random(n)) + np.diag(off, 1) + np.diag(off, -1)
    b = rng.standard_normal(n)
    m = _csr(A)
    x, h = oracle.steffensen_residual(m.row_ptr, m.col, m.val, b, inner_rounds=n + 1, spacing=1,
                                      outer_steps=1)
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-13 * np.abs(x).max()
    assert h[-1] <= 1e-13 * np.abs(b).max()


# ---------------------------------------------------------------------------
# Serial schedule (Section III-C)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["R3", "R4", "nonPSD"])
def test_serial_iteration_counts_same_order(name):
    """Soft pin like the parallel counts: the paper's serial GaBP counts (16,
    13, 25) with the message-change rule at 1e-6, natural node order, and
    fewer rounds than the parallel schedule on the same system."""
    s = paper_systems()[name]
    m = _csr(s["A"])
    r = oracle.gabp_serial(m.row_ptr, m.col, m.val, s["b"], stop=oracle.STOP_MSG,
                           max_rounds=2000, tol=1e-6)
    assert r["status"] == "ok"
    paper = s["serial_gabp_iterations"]
    assert paper / 2 <= r["rounds"] <= paper * 2, (r["rounds"], paper)
    par = oracle.gabp(m.row_ptr, m.col, m.val, s["b"], stop=oracle.STOP_MSG, max_rounds=2000,
                      tol=1e-6)
    assert r["rounds"] < par["rounds"]


def test_serial_poisson_count_same_order():
    p = 10
    m = W.poisson2d(p)
    b = np.full(m.n, 1.0 / (p + 1) ** 2)
    r = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_MSG, max_rounds=5000,
                           tol=1e-6)
    assert r["status"] == "ok"
    paper = paper_systems()["poisson_p3"]["serial_gabp_iterations"]
    assert paper / 3 <= r["rounds"] <= paper * 3, r["rounds"]


@pytest.mark.parametrize("name", ["R3", "R4", "nonPSD", "poisson_p3"])
def test_serial_schedule_converges_to_the_solution(name):
    s = paper_systems()[name]
    m = _csr(s["A"])
    r = oracle.gabp_serial(m.row_ptr, m.col, m.val, s["b"], stop=oracle.STOP_RES_ABS,
                           max_rounds=2000, tol=1e-14)
    assert r["status"] == "ok"
    np.testing.assert_allclose(r["x"], np.linalg.solve(s["A"], s["b"]), rtol=1e-12, atol=1e-13)


def test_colour_classes_give_the_same_serial_round_in_any_inner_order():
    """Nodes of one colour class are not adjacent, so the order inside a
    class does not matter: two orders with the same sequence of classes give
    the same messages and means, bit for bit (the colour-block schedule the
    GPU runs is one serial schedule)."""
    m = W.er_sdd(400, 6, 1.1, 3)
    b = W.normal_rhs(m.n, 1)
    c = oracle.greedy_colouring(m.row_ptr, m.col)
    assert all(c[i] != c[j] for i in range(m.n) for j in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if j != i)
    fwd = np.argsort(c, kind="stable")
    rev_in_class = np.concatenate([np.flatnonzero(c == k)[::-1] for k in range(c.max() + 1)])
    a = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, order=fwd, max_rounds=7, want_messages=True)
    z = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, order=rev_in_class, max_rounds=7,
                           want_messages=True)
    assert np.array_equal(a["x"], z["x"])
    assert np.array_equal(a["P"], z["P"]) and np.array_equal(a["mu"], z["mu"])
    # and a different class sequence is a different schedule
    other = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=7)
    assert not np.array_equal(a["x"], other["x"])


def test_serial_round_on_a_path_propagates_left_to_right_in_one_round():
    """On a path graph visited left to right, every message i -> i+1 of the
    first round already carries all the information to its left: it equals
    the converged message (the synchronous schedule needs i rounds for it)."""
    m = W.path_graph(12, 4)
    b = W.normal_rhs(m.n, 2)
    one = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=1, want_messages=True)
    conv = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=40, want_messages=True)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    fwd = m.col == rows + 1                      # entries (i, i+1): messages i -> i+1
    np.testing.assert_allclose(one["P"][fwd], conv["P"][fwd], rtol=1e-13)
    np.testing.assert_allclose(one["mu"][fwd], conv["mu"][fwd], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# Damping restricted to the messages some nodes send (serial schedule)
# ---------------------------------------------------------------------------
def test_damping_mask_all_or_none_reduces_to_plain_runs():
    m = W.er_sdd(300, 6, 1.1, 4)
    b = W.normal_rhs(m.n, 2)
    full = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=6, want_messages=True,
                              damping=0.4)
    every = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=6, want_messages=True,
                               damping=0.4, damp_from=np.ones(m.n, bool))
    plain = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=6, want_messages=True)
    none = oracle.gabp_serial(m.row_ptr, m.col, m.val, b, max_rounds=6, want_messages=True,
                              damping=0.4, damp_from=np.zeros(m.n, bool))
    for k in ("x", "P", "mu"):
        assert np.array_equal(full[k], every[k])
        assert np.array_equal(plain[k], none[k])
    assert not np.array_equal(full["x"], plain["x"])


def test_damping_mask_first_round_on_an_augmented_system():
    """Round 1 from zero messages, x^ nodes visited before z nodes, damping
    on the z nodes only: the x^ nodes see only zero messages, so what they
    send is the undamped message; each z node sees the same x^ messages as
    in the undamped run, so its information P mu is (1 - gamma) times the
    undamped one and its precision is unchanged."""
    d = W.detection_batch(1, 12, 12, 10.0, seed=4)[0]
    rp, cl, vl, rhs = oracle.augment_lsq(d.S, d.sigma2, d.y)
    K = d.K
    z = np.arange(len(rp) - 1) >= K
    g = 0.3
    plain = oracle.gabp_serial(rp, cl, vl, rhs, max_rounds=1, want_messages=True)
    damp = oracle.gabp_serial(rp, cl, vl, rhs, max_rounds=1, want_messages=True, damping=g,
                              damp_from=z)
    sender = np.repeat(np.arange(len(rp) - 1), np.diff(rp))   # messages sit in the sender's row
    xs = ~z[sender]
    np.testing.assert_array_equal(damp["P"], plain["P"])
    np.testing.assert_array_equal(damp["mu"][xs], plain["mu"][xs])
    zs = z[sender] & (plain["P"] != 0)
    np.testing.assert_allclose(damp["P"][zs] * damp["mu"][zs], (1 - g) * plain["P"][zs] * plain["mu"][zs],
                               rtol=1e-13, atol=1e-16)


def test_damping_mask_keeps_the_fixed_point():
    """System 884 of the 10 dB detection batch (seed 0), where the undamped
    serial schedule does not reach 1e-10 in 600 rounds; damping only the
    messages the z nodes send converges to the Section VII closed form."""
    d = W.detection_batch(885, 16, 256, 10.0, seed=0)[884]
    rp, cl, vl, rhs = oracle.augment_lsq(d.S, d.sigma2, d.y)
    z = np.arange(len(rp) - 1) >= d.K
    plain = oracle.gabp_serial(rp, cl, vl, rhs, stop=oracle.STOP_RES_REL, max_rounds=600, tol=1e-10)
    assert plain["status"] != "ok"
    damp = oracle.gabp_serial(rp, cl, vl, rhs, stop=oracle.STOP_RES_REL, max_rounds=600, tol=1e-12,
                              damping=0.2, damp_from=z)
    assert damp["status"] == "ok" and damp["rounds"] < 200
    A, bb = d.dense_system()
    closed = np.linalg.solve(A, bb)
    assert np.abs(damp["x"][:d.K] - closed).max() < 1e-9 * np.abs(closed).max()
