"""Plant plausible mistakes in a copy of the oracle and check that its pins
catch every one.

Each mutant is the oracle's C source with one edit (a sign, a dropped term, a
transposed operand, a wrong divisor), compiled to a temporary library on the
CPU.  The pins are the same kinds of facts as in test_oracle_pins.py: the
paper's toy-tree tables, exact tree convergence and dense LU on loopy graphs.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1119_gb300 import workloads as W
from golden_io import toy_tree

MUTANTS = {
    "precision_sign": ("Pn[e] = -Aij * Aij / denom;", "Pn[e] = Aij * Aij / denom;"),
    "denominator_adds_reverse": ("const double denom = Pt - Pji;", "const double denom = Pt + Pji;"),
    "mean_drops_reverse_term": ("Mn[e] = (Pt * mut - Pji * muji) / Aij;", "Mn[e] = (Pt * mut) / Aij;"),
    "precision_total_reads_outgoing": ("Psum += Po[twin[e]];                   /* P_ki, k = col[e] */",
                                       "Psum += Po[e];"),
    "mean_total_drops_precision": ("hsum += Po[twin[e]] * Mo[twin[e]];     /* P_ki mu_ki */",
                                   "hsum += Mo[twin[e]];"),
    "self_mean_not_divided": ("const double muii = b[i] / Pii;        /* mu_ii = b_i / A_ii */",
                              "const double muii = b[i];"),
    "marginal_divides_by_self_precision": ("    x[i] = hsum / Psum;\n    if (Pi) Pi[i] = Psum;",
                                           "    x[i] = hsum / Pii;\n    if (Pi) Pi[i] = Psum;"),
    "mean_message_sign": ("Mn[e] = (Pt * mut - Pji * muji) / Aij;", "Mn[e] = -(Pt * mut - Pji * muji) / Aij;"),
    # the synchronous damping blend (reading of Section VI-D): weights swapped,
    # and the blend applied to mu instead of to P mu
    "damping_weights_swapped": ("const double eta = gamma * (Po[e] * Mo[e]) + (1.0 - gamma) * (Pn[e] * Mn[e]);",
                                "const double eta = (1.0 - gamma) * (Po[e] * Mo[e]) + gamma * (Pn[e] * Mn[e]);"),
    "damping_blends_mean": ("const double eta = gamma * (Po[e] * Mo[e]) + (1.0 - gamma) * (Pn[e] * Mn[e]);\n"
                            "          Mn[e] = eta / Pn[e];",
                            "Mn[e] = gamma * Mo[e] + (1.0 - gamma) * Mn[e];"),
}


def _damped_pins_hold(lib) -> bool:
    """Rounds 1 and 2 of the damped toy tree against the hand derivation in
    tests/golden/toy_tree_damped.txt."""
    g = toy_tree("toy_tree_damped.txt")
    A = np.array([[float(v) for v in row] for row in g["A"]])
    m = W.csr_from_dense(A)
    b = np.array([float(v) for v in g["rhs"]])
    pos = {(i, int(m.col[e])): e for i in range(3) for e in range(m.row_ptr[i], m.row_ptr[i + 1])}
    names = {"x": 0, "y": 1, "z": 2}
    for t in (1, 2):
        r = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=t, want_messages=True, lib=lib,
                        damping=float(g["gamma"][0]))
        for key, series in g.items():
            kind, _, pair = key.partition("_")
            if kind in ("P", "mu") and len(pair) == 2:
                got = r["P" if kind == "P" else "mu"][pos[(names[pair[0]], names[pair[1]])]]
            elif kind == "mu" and len(pair) == 1:
                got = r["x"][names[pair]]
            else:
                continue
            if abs(got - float(series[t - 1])) > 1e-12:
                return False
    return True


def _pins_hold(lib) -> bool:
    if not _damped_pins_hold(lib):
        return False
    g = toy_tree()
    A = np.array([[float(v) for v in row] for row in g["A"]])
    m = W.csr_from_dense(A)
    b = np.array([float(v) for v in g["rhs"]])
    pos = {(i, j): e for i in range(3) for e in range(m.row_ptr[i], m.row_ptr[i + 1])
           for j in [int(m.col[e])]}
    names = {"x": 0, "y": 1, "z": 2}
    for t in (1, 2, 3):
        r = oracle.gabp(m.row_ptr, m.col, m.val, b, max_rounds=t, want_messages=True, lib=lib)
        for key, series in g.items():
            kind, _, pair = key.partition("_")
            if kind in ("P", "mu") and len(pair) == 2:
                got = r["P" if kind == "P" else "mu"][pos[(names[pair[0]], names[pair[1]])]]
                if abs(got - float(series[t])) > 1e-12:
                    return False
            if kind == "mu" and len(pair) == 1:
                if abs(r["x"][names[pair]] - float(series[t])) > 1e-12:
                    return False
    for mm in (W.poisson2d(5), W.er_sdd(60, 6, 1.1, 5)):
        rhs = W.uniform_rhs(mm.n, 1)
        r = oracle.gabp(mm.row_ptr, mm.col, mm.val, rhs, stop=oracle.STOP_RES_REL, max_rounds=3000,
                        tol=1e-12, lib=lib)
        x_true = np.linalg.solve(mm.to_dense(), rhs)
        if r["status"] != "ok" or not np.allclose(r["x"], x_true, rtol=1e-9, atol=1e-9):
            return False
    return True


def test_unmodified_source_passes(tmp_path):
    lib = oracle.compile_variant(oracle.source(), str(tmp_path / "orig.so"))
    assert _pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    lib = oracle.compile_variant(src.replace(old, new, 1), str(tmp_path / f"{name}.so"))
    assert not _pins_hold(lib)


# Section VII with Psi = 0 (oracle/augment.py): the same kind of plausible
# mistakes planted in the Python source of pinv_solution / iterated_tikhonov,
# and the facts test_oracle_pins.py pins them to (the normal equations, the
# square inverse, the predicted contraction rate, the closed form as step 1).
PINV_MUTANTS = {
    "residual_sign": ("S.T @ (np.asarray(y, dtype=np.float64) - S @ x)",
                      "S.T @ (np.asarray(y, dtype=np.float64) + S @ x)"),
    "no_accumulation": ("x = x + np.linalg.solve(M, ", "x = np.linalg.solve(M, "),
    "shift_on_the_wrong_gram": ("M = S.T @ S + psi0 * np.eye(K)",
                                "M = S.T @ S[:K, :K].T + psi0 * np.eye(K)"),
    "regularised_not_pinv": ("return np.linalg.lstsq(S, np.asarray(y, dtype=np.float64), rcond=None)[0]",
                             "return np.linalg.solve(S.T @ S + 1e-3 * np.eye(S.shape[1]), S.T @ y)"),
    "transposed_operand": ("return np.linalg.lstsq(S, np.asarray(y, dtype=np.float64), rcond=None)[0]",
                           "return np.linalg.lstsq(S.T @ S, np.asarray(y, dtype=np.float64)[:S.shape[1]], rcond=None)[0]"),
}


def _pinv_namespace(src):
    ns = {}
    exec(compile(src, "augment_mutant.py", "exec"), ns)
    return ns


def _pinv_pins_hold(ns) -> bool:
    try:
        rng = np.random.default_rng(3)
        S = rng.choice([-1.0, 1.0], size=(48, 16)) / np.sqrt(48)
        y = rng.standard_normal(48)
        x = ns["pinv_solution"](S, y)
        if np.abs(S.T @ (y - S @ x)).max() > 1e-12 * np.abs(S.T @ y).max():
            return False
        Sq = np.eye(6) + 0.3 * rng.standard_normal((6, 6))
        yq = rng.standard_normal(6)
        if not np.allclose(ns["pinv_solution"](Sq, yq), np.linalg.solve(Sq, yq), rtol=1e-10):
            return False
        xs = np.linalg.solve(S.T @ S, S.T @ y)
        psi0 = 0.1
        rho = (psi0 / (np.linalg.svd(S, compute_uv=False) ** 2 + psi0)).max()
        it = ns["iterated_tikhonov"](S, y, psi0, 20)
        if not np.allclose(it[0], np.linalg.solve(S.T @ S + psi0 * np.eye(16), S.T @ y), rtol=1e-12):
            return False
        return all(np.linalg.norm(it[k - 1] - xs) <= rho ** k * np.linalg.norm(xs) * (1 + 1e-9) + 1e-13
                   for k in (1, 5, 20))
    except Exception:   # a mutant that does not even run is caught too
        return False


def test_pinv_pins_hold_for_the_oracle():
    import inspect
    from oracle import augment
    assert _pinv_pins_hold(_pinv_namespace(inspect.getsource(augment)))


@pytest.mark.parametrize("name", sorted(PINV_MUTANTS))
def test_pinv_pins_catch_mutant(name):
    import inspect
    from oracle import augment
    src = inspect.getsource(augment)
    old, new = PINV_MUTANTS[name]
    assert src.count(old) == 1, name
    assert not _pinv_pins_hold(_pinv_namespace(src.replace(old, new)))


# Steffensen's iteration in residual form (oracle.steffensen_residual): the
# same kind of mistakes planted in its Python source, checked against the
# facts test_oracle_pins.py pins it to (the LAPACK solution of 2D Poisson,
# at least 1000 x below plain refinement with the same rounds, and one-step
# exactness on a chain).
STEFFENSEN_MUTANTS = {
    "update_sign": ("x = x + y", "x = x - y"),
    "correction_replaces_x": ("x = x + y", "x = y"),
    "residual_sign": ("r = b - A @ x", "r = A @ x - b"),
    "no_extrapolation": ("y = aitken(*ds)", "y = ds[-1]"),
    "oldest_iterate": ("y = aitken(*ds)", "y = ds[0]"),
}


def _steffensen_pins_hold(fn) -> bool:
    try:
        m = W.poisson2d(10)
        b = W.uniform_rhs(m.n, 0)
        A = np.zeros((m.n, m.n))
        for i in range(m.n):
            A[i, m.col[m.row_ptr[i]:m.row_ptr[i + 1]]] = m.val[m.row_ptr[i]:m.row_ptr[i + 1]]
        ref = np.linalg.solve(A, b)
        xs, hs = fn(m.row_ptr, m.col, m.val, b, inner_rounds=32, spacing=2, outer_steps=6)
        _, hp = fn(m.row_ptr, m.col, m.val, b, inner_rounds=32, spacing=0, outer_steps=6)
        if not (np.abs(xs - ref).max() <= 1e-11 * np.abs(ref).max() and hs[-1] <= 1e-3 * hp[-1]):
            return False
        rng = np.random.default_rng(9)
        n = 12
        off = -(0.2 + rng.random(n - 1))
        T = np.diag(2.5 + rng.random(n)) + np.diag(off, 1) + np.diag(off, -1)
        bt = rng.standard_normal(n)
        mt = W.csr_from_dense(T)
        x, _ = fn(mt.row_ptr, mt.col, mt.val, bt, inner_rounds=n + 1, spacing=1, outer_steps=1)
        return np.abs(x - np.linalg.solve(T, bt)).max() <= 1e-13 * np.abs(x).max()
    except Exception:   # a mutant that does not even run is caught too
        return False


def _steffensen_variant(src):
    ns = dict(oracle.__dict__)
    exec(compile(src, "steffensen_mutant.py", "exec"), ns)
    return ns["steffensen_residual"]


def test_steffensen_pins_hold_for_the_oracle():
    assert _steffensen_pins_hold(oracle.steffensen_residual)


@pytest.mark.parametrize("name", sorted(STEFFENSEN_MUTANTS))
def test_steffensen_pins_catch_mutant(name):
    import inspect
    src = inspect.getsource(oracle.steffensen_residual)
    old, new = STEFFENSEN_MUTANTS[name]
    assert src.count(old) == 1, name
    assert not _steffensen_pins_hold(_steffensen_variant(src.replace(old, new)))
