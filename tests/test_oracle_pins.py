"""Pins for the FP64 oracle: each test checks it against something other than
itself (closed forms, brute force, a library routine, finite differences,
weak duality, invariances), so that a dropped term, a wrong sign or index, or
a transposed operand in the oracle fails one of them.  CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import kqr_oracle as O
from paper_2510_07929_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- kernel entries
def test_gram_closed_forms():
    X = np.array([[0.0, 0.0], [1.0, 2.0], [-1.0, 0.5]])
    K = O.gram(X, X, O.RBF, 0.5)
    assert K[0, 1] == pytest.approx(math.exp(-0.5 * 5.0), rel=1e-15)
    assert K[1, 2] == pytest.approx(math.exp(-0.5 * (4.0 + 2.25)), rel=1e-15)
    L = O.gram(X, X, O.LAPLACIAN, 0.5)
    assert L[0, 1] == pytest.approx(math.exp(-0.5 * 3.0), rel=1e-15)
    assert L[2, 1] == pytest.approx(math.exp(-0.5 * (2.0 + 1.5)), rel=1e-15)
    for M in (K, L):
        np.testing.assert_allclose(np.diag(M), 1.0)
        np.testing.assert_allclose(M, M.T)


def test_gram_positive_definite_and_translation_invariant():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, 3))
    for kind in (O.RBF, O.LAPLACIAN):
        K = O.gram(X, X, kind, 0.7)
        assert np.linalg.eigvalsh(K).min() > 0
        np.testing.assert_allclose(O.gram(X + 3.25, X + 3.25, kind, 0.7), K, rtol=1e-13, atol=1e-15)


def test_kmatvec_matches_python_loops():
    rng = np.random.default_rng(2)
    X = rng.random((9, 4))
    v = rng.standard_normal(9)
    for kind, dist in ((O.RBF, lambda a, b: sum((ai - bi) ** 2 for ai, bi in zip(a, b))),
                       (O.LAPLACIAN, lambda a, b: sum(abs(ai - bi) for ai, bi in zip(a, b)))):
        ref = [sum(math.exp(-0.3 * dist(X[i], X[j])) * v[j] for j in range(9)) for i in range(9)]
        np.testing.assert_allclose(O.kmatvec(X, v, kind, 0.3), ref, rtol=1e-14)
        np.testing.assert_allclose(O.kmatvec(X, v, kind, 0.3, rows=[4, 1]), [ref[4], ref[1]], rtol=1e-14)
        V = rng.standard_normal((9, 3))
        np.testing.assert_allclose(O.kmatvec(X, V, kind, 0.3, max_elems=10)[:, 2],
                                   O.kmatvec(X, V[:, 2], kind, 0.3), rtol=1e-14)


# ----------------------------------------------------------- loss, box, Jacobian
def test_check_loss_and_projection():
    z = np.array([-2.0, 0.0, 3.0])
    assert O.check_loss(z, 0.25) == pytest.approx(0.75 * 2.0 + 0.25 * 3.0)
    np.testing.assert_array_equal(O.proj_box([-1.0, -0.75, 0.1, 0.25, 2.0], 0.25),
                                  [-0.75, -0.75, 0.1, 0.25, 0.25])
    np.testing.assert_array_equal(O.jacobian_diag([-1.0, -0.75, 0.1, 0.25, 2.0], 0.25), [0, 0, 1, 0, 0])
    # rho_tau is the support function of [tau - 1, tau] (its conjugate is the box indicator)
    for t in (0.1, 0.5, 0.9):
        for zi in (-3.0, -0.5, 0.0, 0.7, 4.0):
            assert O.check_loss([zi], t) == pytest.approx(max(t * zi, (t - 1.0) * zi))


# --------------------------------------------------- phi_k, gradient, Hessian
def _phi_setup(seed=3, n=12, kind=O.RBF):
    rng = np.random.default_rng(seed)
    X = rng.random((n, 3))
    K = O.gram(X, X, kind, 0.8)
    y = rng.standard_normal(n)
    alpha = rng.uniform(-1.5, 1.5, n)
    z = rng.standard_normal(n)
    return K, y, alpha, z


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACIAN])
def test_grad_phi_matches_finite_differences(kind):
    K, y, alpha, z = _phi_setup(kind=kind)
    beta, sigma, tau, lam = 0.3, 2.0, 0.3, 0.05
    f = lambda a: O.phi(a, K @ a, y, beta, z, sigma, tau, lam)
    g = O.grad_phi(alpha, K @ alpha, y, beta, z, sigma, tau, lam)
    h = 1e-6
    fd = np.array([(f(alpha + h * e) - f(alpha - h * e)) / (2 * h) for e in np.eye(alpha.size)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6)


def test_generalized_hessian_matches_finite_differences_off_kinks():
    K, y, alpha, z = _phi_setup(seed=4)
    beta, sigma, tau, lam = -0.2, 1.5, 0.6, 0.1
    w = alpha + z / sigma
    assert np.min(np.minimum(np.abs(w - tau), np.abs(w - tau + 1))) > 1e-3
    S = O.jacobian_diag(w, tau)
    n = alpha.size
    H = K / lam + sigma * (np.ones((n, n)) + np.diag(1.0 - S))
    gr = lambda a: O.grad_phi(a, K @ a, y, beta, z, sigma, tau, lam)
    h = 1e-7
    fd = np.array([(gr(alpha + h * e) - gr(alpha - h * e)) / (2 * h) for e in np.eye(n)]).T
    np.testing.assert_allclose(H, fd, rtol=1e-6, atol=1e-5)
    assert np.linalg.eigvalsh(H).min() > 0          # every generalized Hessian is PD
    L = O.newton_diag(w, tau, sigma, lam, 0.0)
    np.testing.assert_allclose(lam * H, K + lam * sigma * np.ones((n, n)) + np.diag(L), rtol=1e-13)


# ---------------------------------------------------------- preconditioner
def test_woodbury_matches_dense_inverse():
    rng = np.random.default_rng(5)
    n, r = 30, 6
    F = rng.standard_normal((n, r))
    L = rng.uniform(1e-3, 2.0, n)
    gam = 0.37
    P = F @ F.T + gam * np.ones((n, n)) + np.diag(L)
    b = rng.standard_normal(n)
    np.testing.assert_allclose(O.woodbury_apply(F, L, gam, b), np.linalg.solve(P, b), rtol=1e-9)


def test_rpcholesky_pivot_rule_and_exactness():
    rng = np.random.default_rng(6)
    X = rng.random((25, 2))
    K = O.gram(X, X, O.RBF, 3.0)
    u = rng.random(25)
    F, piv = O.rpcholesky(lambda s: K[:, s], np.diag(K), 25, u)
    assert sorted(piv.tolist()) == list(range(25))               # without replacement
    np.testing.assert_allclose(F @ F.T, K, atol=1e-9)            # r = n recovers K
    F8, piv8 = O.rpcholesky(lambda s: K[:, s], np.diag(K), 8, u)
    np.testing.assert_array_equal(piv8, piv[:8])                 # prefix property of the sequence
    E = K - F8 @ F8.T
    assert np.linalg.eigvalsh(E).min() > -1e-12                  # K >= K_hat
    # first pivot: inverse-CDF of the uniform diagonal (all ones)
    assert piv[0] == int(np.floor(u[0] * 25))
    # second pivot by hand: residual diagonal after one step is 1 - K[:, s0]^2
    d1 = 1.0 - K[:, piv[0]] ** 2
    c = np.cumsum(d1)
    assert piv[1] == int(np.argmax(c > u[1] * d1.sum()))


def test_rank_from_spectrum():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 6)))
    sv = np.sqrt(np.array([100.0, 30.0, 5.0, 0.09, 0.05, 0.01]))
    F0 = Q * sv
    # eigenvalues of F0^T F0: 100, 30, 5, 0.09, 0.05, 0.01; xi = 1e-3 -> 0.1 >= 0.09 at r = 4
    assert O.rank_from_spectrum(F0, 1e-3) == 4
    assert O.rank_from_spectrum(F0, 0.5) == 2
    assert O.rank_from_spectrum(F0, 1e-6) == 6


def test_pcg_and_preconditioned_spectrum_bound():
    rng = np.random.default_rng(8)
    n = 60
    X = rng.random((n, 2))
    K = O.gram(X, X, O.RBF, 2.0)
    F, _ = O.rpcholesky(lambda s: K[:, s], np.diag(K), 10, rng.random(10))
    lam, sigma, eps = 0.05, 1.3, 1e-3
    S = (rng.random(n) < 0.4).astype(float)
    L = lam * sigma * (1.0 - S) + lam * eps
    A = K + lam * sigma * np.ones((n, n)) + np.diag(L)
    P = F @ F.T + lam * sigma * np.ones((n, n)) + np.diag(L)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(P, A)).real)
    # Appendix C: spec(P^-1 A) in [1, 1 + tr(K - K_hat) / min L]
    assert ev[0] > 1.0 - 1e-8
    assert ev[-1] < 1.0 + np.trace(K - F @ F.T) / L.min() + 1e-8
    b = rng.standard_normal(n)
    x, it, rn = O.pcg(lambda p: A @ p, b, lambda r: O.woodbury_apply(F, L, lam * sigma, r), 1e-10, 500)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-7, atol=1e-9)
    x1, it1, _ = O.pcg(lambda p: A @ p, b, lambda r: np.linalg.solve(A, r), 1e-9, 5)
    assert it1 == 1                                             # exact preconditioner: one step


# ---------------------------------------------------------------- solver
def brute_force_dual(K, y, tau, lam):
    """Enumerate every labelling of the points as lower bound / upper bound /
    free, solve the KKT equations of (1.3) on the free set, keep the labelling
    whose box and sign conditions hold (Sec. 4 KKT at zero residual)."""
    n = y.size
    best = None
    for lab in itertools.product((0, 1, 2), repeat=n):
        lab = np.array(lab)
        a = np.where(lab == 0, tau - 1.0, tau).astype(float)
        E = np.flatnonzero(lab == 2)
        N = np.flatnonzero(lab != 2)
        if E.size:
            A = np.zeros((E.size + 1, E.size + 1))
            A[:E.size, :E.size] = K[np.ix_(E, E)] / lam
            A[:E.size, E.size] = 1.0
            A[E.size, :E.size] = 1.0
            rhs = np.concatenate([y[E] - K[np.ix_(E, N)] @ a[N] / lam, [-a[N].sum()]])
            sol = np.linalg.solve(A, rhs)
            a[E] = sol[:E.size]
            beta = sol[E.size]
            viol = max(0.0, np.max(np.maximum(a[E] - tau, tau - 1.0 - a[E])))
        else:
            if abs(a.sum()) > 1e-12:
                continue
            r = y - K @ a / lam
            lo = np.max(r[lab == 0]) if np.any(lab == 0) else -np.inf
            hi = np.min(r[lab == 1]) if np.any(lab == 1) else np.inf
            beta = 0.5 * (lo + hi) if np.isfinite(lo) and np.isfinite(hi) else (lo if np.isfinite(lo) else hi)
            viol = 0.0
        zres = y - beta - K @ a / lam
        viol = max(viol, np.max(np.where(lab == 1, -zres, 0.0)), np.max(np.where(lab == 0, zres, 0.0)))
        if best is None or viol < best[0]:
            best = (viol, a.copy(), beta)
    return best


@pytest.mark.parametrize("seed,tau,lam,kind", [(0, 0.5, 0.3, O.RBF), (1, 0.2, 0.05, O.LAPLACIAN),
                                               (2, 0.75, 1.0, O.RBF), (3, 0.35, 0.02, O.LAPLACIAN)])
def test_solver_matches_brute_force_active_sets(seed, tau, lam, kind):
    rng = np.random.default_rng(seed)
    n = 7
    X = rng.random((n, 2))
    y = rng.standard_normal(n)
    K = O.gram(X, X, kind, 1.0)
    viol, a_bf, b_bf = brute_force_dual(K, y, tau, lam)
    assert viol < 1e-10
    res = O.solve_dense(K, y, tau, lam, tol=1e-10)
    np.testing.assert_allclose(res["alpha"], a_bf, atol=1e-7)
    assert res["kkt"]["eta_kkt"] <= 1e-10


def test_solver_matches_library_qp():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    n, tau, lam = 25, 0.3, 0.2
    X = rng.random((n, 3))
    y = rng.standard_normal(n)
    K = O.gram(X, X, O.LAPLACIAN, 0.5)
    f = lambda a: a @ K @ a / (2 * lam) - y @ a
    jac = lambda a: K @ a / lam - y
    qp = scipy_opt.minimize(f, np.zeros(n), jac=jac, method="SLSQP", bounds=[(tau - 1, tau)] * n,
                            constraints=[{"type": "eq", "fun": lambda a: a.sum(), "jac": lambda a: np.ones(n)}],
                            options=dict(ftol=1e-15, maxiter=1000))
    res = O.solve_dense(K, y, tau, lam, tol=1e-10)
    assert -f(res["alpha"]) >= -f(qp.x) - 1e-9
    np.testing.assert_allclose(res["alpha"], qp.x, atol=1e-5)


def test_large_lambda_reaches_lp_vertex():
    """max y^T alpha over the box with 1^T alpha = 0: top of y at tau, bottom at
    tau - 1, one fractional coordinate.  For lambda above
    max_i |(K a)_i - (K a)_q| / |y_i - y_q| the dual solution is that vertex."""
    rng = np.random.default_rng(12)
    n, tau = 10, 0.25
    X = rng.random((n, 2))
    y = rng.standard_normal(n)
    K = O.gram(X, X, O.RBF, 1.0)
    order = np.argsort(-y)
    k = int(math.ceil(n * (1 - tau) - 1))
    a = np.full(n, tau - 1.0)
    a[order[:k]] = tau
    q = order[k]
    a[q] = (n - k - 1) - (n - 1) * tau
    assert tau - 1 < a[q] < tau and abs(a.sum()) < 1e-14
    Ka = K @ a
    thr = max(abs(Ka[i] - Ka[q]) / abs(y[i] - y[q]) for i in range(n) if i != q)
    res = O.solve_dense(K, y, tau, 10 * thr, tol=1e-10)
    np.testing.assert_allclose(res["alpha"], a, atol=1e-8)


def test_two_point_closed_form_fixture():
    data = json.load(open(os.path.join(GOLDEN, "two_point.json")))
    env = {"exp": math.exp}
    for c in data["cases"]:
        X, y = np.array(c["x"]), np.array(c["y"])
        K = O.gram(X, X, c["kind"], c["gamma"])
        assert K[0, 1] == pytest.approx(eval(c["k12"], env), rel=1e-15)
        res = O.solve_dense(K, y, c["tau"], c["lam"], tol=1e-12)
        np.testing.assert_allclose(res["alpha"], [eval(s, env) for s in c["alpha"]], atol=1e-10)
        if c["beta"] is not None:
            assert res["beta"] == pytest.approx(eval(c["beta"], env), abs=1e-9)


def _small_problem(seed=21, n=120, kind=O.RBF):
    wl = W.rbf_small(n=n, seed=seed) if kind == O.RBF else W.lap_large(n=n, p=6, seed=seed)
    return wl, O.gram(wl.X, wl.X, wl.kind, wl.gamma)


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACIAN])
def test_solution_feasible_quantile_and_certified(kind):
    wl, K = _small_problem(kind=kind)
    res = O.solve_dense(K, wl.y, wl.tau, wl.lam, tol=1e-10)
    a, v = res["alpha"], res["v"]
    assert np.all(v >= wl.tau - 1) and np.all(v <= wl.tau)          # v is the projection
    assert np.max(np.abs(a - v)) < 1e-8 and abs(a.sum()) < 1e-8     # alpha -> v as eta_d -> 0
    # quantile property: N_minus <= n tau <= n - N_plus (KKT + 1^T alpha = 0)
    zres = wl.y - res["beta"] - K @ a / wl.lam
    tol = 1e-7 * (1 + np.abs(wl.y))
    assert np.sum(zres < -tol) <= wl.n * wl.tau + 1e-9
    assert np.sum(zres > tol) <= wl.n * (1 - wl.tau) + 1e-9
    cert = O.certified_gap(a, K, wl.y, wl.tau, wl.lam)
    assert 0 <= cert["gap"] < 1e-8
    # weak duality: any feasible alpha and any (theta, beta) give P >= D
    rng = np.random.default_rng(0)
    other = O.project_feasible(rng.uniform(-1, 1, wl.n), wl.tau)
    c2 = O.certified_gap(other, K, wl.y, wl.tau, wl.lam)
    assert c2["P"] >= c2["D"] and c2["D"] <= cert["D"] + 1e-9
    # representer form at the training points: y - f(x_i) = primal residual
    f = O.predict(wl.X, a, res["beta"], wl.X, wl.kind, wl.gamma, wl.lam)
    np.testing.assert_allclose(wl.y - f, res["z"], atol=1e-7 * (1 + np.linalg.norm(wl.y)))


def test_exact_invariances():
    wl, K = _small_problem(seed=22, n=60)
    y, tau, lam = wl.y, wl.tau, wl.lam
    tau = 0.3
    base = O.solve_dense(K, y, tau, lam, tol=1e-11)
    sh = O.solve_dense(K, y + 2.5, tau, lam, tol=1e-11)
    np.testing.assert_allclose(sh["alpha"], base["alpha"], atol=1e-7)
    assert sh["beta"] == pytest.approx(base["beta"] + 2.5, abs=1e-6)
    sc = O.solve_dense(K, 3.0 * y, tau, lam / 3.0, tol=1e-11)
    np.testing.assert_allclose(sc["alpha"], base["alpha"], atol=1e-7)
    ng = O.solve_dense(K, -y, 1 - tau, lam, tol=1e-11)
    np.testing.assert_allclose(ng["alpha"], -base["alpha"], atol=1e-7)
    perm = np.random.default_rng(3).permutation(y.size)
    pm = O.solve_dense(K[np.ix_(perm, perm)], y[perm], tau, lam, tol=1e-11)
    np.testing.assert_allclose(pm["alpha"], base["alpha"][perm], atol=1e-7)


def test_kkt_residuals_vanish_at_closed_form_solution():
    c = json.load(open(os.path.join(GOLDEN, "two_point.json")))["cases"][0]
    X, y = np.array(c["x"]), np.array(c["y"])
    K = O.gram(X, X, c["kind"], c["gamma"])
    a = np.array([eval(s, {"exp": math.exp}) for s in c["alpha"]])
    beta = 0.5
    z = y - beta - K @ a / c["lam"]
    res = O.kkt_residuals(a, a.copy(), beta, z, y, K @ a, c["tau"], c["lam"])
    assert res["eta_kkt"] < 1e-15 and res["eta_gap"] < 1e-15
    bad = O.kkt_residuals(a, a.copy(), beta + 0.1, z, y, K @ a, c["tau"], c["lam"])
    assert bad["eta_p"] == pytest.approx(0.1 * math.sqrt(2) / (1 + np.linalg.norm(y)))


def test_kkt_residuals_three_point_golden():
    """Sec. 4 residuals at a hand-computed point with z != 0, alpha != v and
    1^T alpha != 0 (tests/golden/kkt_three_point.json): pins eta_d and eta_c,
    which vanish at any solution and so are not fixed by the closed forms."""
    c = json.load(open(os.path.join(GOLDEN, "kkt_three_point.json")))
    env = {"sqrt": math.sqrt, "log": math.log}
    X = np.array(c["x"])
    K = O.gram(X, X, c["kind"], eval(c["gamma"], env))
    np.testing.assert_allclose(K, [[eval(s, env) for s in row] for row in c["K"]], rtol=1e-15)
    a, v, z, y = (np.array(c[k]) for k in ("alpha", "v", "z", "y"))
    res = O.kkt_residuals(a, v, c["beta"], z, y, K @ a, c["tau"], c["lam"])
    for key, expr in c["expected"].items():
        assert res[key] == pytest.approx(eval(expr, env), rel=1e-13), key
    assert res["eta_kkt"] == max(res["eta_p"], res["eta_d"], res["eta_c"])


@pytest.mark.parametrize("kind", [O.RBF, O.LAPLACIAN])
def test_native_products_match_numpy_oracle(kind):
    """The oracle's C form of K and K.V (kernel_native.c, used at sizes numpy
    cannot reach) against the numpy definitions, on ragged sizes and row subsets."""
    from oracle import native as N

    rng = np.random.default_rng(31)
    X = rng.standard_normal((1037, 7))
    Z = rng.standard_normal((515, 7))
    V = rng.standard_normal((1037, 3))
    ref = O.kmatvec(X, V, kind, 0.3)
    np.testing.assert_allclose(N.kmatvec(X, V, kind, 0.3), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    rows = rng.choice(1037, 33, replace=False)
    np.testing.assert_allclose(N.kmatvec(X, V[:, 1], kind, 0.3, rows=rows), ref[rows, 1], rtol=1e-12,
                               atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(N.gram(X[:40], Z, kind, 0.3), O.gram(X[:40], Z, kind, 0.3), rtol=1e-13, atol=1e-300)
    assert N.threads() >= 1
