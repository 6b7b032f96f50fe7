"""Grid solves (kqr_solve_grid, kqr_solve_grid_batch): many (tau, lambda) pairs
on one problem, and many problems of different sizes, with the pairs' Gram
products taken together.  Each pair is checked against the FP64 oracle's
optimum of eq. (1.3): relative dual-objective gap <= 1e-6 of the feasibly
projected alpha, the library's own Sec. 4 residual <= tol, and a weak-duality
certificate computed by the oracle."""
import numpy as np
import pytest

from oracle import kqr_oracle as O
from paper_2510_07929_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAIRS = [(0.1, 5e-3), (0.5, 1e-2), (0.9, 1e-1), (0.25, 3e-2)]


@pytest.fixture(scope="module")
def K_():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    return kqr


def _problems(sizes, p=8):
    """The batched workload's generator: the rbf_small recipe at p = 8 with
    problem b drawn from seed 1000 + b (RBF gamma = 1/p)."""
    return [W.rbf_small(n=n, p=p, seed=1000 + b) for b, n in enumerate(sizes)]


def _check_pair(wl, K, alpha, beta, kkt, tau, lam, tol=1e-7):
    assert kkt <= tol * 10
    ref = O.solve_dense(K, wl.y, tau, lam, tol=1e-10)
    a = O.project_feasible(alpha, tau)
    d_gpu = O.dual_objective(a, K @ a, wl.y, lam)
    d_ref = O.dual_objective(ref["alpha"], K @ ref["alpha"], wl.y, lam)
    assert abs(d_gpu - d_ref) / (1 + abs(d_ref)) <= 1e-6, (tau, lam, d_gpu, d_ref)
    cert = O.certified_gap(alpha, K, wl.y, tau, lam)
    assert 0 <= cert["gap"] <= 1e-3


def test_grid_pairs_match_oracle(K_):
    """Three problems of different sizes, four (tau, lambda) pairs each; CG
    products chosen automatically (FP64-class on this smooth kernel, whose
    spectrum lies mostly below FP32 resolution)."""
    taus = np.array([t for t, _ in PAIRS])
    lams = np.array([l for _, l in PAIRS])
    for wl in _problems([300, 517, 1000]):
        K = O.gram(wl.X, wl.X, wl.kind, wl.gamma)
        with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, cg_high=2, time_limit_s=120.0) as prob:
            alpha, beta, kkt, status, infos = prob.solve_grid(taus, lams, tol=1e-7)
        assert alpha.shape == (wl.n, len(PAIRS))
        assert np.all(status == K_.OK), status
        for c, (tau, lam) in enumerate(PAIRS):
            assert infos[c]["eta_kkt"] == kkt[c] and infos[c]["pcg_iters"] > 0
            _check_pair(wl, K, alpha[:, c], beta[c], kkt[c], tau, lam)


def test_grid_fp64_class_products_match_oracle(K_):
    """The grid's shared products in FP64-class arithmetic (options.cg_high = 1):
    every CG, gradient and residual product of the pairs goes through the
    multi-right-hand-side FP64-class product."""
    wl = _problems([300], p=4)[0]
    K = O.gram(wl.X, wl.X, wl.kind, wl.gamma)
    pairs = [(0.3, 2e-2), (0.7, 5e-2)]
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, cg_high=1, time_limit_s=120.0) as prob:
        alpha, beta, kkt, status, infos = prob.solve_grid([t for t, _ in pairs], [l for _, l in pairs], tol=1e-7)
    assert np.all(status == K_.OK), status
    for c, (tau, lam) in enumerate(pairs):
        assert infos[c]["matvecs_fp32"] == 0 and infos[c]["cg_high_used"] == 1
        _check_pair(wl, K, alpha[:, c], beta[c], kkt[c], tau, lam)


def test_grid_batch_over_problems_matches_single_problem_grids(K_):
    """kqr_solve_grid_batch over three problems equals (to the tolerance) each
    problem's own grid, and every pair meets the oracle's optimum."""
    taus = np.array([t for t, _ in PAIRS])
    lams = np.array([l for _, l in PAIRS])
    wls = _problems([257, 640, 129])
    probs = [K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, cg_high=2, time_limit_s=120.0) for wl in wls]
    try:
        out = K_.solve_grid_batch(probs, taus, lams, tol=1e-7, workers=2)
    finally:
        for p in probs:
            p.close()
    for wl, (alpha, beta, kkt, status) in zip(wls, out):
        K = O.gram(wl.X, wl.X, wl.kind, wl.gamma)
        assert np.all(status == K_.OK), status
        for c, (tau, lam) in enumerate(PAIRS):
            _check_pair(wl, K, alpha[:, c], beta[c], kkt[c], tau, lam)


def test_grid_pair_statuses_are_independent(K_):
    """A pair that hits its iteration cap reports KQR_NOT_CONVERGED with its
    last iterate while the other pairs converge; the call itself returns OK."""
    wl = _problems([400])[0]
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, alm_maxit=2, admm_maxit=3, cg_high=2) as prob:
        alpha, beta, kkt, status, infos = prob.solve_grid([0.5, 0.5], [1.0, 1e-3], tol=1e-9)
    assert set(status.tolist()) <= {K_.OK, K_.NOT_CONVERGED}
    assert status[1] == K_.NOT_CONVERGED and np.all(np.isfinite(alpha[:, 1])) and kkt[1] > 1e-9


def test_grid_rejects_bad_arguments(K_):
    wl = _problems([100])[0]
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma) as prob:
        for taus, lams in (([0.0], [1e-2]), ([0.5], [-1.0]), ([1.0], [1.0])):
            with pytest.raises(K_.KQRError) as e:
                prob.solve_grid(taus, lams)
            assert e.value.status == K_.INVALID_ARG
