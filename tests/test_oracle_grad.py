"""Pins for the oracle's held-out-loss gradient: central finite differences
of the oracle's own tightly solved loss (an independent route: no adjoint, no
explicit derivative matrices)."""
import numpy as np
import pytest

from oracle import kqr_oracle as O


def _problem(seed=0, n=36, nh=25, p=3):
    rng = np.random.default_rng(seed)
    X = rng.random((n, p))
    y = np.sin(2 * np.pi * X[:, 0]) + 0.3 * rng.standard_normal(n)
    Xh = rng.random((nh, p))
    yh = np.sin(2 * np.pi * Xh[:, 0]) + 0.3 * rng.standard_normal(nh)
    return X, y, Xh, yh


@pytest.mark.parametrize("seed,tau,lam,gamma", [(0, 0.5, 0.05, 2.0), (1, 0.3, 0.2, 1.0)])
def test_heldout_gradient_matches_finite_differences(seed, tau, lam, gamma):
    X, y, Xh, yh = _problem(seed)
    gr = O.heldout_grad(X, y, Xh, yh, gamma, tau, lam)
    loss = lambda Xv, gm, lm: O.heldout_loss(Xv, y, Xh, yh, gm, tau, lm)["loss"]
    h = 1e-5
    fd_lam = (loss(X, gamma, lam * np.exp(h)) - loss(X, gamma, lam * np.exp(-h))) / (2 * h)
    fd_gam = (loss(X, gamma * np.exp(h), lam) - loss(X, gamma * np.exp(-h), lam)) / (2 * h)
    scale = 1.0 + abs(gr["loss"])
    assert abs(fd_lam - gr["d_loglambda"]) <= 1e-5 * scale, (fd_lam, gr["d_loglambda"])
    assert abs(fd_gam - gr["d_loggamma"]) <= 1e-5 * scale, (fd_gam, gr["d_loggamma"])
    rng = np.random.default_rng(seed + 10)
    for _ in range(6):
        k, c = int(rng.integers(X.shape[0])), int(rng.integers(X.shape[1]))
        Xp, Xm = X.copy(), X.copy()
        Xp[k, c] += h
        Xm[k, c] -= h
        fd = (loss(Xp, gamma, lam) - loss(Xm, gamma, lam)) / (2 * h)
        assert abs(fd - gr["dX"][k, c]) <= 1e-5 * scale, (k, c, fd, gr["dX"][k, c])
    assert 0 < gr["elbow"].size < X.shape[0]      # a genuine active set, not all free or all bound
