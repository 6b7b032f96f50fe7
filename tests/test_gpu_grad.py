"""Held-out loss gradients on the GPU (kqr_heldout_grad) against the oracle's
dense implicit-differentiation formula, and against central finite
differences of GPU solves at a size the dense formula cannot reach."""
import numpy as np
import pytest

from oracle import kqr_oracle as O
from paper_2510_07929_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K_():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    return kqr


def _split(n, nh, p, seed, tau, lam):
    tr = W.rbf_small(n=n, p=p, seed=seed, tau=tau, lam=lam)
    ho = W.rbf_small(n=nh, p=p, seed=seed + 1000, tau=tau, lam=lam)
    return tr, ho.X, ho.y


@pytest.mark.parametrize("n,nh,p,tau,lam,gamma,tc", [(300, 200, 4, 0.5, 1e-2, 0.5, 1),
                                                     (257, 131, 3, 0.3, 5e-2, 1.0, 0),
                                                     (390, 170, 6, 0.7, 2e-2, 0.25, 1)])
def test_heldout_grad_matches_oracle(K_, n, nh, p, tau, lam, gamma, tc):
    tr, Xh, yh = _split(n, nh, p, 3, tau, lam)
    ref = O.heldout_grad(tr.X, tr.y, Xh, yh, gamma, tau, lam)
    with K_.Problem(tr.X, tr.y, "rbf", gamma, rbf_tensor_cores=tc) as prob:
        prob.solve(tau, lam, 1e-8)
        loss, dg, dl, dX = prob.heldout_grad(Xh, yh)
    scale = 1.0 + abs(ref["loss"])
    assert abs(loss - ref["loss"]) <= 1e-7 * scale, (loss, ref["loss"])
    # FP32 Gram products in the adjoint terms: relative 1e-4 of the gradient's scale
    assert abs(dl - ref["d_loglambda"]) <= 1e-4 * scale, (dl, ref["d_loglambda"])
    assert abs(dg - ref["d_loggamma"]) <= 1e-4 * scale, (dg, ref["d_loggamma"])
    err = np.abs(dX - ref["dX"]).max()
    assert err <= 1e-4 * (1.0 + np.abs(ref["dX"]).max()), err


def test_heldout_grad_sixteen_features_matches_oracle(K_):
    """p = 16, n = 1500 (+ 400 held-out), gamma = 0.25, lambda = 0.1: about a
    quarter of the points on the elbow; scalar derivatives against the oracle."""
    tau, lam, gamma = 0.5, 0.1, 0.25
    tr, Xh, yh = _split(1500, 400, 16, 0, tau, lam)
    ref = O.heldout_grad(tr.X, tr.y, Xh, yh, gamma, tau, lam, tol=1e-10, want_dX=False)
    with K_.Problem(tr.X, tr.y, "rbf", gamma) as prob:
        prob.solve(tau, lam, 1e-8)
        loss, dg, dl, _ = prob.heldout_grad(Xh, yh, want_dX=False)
    scale = 1.0 + abs(ref["loss"])
    assert abs(loss - ref["loss"]) <= 1e-6 * scale, (loss, ref["loss"])
    assert abs(dl - ref["d_loglambda"]) <= 1e-4 * scale, (dl, ref["d_loglambda"])
    assert abs(dg - ref["d_loggamma"]) <= 1e-4 * scale, (dg, ref["d_loggamma"])


def test_heldout_grad_finite_differences(K_):
    """n = 3000 training and 750 held-out points, p = 16, gamma = 0.25,
    lambda = 0.1 (the gradient workload's generator and constants at a smaller
    n): log-lambda and log-gamma derivatives against central differences of GPU
    solves.  The loss is piecewise smooth: its slope changes where a training
    point enters or leaves the elbow set or a held-out residual changes sign.
    The test checks, from the solutions at +-h (oracle predictions of the
    held-out points), whether the step crossed such a kink; without one the
    difference must agree to 2e-4 of (1 + |loss|), across one to 1e-3."""
    tau, lam, gamma = 0.5, 0.1, 0.25
    tr, Xh, yh = _split(3000, 750, 16, 11, tau, lam)

    def at(gm, lm):
        with K_.Problem(tr.X, tr.y, "rbf", gm) as prob:
            alpha, beta, _, _ = prob.solve(tau, lm, 1e-9)
            loss, dg, dl, _ = prob.heldout_grad(Xh, yh, want_dX=False)
        f = O.predict(tr.X, alpha, beta, Xh, "rbf", gm, lm)
        elbow = frozenset(np.flatnonzero((alpha > tau - 1 + 1e-6) & (alpha < tau - 1e-6)).tolist())
        return loss, dg, dl, elbow, np.sign(yh - f)

    loss, dg, dl, E0, s0 = at(gamma, lam)
    h = 1e-4
    pts = {"l+": at(gamma, lam * np.exp(h)), "l-": at(gamma, lam * np.exp(-h)),
           "g+": at(gamma * np.exp(h), lam), "g-": at(gamma * np.exp(-h), lam)}
    fd_l = (pts["l+"][0] - pts["l-"][0]) / (2 * h)
    fd_g = (pts["g+"][0] - pts["g-"][0]) / (2 * h)
    scale = 1.0 + abs(loss)
    for name, fd, ad in (("l", fd_l, dl), ("g", fd_g, dg)):
        kink = [k for k in (name + "+", name + "-") if pts[k][3] != E0 or np.any(pts[k][4] != s0)]
        tol = 1e-3 if kink else 2e-4
        assert abs(fd - ad) <= tol * scale, (name, fd, ad, kink)


def test_heldout_grad_rejects_bad_calls(K_):
    tr, Xh, yh = _split(200, 50, 3, 5, 0.5, 1e-2)
    with K_.Problem(tr.X, tr.y, "rbf", 0.5) as prob:
        with pytest.raises(K_.KQRError):
            prob.heldout_grad(Xh, yh)          # no solve yet
    lap = W.lap_large(n=300, p=4)
    with K_.Problem(lap.X, lap.y, "laplacian", lap.gamma) as prob:
        prob.solve(lap.tau, 1e-2, 1e-6)
        with pytest.raises(K_.KQRError):
            prob.heldout_grad(lap.X[:20], lap.y[:20])


def test_autograd_wrapper_matches_entry_point(K_):
    import torch

    tau, lam, gamma = 0.5, 2e-2, 0.4
    tr, Xh, yh = _split(400, 150, 5, 21, tau, lam)
    with K_.Problem(tr.X, tr.y, "rbf", gamma) as prob:
        prob.solve(tau, lam, 1e-8)
        loss, dg, dl, dX = prob.heldout_grad(Xh, yh)
    Xt = torch.tensor(tr.X, requires_grad=True)
    lg = torch.tensor(np.log(gamma), dtype=torch.float64, requires_grad=True)
    ll = torch.tensor(np.log(lam), dtype=torch.float64, requires_grad=True)
    out = K_.heldout_check_loss(Xt, tr.y, Xh, yh, lg, ll, tau, tol=1e-8)
    (2.0 * out).backward()
    # two independent solves to KKT 1e-8 (the FP32 products accumulate in no fixed order)
    assert float(out.detach()) == pytest.approx(loss, rel=1e-7)
    assert float(lg.grad) == pytest.approx(2 * dg, rel=1e-3, abs=1e-6)
    assert float(ll.grad) == pytest.approx(2 * dl, rel=1e-3, abs=1e-6)
    assert np.abs(Xt.grad.numpy() - 2 * dX).max() <= 1e-3 * (1 + np.abs(dX).max())
