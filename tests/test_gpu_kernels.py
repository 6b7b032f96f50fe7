"""GPU parity of the hot-path kernels against the FP64 oracle, through the C ABI.

Tolerances: FP32 Gram products within 1e-5 of max|K v| (FP32 entries, about
1e-7 relative each); the FP64-class product within 1e-12 of sum_j |K_ij v_j|
per row; FP64 vector kernels within 1e-11 relative."""
import json
import math
import os

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


def _data(kind, n, p, seed=0):
    if kind == "laplacian":
        wl = W.lap_large(n=n, p=p, seed=seed)
    else:
        wl = W.rbf_mid(n=n, p=p, seed=seed)
    return wl


GRAM_CASES = [("rbf", 2, 1), ("laplacian", 2, 1), ("rbf", 129, 3), ("laplacian", 129, 3),
              ("rbf", 1000, 10), ("laplacian", 1000, 10), ("rbf", 3001, 20), ("laplacian", 3001, 50),
              ("laplacian", 700, 64), ("rbf", 257, 64)]


PATHS = {"sym_tc": dict(symmetric_gram=1, rbf_tensor_cores=1, gram_store=0),
         "plain_tc": dict(symmetric_gram=0, rbf_tensor_cores=1, gram_store=0),
         "sym_cuda": dict(symmetric_gram=1, rbf_tensor_cores=0, gram_store=0),
         "plain_cuda": dict(symmetric_gram=0, rbf_tensor_cores=0, gram_store=0),
         "stored": dict(gram_store=1)}


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("kind,n,p", GRAM_CASES)
def test_gram_products_match_oracle(K_, kind, n, p, path):
    """Every Gram-product path: symmetric or plain tiles; RBF cross term on
    tcgen05 (three TF32 terms) or on FP32 CUDA cores."""
    if kind == "laplacian" and path.endswith("_cuda"):
        pytest.skip("the tensor-core switch applies to the RBF kernel only")
    if path == "stored" and n > 1000:
        pytest.skip("stored-K parity at larger n: test_stored_gram_matches_oracle")
    wl = _data(kind, n, p)
    with K_.Problem(wl.X, wl.y, kind, wl.gamma, **PATHS[path]) as prob:
        for m in (1, 3, 8):
            V = W.random_vectors(n, m, seed=m)
            ref = O.kmatvec(wl.X, V, kind, wl.gamma)
            absref = O.kmatvec(wl.X, np.abs(V), kind, wl.gamma)
            u32 = prob.kmatvec(V, K_.PREC_FP32)
            assert np.max(np.abs(u32 - ref)) <= 1e-5 * np.max(np.abs(ref)), (m, np.max(np.abs(u32 - ref)))
            uhp = prob.kmatvec(V, K_.PREC_HIGH)
            err = np.abs(uhp - ref) / absref
            assert np.max(err) <= 1e-12, (m, np.max(err))


@pytest.mark.parametrize("n,p", [(3001, 20), (1000, 10), (515, 50)])
def test_tf32_gram_error_is_bounded(K_, n, p):
    """KQR_PREC_TF32 (one TF32 tensor-core product for the cross term): the
    exponent's cross term has relative error ~2^-11, so entries err by about
    2^-11 * 2 |xs_i||xs_j|; check the product against that bound and that the
    FP32 form is far more accurate."""
    wl = _data("rbf", n, p)
    v = W.random_vectors(n, seed=3)
    ref = O.kmatvec(wl.X, v, "rbf", wl.gamma)
    absref = O.kmatvec(wl.X, np.abs(v), "rbf", wl.gamma)
    Xc = wl.X - wl.X.mean(0)
    s2 = wl.gamma / np.log(2.0) * np.max(np.sum(Xc * Xc, axis=1))   # max |xs|^2
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma) as prob:
        u_tf32 = prob.kmatvec(v, K_.PREC_TF32)
        u_fp32 = prob.kmatvec(v, K_.PREC_FP32)
    err_tf32 = np.max(np.abs(u_tf32 - ref) / absref)
    err_fp32 = np.max(np.abs(u_fp32 - ref) / absref)
    bound = 2.0 ** -10 * 2 * s2 * np.log(2.0) + 1e-5
    assert err_tf32 <= bound, (err_tf32, bound)
    assert err_fp32 <= 1e-5
    assert err_fp32 < err_tf32


@pytest.mark.parametrize("n,p", [(3001, 20), (515, 50), (257, 3)])
def test_bf16_gram_error_is_bounded(K_, n, p):
    """KQR_PREC_BF16 (coordinates rounded to bf16, 2^-9 each, one bf16 product
    for the cross term): the cross term errs by at most 2^-8 |xs_i||xs_j|, so
    entries err by about 2^-7 |xs|^2 ln 2 relative; check that bound (2x margin)
    and that TF32 is more accurate."""
    wl = _data("rbf", n, p)
    v = W.random_vectors(n, seed=4)
    ref = O.kmatvec(wl.X, v, "rbf", wl.gamma)
    absref = O.kmatvec(wl.X, np.abs(v), "rbf", wl.gamma)
    Xc = wl.X - wl.X.mean(0)
    s2 = wl.gamma / np.log(2.0) * np.max(np.sum(Xc * Xc, axis=1))   # max |xs|^2
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma) as prob:
        u_bf16 = prob.kmatvec(v, K_.PREC_BF16)
        u_tf32 = prob.kmatvec(v, K_.PREC_TF32)
        V3 = W.random_vectors(n, 3, seed=5)
        u3 = prob.kmatvec(V3, K_.PREC_BF16)
    err_bf16 = np.max(np.abs(u_bf16 - ref) / absref)
    err_tf32 = np.max(np.abs(u_tf32 - ref) / absref)
    bound = 2.0 ** -6 * s2 * np.log(2.0) + 1e-5
    assert err_bf16 <= bound, (err_bf16, bound)
    assert err_tf32 < err_bf16
    ref3 = O.kmatvec(wl.X, V3, "rbf", wl.gamma)
    abs3 = O.kmatvec(wl.X, np.abs(V3), "rbf", wl.gamma)
    assert np.max(np.abs(u3 - ref3) / abs3) <= bound


def test_gram_device_entry_and_stream(K_):
    import torch

    wl = _data("laplacian", 1500, 12, seed=4)
    v = W.random_vectors(1500, seed=9)
    ref = O.kmatvec(wl.X, v, "laplacian", wl.gamma)
    with K_.Problem(wl.X, wl.y, "laplacian", wl.gamma) as prob:
        s = torch.cuda.Stream()
        V = torch.from_numpy(v).cuda()
        U = torch.empty_like(V)
        prob.kmatvec_dev(V, U, K_.PREC_HIGH, stream=s)
        s.synchronize()
        assert np.max(np.abs(U.cpu().numpy() - ref)) <= 1e-11 * np.max(np.abs(ref))
        before = prob.launches
        prob.kmatvec_dev(V, U, K_.PREC_FP32)
        torch.cuda.synchronize()
        assert prob.launches > before


def test_gram_full_size_sampled_rows(K_):
    """The n = 200000, p = 50 Laplacian workload in the launch configuration
    the benchmark uses: sampled rows of K v against the oracle row by row."""
    wl = W.lap_large()
    v = W.random_vectors(wl.n, seed=11)
    rows = np.random.default_rng(5).choice(wl.n, 24, replace=False)
    ref = O.kmatvec(wl.X, v, wl.kind, wl.gamma, rows=rows)
    absref = O.kmatvec(wl.X, np.abs(v), wl.kind, wl.gamma, rows=rows)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=16, gram_store=0) as prob:
        uhp = prob.kmatvec(v, K_.PREC_HIGH)
        u32 = prob.kmatvec(v, K_.PREC_FP32)
    assert np.max(np.abs(uhp[rows] - ref) / absref) <= 1e-12
    assert np.max(np.abs(u32[rows] - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_rbf_full_size_sampled_rows_symmetric_tiles(K_):
    """The n = 50000, p = 20 RBF workload on the default single-vector path
    (symmetric tcgen05 tiles, each off-diagonal tile used for its row and its
    column sums): sampled rows of K v against the oracle."""
    wl = W.rbf_mid()
    v = W.random_vectors(wl.n, seed=12)
    rows = np.random.default_rng(6).choice(wl.n, 32, replace=False)
    ref = O.kmatvec(wl.X, v, wl.kind, wl.gamma, rows=rows)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=16, gram_store=0) as prob:
        u32 = prob.kmatvec(v, K_.PREC_FP32)
    assert np.max(np.abs(u32[rows] - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("path", ["sym_tc", "plain_tc"])
def test_rbf_tiles_without_row_folding(K_, path):
    """One far outlier puts max_i gamma log2(e) |x_i - mean|^2 above 60, so the
    tensor-core tiles keep exp2(-n_i) inside each entry instead of folding it
    into the row and column factors (exp2(n_i) would overflow FP32 there)."""
    rng = np.random.default_rng(21)
    n, p, gamma = 1000, 10, 0.1
    X = rng.standard_normal((n, p))
    X[7, 0] += 25.0
    xs2 = gamma * math.log2(math.e) * np.sum((X - X.mean(axis=0)) ** 2, axis=1)
    assert xs2.max() > 60.0
    y = rng.standard_normal(n)
    with K_.Problem(X, y, "rbf", gamma, **PATHS[path]) as prob:
        for m in (1, 3):
            V = W.random_vectors(n, m, seed=30 + m)
            ref = O.kmatvec(X, V, "rbf", gamma)
            u32 = prob.kmatvec(V, K_.PREC_FP32)
            assert np.max(np.abs(u32 - ref)) <= 1e-5 * np.max(np.abs(ref)), (m, np.max(np.abs(u32 - ref)))


@pytest.mark.parametrize("kind,n,p", [("rbf", 2000, 10), ("laplacian", 1500, 50), ("rbf", 700, 2)])
def test_rpcholesky_factor_and_rank_match_oracle(K_, kind, n, p):
    wl = W.rbf_small(n=n, p=p) if kind == "rbf" else W.lap_large(n=n, p=p)
    r0 = int(np.ceil(np.sqrt(n)))
    u = W.pivot_uniforms(r0, seed=77)
    with K_.Problem(wl.X, wl.y, kind, wl.gamma, pivot_uniforms=u, xi=1e-3) as prob:
        F, piv, r, rr0 = prob.factor()
    K = O.gram(wl.X, wl.X, kind, wl.gamma)
    F0, piv_o = O.rpcholesky(lambda s: K[:, s], np.diag(K), r0, u)
    assert rr0 == piv_o.size
    np.testing.assert_array_equal(piv, piv_o)
    assert r == O.rank_from_spectrum(F0, 1e-3)
    np.testing.assert_allclose(F, F0[:, :r], atol=2e-6 * np.max(np.abs(F0)))


def test_woodbury_apply_matches_lemma1(K_):
    import torch

    wl = W.rbf_small(n=1200)
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma) as prob:
        F, _, r, _ = prob.factor()
        rng = np.random.default_rng(3)
        for L, gam in ((rng.uniform(1e-3, 1.0, wl.n), 0.3), (np.where(rng.random(wl.n) < 0.5, 1e-7, 2e-2), 1e-4)):
            rv = rng.standard_normal(wl.n)
            out = torch.empty(wl.n, dtype=torch.float64, device="cuda")
            prob.precond_apply_dev(torch.from_numpy(L).cuda(), gam, torch.from_numpy(rv).cuda(), out)
            ref = O.woodbury_apply(F.astype(np.float64), L, gam, rv)
            assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_pcg_solves_newton_system(K_, precond):
    import torch

    wl = W.lap_large(n=1500, p=20)
    K = O.gram(wl.X, wl.X, wl.kind, wl.gamma)
    rng = np.random.default_rng(4)
    L = np.where(rng.random(wl.n) < 0.6, 1e-3, 5e-2)
    gam = 0.05
    b = rng.standard_normal(wl.n)
    A = K + gam * np.ones((wl.n, wl.n)) + np.diag(L)
    x_ref = np.linalg.solve(A, b)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, precond=precond) as prob:
        x = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
        its = prob.pcg_dev(torch.from_numpy(L).cuda(), gam, torch.from_numpy(b).cuda(), x, 1e-9 * np.linalg.norm(b),
                           3000)
    assert 0 < its < 3000
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-4 * np.linalg.norm(x_ref)


def test_box_grad_matches_eq_2_3(K_):
    import torch

    wl = W.rbf_small(n=777)
    rng = np.random.default_rng(8)
    tau, lam, sigma, beta, eps = 0.3, 0.02, 2.5, -0.4, 1e-3
    alpha = rng.uniform(-1.2, 0.8, wl.n)
    z = rng.standard_normal(wl.n)
    # put some w exactly on the box boundary
    z[:5] = sigma * (tau - alpha[:5])
    z[5:10] = sigma * (tau - 1.0 - alpha[5:10])
    Ka = rng.standard_normal(wl.n)
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma) as prob:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        v, S, g, L = (torch.empty(wl.n, dtype=torch.float64, device="cuda") for _ in range(4))
        g2 = prob.box_grad_dev(t(alpha), t(z), t(Ka), beta, sigma, tau, lam, eps, v, S, g, L)
    w = alpha + z / sigma
    np.testing.assert_allclose(v.cpu().numpy(), O.proj_box(w, tau), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(S.cpu().numpy(), O.jacobian_diag(w, tau))
    gref = O.grad_phi(alpha, Ka, wl.y, beta, z, sigma, tau, lam)
    np.testing.assert_allclose(g.cpu().numpy(), gref, rtol=1e-11, atol=1e-11 * np.max(np.abs(gref)))
    np.testing.assert_allclose(L.cpu().numpy(), O.newton_diag(w, tau, sigma, lam, eps), rtol=1e-14)
    assert g2 == pytest.approx(float(gref @ gref), rel=1e-10)


def test_kkt_residuals_match_sec4(K_):
    wl = W.lap_large(n=900, p=8)
    rng = np.random.default_rng(2)
    alpha = rng.uniform(wl.tau - 1, wl.tau, wl.n)
    v = O.proj_box(alpha + 1e-3 * rng.standard_normal(wl.n), wl.tau)
    z = rng.standard_normal(wl.n)
    beta = 0.7
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma) as prob:
        got = prob.kkt(alpha, v, beta, z, wl.tau, wl.lam)
    K = O.gram(wl.X, wl.X, wl.kind, wl.gamma)
    ref = O.kkt_residuals(alpha, v, beta, z, wl.y, K @ alpha, wl.tau, wl.lam)
    for key in ("eta_p", "eta_d", "eta_c", "eta_kkt", "eta_gap", "obj_p", "obj_d"):
        assert got[key] == pytest.approx(ref[key], rel=1e-9), key


def test_invalid_arguments_are_rejected(K_):
    wl = W.rbf_small(n=50)
    with pytest.raises(K_.KQRError) as e:
        K_.Problem(wl.X, wl.y, "rbf", -1.0)
    assert e.value.status == K_.INVALID_ARG
    y = wl.y.copy()
    y[3] = np.nan
    with pytest.raises(K_.KQRError):
        K_.Problem(wl.X, y, "rbf", 0.1)
    with pytest.raises(K_.KQRError):
        K_.Problem(np.zeros((10, 65)), np.zeros(10), "rbf", 0.1)
    with pytest.raises(K_.KQRError):
        K_.Problem(wl.X[:1], wl.y[:1], "rbf", 0.1)
    with K_.Problem(wl.X, wl.y, "rbf", 0.1) as prob:
        for tau, lam in ((0.0, 0.1), (1.0, 0.1), (0.5, 0.0), (0.5, -1.0)):
            with pytest.raises(K_.KQRError) as e:
                prob.solve(tau, lam)
            assert e.value.status == K_.INVALID_ARG
        with pytest.raises(K_.KQRError):
            prob.kmatvec(np.zeros((50, 9)))


def test_kkt_residuals_three_point_golden(K_):
    """The hand-computed Sec. 4 residuals of tests/golden/kkt_three_point.json
    (z != 0, alpha != v, 1^T alpha != 0) through kqr_kkt."""
    c = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kkt_three_point.json")))
    env = {"sqrt": math.sqrt, "log": math.log}
    with K_.Problem(np.array(c["x"]), np.array(c["y"]), c["kind"], eval(c["gamma"], env), rank0=2) as prob:
        got = prob.kkt(np.array(c["alpha"]), np.array(c["v"]), c["beta"], np.array(c["z"]), c["tau"], c["lam"])
    for key, expr in c["expected"].items():
        assert got[key] == pytest.approx(eval(expr, env), rel=1e-12), key


def test_pcg_reports_unconverged(K_):
    """kqr_pcg_dev stopped by maxit before its tolerance returns
    KQR_NOT_CONVERGED (x holds the last iterate), not KQR_OK."""
    import torch

    wl = W.lap_large(n=900, p=10)
    rng = np.random.default_rng(6)
    L = np.full(wl.n, 1e-4)
    b = rng.standard_normal(wl.n)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, precond=2) as prob:
        x = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
        with pytest.raises(K_.KQRError) as e:
            prob.pcg_dev(torch.from_numpy(L).cuda(), 1e-4, torch.from_numpy(b).cuda(), x, 1e-14, 2)
        assert e.value.status == K_.NOT_CONVERGED and "maxit" in str(e.value)
        assert np.all(np.isfinite(x.cpu().numpy())) and float(x.abs().sum()) > 0


def test_bounded_wait_timeout_is_reported(K_):
    """A kernel that gives up a bounded wait (here on a barrier nothing
    completes, with no copy in flight) leaves the timeout in the device error
    word; kqr_check_device reports it once and the context stays usable."""
    wl = W.rbf_small(n=300)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma) as prob:
        assert prob.check_device() == K_.OK
        prob.test_bounded_wait(64)
        assert prob.check_device() == K_.DEVICE_WAIT_TIMEOUT
        assert prob.check_device() == K_.OK
        v = W.random_vectors(wl.n, seed=2)
        ref = O.kmatvec(wl.X, v, wl.kind, wl.gamma)
        assert np.max(np.abs(prob.kmatvec(v) - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind,n,p", [("rbf", 2000, 10), ("laplacian", 2000, 50), ("rbf", 20000, 20),
                                      ("laplacian", 20000, 50), ("rbf", 130, 3), ("laplacian", 257, 4)])
def test_stored_gram_matches_oracle(K_, kind, n, p):
    """The stored-K product (packed upper-triangle tiles filled once, then
    streamed; options.gram_store = 1) against the FP64 oracle (the C form at
    n = 20000) and against the on-the-fly symmetric tiles, over two products
    in a row on one handle."""
    from oracle import native as N

    wl = _data(kind, n, p, seed=3)
    with K_.Problem(wl.X, wl.y, kind, wl.gamma, gram_store=1, rank0=8) as prob, \
            K_.Problem(wl.X, wl.y, kind, wl.gamma, gram_store=0, rank0=8) as fly:
        for seed in (1, 2):
            v = W.random_vectors(n, seed=seed)
            ref = N.kmatvec(wl.X, v, kind, wl.gamma)
            u = prob.kmatvec(v, K_.PREC_FP32)
            assert np.max(np.abs(u - ref)) <= 1e-5 * np.max(np.abs(ref)), np.max(np.abs(u - ref))
            assert np.max(np.abs(u - fly.kmatvec(v, K_.PREC_FP32))) <= 1e-5 * np.max(np.abs(ref))
        prob.profile(True)
        prob.kmatvec(v, K_.PREC_FP32)
        launches, ms = prob.profile_read(2)
        assert launches == 1 and ms > 0


def test_stored_gram_falls_back_when_not_asked_or_too_large(K_):
    """gram_store = 0 never stores; the automatic mode stores small problems, and
    large ones unless their on-the-fly tiles are the faster product."""
    wl = _data("rbf", 500, 4)
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma, gram_store=0) as prob:
        prob.kmatvec(W.random_vectors(500))
        prob.profile(True)
        prob.kmatvec(W.random_vectors(500))
        assert prob.profile_read(2)[0] == 0
        _, _, _, info = prob.solve(0.5, 1e-2, 1e-6)
        assert info["gram_stored"] == 0
    with K_.Problem(wl.X, wl.y, "rbf", wl.gamma) as prob:
        _, _, _, info = prob.solve(0.5, 1e-2, 1e-6)
        assert info["gram_stored"] == 1
    # past 64 MB of stored tiles (n = 6400: 1275 tiles, 83.6 MB) the automatic mode keeps
    # RBF kernels with p <= 32 on the symmetric tensor-core tiles, and stores Laplacian ones
    for kind, stored in (("rbf", 0), ("laplacian", 1)):
        wl = _data(kind, 6400, 8)
        with K_.Problem(wl.X, wl.y, kind, wl.gamma, rank0=8) as prob:
            prob.profile(True)
            prob.kmatvec(W.random_vectors(6400))
            assert prob.profile_read(2)[0] == stored, kind
