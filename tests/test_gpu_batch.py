"""Batched multi-right-hand-side RBF products (kqr_batch_kmatmul) against the
oracle's Gram matrices, problem by problem.

The kernel computes in TF32 (coordinates, Gram entries and right-hand sides
rounded to TF32, FP32 accumulation), so each entry is compared with the bound
|U_ic - (K V)_ic| <= 2^-8 (K |V|)_ic: four times the 2^-10 that the two
roundings of each term (2^-11 each) and the perturbed coordinates give."""
import ctypes

import numpy as np
import pytest

from oracle import kqr_oracle as O

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


def _batch(sizes, p, seed):
    rng = np.random.default_rng(seed)
    Xs = [rng.random((n, p)) for n in sizes]
    gammas = rng.uniform(0.05, 1.0, size=len(sizes))
    return Xs, gammas


def _check(Xs, gammas, V, U, rows=None):
    off = np.concatenate([[0], np.cumsum([x.shape[0] for x in Xs])])
    worst = 0.0
    for b, (X, g) in enumerate(zip(Xs, gammas)):
        Vb = V[off[b]:off[b + 1]]
        idx = np.arange(X.shape[0]) if rows is None else rows[b]
        Kb = O.gram(X[idx], X, "rbf", g)
        ref = Kb @ Vb
        bound = 2.0 ** -8 * (Kb @ np.abs(Vb)) + 1e-12
        err = np.abs(U[off[b] + idx] - ref)
        assert np.all(err <= bound), (b, float((err / bound).max()))
        worst = max(worst, float((err / bound).max()))
    return worst


@pytest.mark.parametrize("p_in_smem", [False, True])
@pytest.mark.parametrize("sizes,p,m", [([1, 63, 129, 300, 517], 8, 64), ([130, 64, 65], 3, 7),
                                       ([700, 256], 20, 1), ([2, 1000], 32, 33)])
def test_batch_products_match_oracle(K_, sizes, p, m, p_in_smem):
    """Gram tile kept in tensor memory (default) or staged through shared memory."""
    Xs, gammas = _batch(sizes, p, seed=len(sizes) * 100 + p)
    V = np.random.default_rng(p).standard_normal((sum(sizes), m))
    with K_.Batch(Xs, gammas, p_in_smem=p_in_smem) as bt:
        U = bt.kmatmul(V)
        assert bt.launches >= 2
    _check(Xs, gammas, V, U)


def test_batch_products_c4_shape_sampled_rows(K_):
    """64 problems, n_b ~ U{1000..20000}, p = 8, gamma = 1/8, 64 right-hand
    sides (the batched workload at full size); 24 sampled rows per problem."""
    rng = np.random.default_rng(4)
    sizes = rng.integers(1000, 20001, size=64).tolist()
    Xs = [rng.random((n, 8)) for n in sizes]
    V = rng.standard_normal((sum(sizes), 64))
    with K_.Batch(Xs, 0.125) as bt:
        U = bt.kmatmul(V)
    rows = [np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 22)])) for n in sizes]
    _check(Xs, np.full(64, 0.125), V, U, rows)


def test_batch_device_entry_matches_host_entry(K_):
    import torch

    Xs, gammas = _batch([333, 129], 5, seed=9)
    V = np.random.default_rng(1).standard_normal((462, 16))
    with K_.Batch(Xs, gammas) as bt:
        U = bt.kmatmul(V)
        Vd = torch.tensor(V, device="cuda")
        Ud = torch.empty_like(Vd)
        bt.kmatmul_dev(Vd, Ud)
        torch.cuda.synchronize()
    assert np.array_equal(Ud.cpu().numpy(), U)


def test_batch_rejects_bad_arguments(K_):
    lib = K_.lib()
    rng = np.random.default_rng(0)
    with pytest.raises(K_.KQRError):
        K_.Batch([rng.random((10, 33))], 1.0)                # p > 32
    with pytest.raises(K_.KQRError):
        K_.Batch([rng.random((10, 3)), np.zeros((0, 3))], 1.0)   # empty problem
    with pytest.raises(K_.KQRError):
        K_.Batch([rng.random((10, 3))], -1.0)                # gamma <= 0
    with K_.Batch([rng.random((10, 3))], 1.0) as bt:
        with pytest.raises(K_.KQRError):
            bt.kmatmul(np.zeros((10, 65)))                   # m > 64
        v = np.zeros(10)
        u = np.zeros(10)
        st = lib.kqr_kmatvec(bt._h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, K_.PREC_FP32)
        assert st == K_.INVALID_ARG                          # single-problem call on a batch handle
