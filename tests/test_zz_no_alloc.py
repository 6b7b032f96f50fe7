"""The allocation-free FP32 Gram product (kqr_kmatvec_fp32_noalloc_dev).

It serves callers that cannot allocate device memory when they need a
product (a fully pre-reserved memory pool, an allocator callback, a loop that
must not synchronise on cudaMalloc): its scratch is a static device array.
Checked against the oracle (1e-5 of max|K V|, the FP32 contract) and against
the allocating entry point, for both kernels (the RBF path of this entry point
is the CUDA-core kernel, the allocating one defaults to tcgen05), two calls in
a row sharing the static array.  This file is collected last so that a run
stopping at its first failure has already run every other test; it also
passes on its own in a fresh process."""
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


@pytest.mark.parametrize("kind", ["laplacian", "rbf"])
def test_noalloc_product_matches_oracle_and_allocating_entry_point(K_, kind):
    import torch

    wl = W.lap_large(n=3001, p=20, seed=2) if kind == "laplacian" else W.rbf_mid(n=3001, p=20, seed=2)
    with K_.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=8) as prob:
        for call, m in enumerate((3, 1, 8)):       # calls in a row share the static scratch
            Vh = W.random_vectors(wl.n, m, seed=20 + call)
            V = torch.from_numpy(Vh).cuda().contiguous()
            U_ref = torch.empty_like(V)
            U = torch.full_like(V, float("nan"))
            prob.kmatvec_dev(V, U_ref, K_.PREC_FP32)
            prob.kmatvec_noalloc_dev(V, U)
            torch.cuda.synchronize()
            assert prob.check_device() == K_.OK
            ref = O.kmatvec(wl.X, Vh, wl.kind, wl.gamma)
            got = U.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), (m, np.max(np.abs(got - ref)))
            assert np.max(np.abs(got - U_ref.cpu().numpy())) <= 1e-5 * np.max(np.abs(ref))


def test_noalloc_product_rejects_oversized_problems(K_):
    import torch

    n = 600_000                                    # ldn * 8 * 4 * 2 bytes > 32 MiB at m = 8
    rng = np.random.default_rng(0)
    X = rng.random((n, 2))
    y = rng.standard_normal(n)
    with K_.Problem(X, y, "rbf", 0.5, rank0=2) as prob:
        V = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
        U = torch.zeros_like(V)
        with pytest.raises(K_.KQRError) as e:
            prob.kmatvec_noalloc_dev(V, U)
        assert e.value.status == K_.INVALID_ARG
        assert "bytes of scratch" in str(e.value)
