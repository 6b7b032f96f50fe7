"""ctypes binding of the kqr C ABI (``include/kqr.h``).

Argument marshalling only: every computation runs in the CUDA library
``_build/libkqr.so``.  Host arrays are numpy float64; device arrays are CUDA
torch tensors (float64, contiguous) passed by data pointer.  Importing this
module fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkqr.so")

RBF, LAPLACIAN = 0, 1
PREC_HIGH, PREC_FP32, PREC_TF32, PREC_BF16 = 0, 1, 2, 3
PRECOND_NYSTROM_DIAG, PRECOND_PAPER, PRECOND_NONE = 0, 1, 2
KIND = {"rbf": RBF, "laplacian": LAPLACIAN}

STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "not converged",
          5: "breakdown", 6: "time limit", 7: "device wait timeout"}
OK, INVALID_ARG, OOM, CUDA_ERROR, NOT_CONVERGED, BREAKDOWN, TIMEOUT, DEVICE_WAIT_TIMEOUT = range(8)


class Options(ctypes.Structure):
    _fields_ = [
        ("rank0", ctypes.c_int32), ("adaptive_rank", ctypes.c_int32), ("xi", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("pivot_uniforms", ctypes.POINTER(ctypes.c_double)),
        ("precond", ctypes.c_int32),
        ("sigma0", ctypes.c_double), ("gamma_admm", ctypes.c_double), ("admm_tol", ctypes.c_double), ("admm_cg_rtol", ctypes.c_double),
        ("admm_maxit", ctypes.c_int32), ("balance_every", ctypes.c_int32), ("balance_ratio", ctypes.c_double),
        ("balance_factor", ctypes.c_double),
        ("alm_maxit", ctypes.c_int32), ("sigma_alm_scale", ctypes.c_double), ("sigma_factor", ctypes.c_double), ("sigma_max", ctypes.c_double),
        ("eta_bar", ctypes.c_double), ("iota", ctypes.c_double), ("mu", ctypes.c_double), ("r_ls", ctypes.c_double),
        ("tau1", ctypes.c_double), ("tau2", ctypes.c_double),
        ("ssn_maxit", ctypes.c_int32), ("ls_maxit", ctypes.c_int32), ("pcg_maxit", ctypes.c_int32),
        ("core_reuse_rtol", ctypes.c_double),
        ("time_limit_s", ctypes.c_double), ("phase1_only", ctypes.c_int32),
        ("symmetric_gram", ctypes.c_int32), ("rbf_tensor_cores", ctypes.c_int32), ("cg_tf32", ctypes.c_int32),
        ("verbose", ctypes.c_int32), ("cg_high", ctypes.c_int32), ("gram_store", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("phase1_iters", ctypes.c_int32), ("phase2_iters", ctypes.c_int32), ("newton_steps", ctypes.c_int32),
        ("pcg_iters", ctypes.c_int32), ("matvecs_fp32", ctypes.c_int32), ("matvecs_high", ctypes.c_int32),
        ("matvecs_low", ctypes.c_int32),
        ("rank", ctypes.c_int32), ("core_builds", ctypes.c_int32), ("cg_truncations", ctypes.c_int32),
        ("eta_p", ctypes.c_double), ("eta_d", ctypes.c_double), ("eta_c", ctypes.c_double),
        ("eta_kkt", ctypes.c_double), ("eta_gap", ctypes.c_double), ("obj_p", ctypes.c_double),
        ("obj_d", ctypes.c_double), ("sigma_final", ctypes.c_double), ("seconds", ctypes.c_double),
        ("gram_stored", ctypes.c_int32), ("cg_high_used", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# Every symbol kqr.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_D = ctypes.c_double
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "kqr_default_options": (None, [ctypes.POINTER(Options)]),
    "kqr_set_allocator": (None, [_P, _P, _P]),
    "kqr_create": (ctypes.c_int, [_DP, _DP, _I64, _I64, ctypes.c_int, _D, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "kqr_solve": (ctypes.c_int, [_P, _D, _D, _D, _DP, _DP, _DP, ctypes.POINTER(Info)]),
    "kqr_get_state": (ctypes.c_int, [_P, _DP, _DP]),
    "kqr_solve_grid": (ctypes.c_int, [_P, _I64, _DP, _DP, _D, _DP, _DP, _DP, ctypes.POINTER(_I32),
                                      ctypes.POINTER(Info)]),
    "kqr_solve_grid_batch": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _DP, _DP, _D, _I32, _DP, _DP, _DP,
                                            ctypes.POINTER(_I32)]),
    "kqr_kmatvec": (ctypes.c_int, [_P, _DP, _DP, _I64, ctypes.c_int]),
    "kqr_kmatvec_dev": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, _P]),
    "kqr_kmatvec_fp32_noalloc_dev": (ctypes.c_int, [_P, _P, _P, _I64, _P]),
    "kqr_check_device": (ctypes.c_int, [_P]),
    "kqr_test_bounded_wait": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "kqr_box_grad_dev": (ctypes.c_int, [_P, _P, _P, _P, _D, _D, _D, _D, _D, _P, _P, _P, _P, _DP, _P]),
    "kqr_precond_apply_dev": (ctypes.c_int, [_P, _P, _D, _P, _P, _P]),
    "kqr_pcg_dev": (ctypes.c_int, [_P, _P, _D, _P, _P, _D, _I32, ctypes.POINTER(_I32), _P]),
    "kqr_kkt": (ctypes.c_int, [_P, _DP, _DP, _D, _DP, _D, _D, _DP]),
    "kqr_get_factor": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "kqr_refactor": (ctypes.c_int, [_P, _DP]),
    "kqr_heldout_grad": (ctypes.c_int, [_P, _DP, _DP, _DP, _I64, _DP, _DP, _DP, _DP]),
    "kqr_batch_create": (ctypes.c_int, [_DP, ctypes.POINTER(_I64), _I64, _I64, _DP, _I32, ctypes.POINTER(_P)]),
    "kqr_batch_kmatmul": (ctypes.c_int, [_P, _DP, _DP, _I64]),
    "kqr_batch_kmatmul_dev": (ctypes.c_int, [_P, _P, _P, _I64]),
    "kqr_profile": (ctypes.c_int, [_P, _I32]),
    "kqr_profile_read": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_I64), _DP]),
    "kqr_set_stream": (ctypes.c_int, [_P, _P]),
    "kqr_n": (_I64, [_P]),
    "kqr_p": (_I64, [_P]),
    "kqr_launch_count": (_I64, [_P]),
    "kqr_last_error": (ctypes.c_char_p, [_P]),
    "kqr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "kqr_destroy": (None, [_P]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -m paper_2510_07929_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class KQRError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def default_options(**overrides) -> Options:
    o = Options()
    lib().kqr_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _tptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device arguments must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Problem:
    """A kernel quantile regression problem on the current CUDA device
    (``kqr_create``): X (n x p) and y (n), kernel 'rbf' or 'laplacian', gamma."""

    def __init__(self, X, y, kind: str = "rbf", gamma: float = 1.0, options: Options | None = None,
                 pivot_uniforms=None, **opts):
        self._lib = lib()
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        if self.X.ndim != 2 or self.y.shape != (self.X.shape[0],):
            raise ValueError("X must be (n, p) and y (n,)")
        o = options if options is not None else default_options(**opts)
        self._uniforms = None
        if pivot_uniforms is not None:
            self._uniforms = np.ascontiguousarray(pivot_uniforms, dtype=np.float64)
            o.pivot_uniforms = _dptr(self._uniforms)
        self.options = o
        h = ctypes.c_void_p()
        n, p = self.X.shape
        st = self._lib.kqr_create(_dptr(self.X), _dptr(self.y), n, p, KIND[kind], float(gamma), ctypes.byref(o),
                                  ctypes.byref(h))
        self._h = h
        if st != OK:
            msg = self._lib.kqr_last_error(h).decode() if h.value else ""
            self.close()
            raise KQRError(st, msg)
        self.n, self.p, self.kind, self.gamma = n, p, kind, gamma

    def _check(self, st: int, allow=(OK,)):
        if st not in allow:
            raise KQRError(st, self._lib.kqr_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.kqr_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- the calls of the C ABI ------------------------------------------------
    def solve(self, tau: float, lam: float, tol: float = 1e-6, allow_not_converged: bool = False):
        alpha = np.empty(self.n)
        beta = ctypes.c_double()
        kkt = ctypes.c_double()
        info = Info()
        allow = (OK, NOT_CONVERGED, TIMEOUT) if allow_not_converged else (OK,)
        st = self._check(self._lib.kqr_solve(self._h, tau, lam, tol, _dptr(alpha), ctypes.byref(beta),
                                             ctypes.byref(kkt), ctypes.byref(info)), allow)
        d = info.as_dict()
        d["status"] = st
        return alpha, beta.value, kkt.value, d

    def solve_grid(self, taus, lambdas, tol: float = 1e-6):
        """kqr_solve_grid: every (taus[c], lambdas[c]) pair on this problem.  Returns
        alpha (n x m), beta (m), kkt (m), status (m) and the per-pair info dicts."""
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
        m = taus.size
        if lambdas.shape != taus.shape:
            raise ValueError("taus and lambdas must have the same length")
        alpha = np.empty((m, self.n))
        beta, kkt = np.empty(m), np.empty(m)
        status = np.empty(m, dtype=np.int32)
        infos = (Info * m)()
        self._check(self._lib.kqr_solve_grid(self._h, m, _dptr(taus), _dptr(lambdas), tol, _dptr(alpha), _dptr(beta),
                                             _dptr(kkt), status.ctypes.data_as(ctypes.POINTER(_I32)), infos))
        return alpha.T, beta, kkt, status, [i.as_dict() for i in infos]

    def state(self):
        v = np.empty(self.n)
        z = np.empty(self.n)
        self._check(self._lib.kqr_get_state(self._h, _dptr(v), _dptr(z)))
        return v, z

    def kmatvec(self, V, prec: int = PREC_FP32) -> np.ndarray:
        V = np.ascontiguousarray(V, dtype=np.float64)
        m = 1 if V.ndim == 1 else V.shape[1]
        U = np.empty_like(V)
        self._check(self._lib.kqr_kmatvec(self._h, _dptr(V), _dptr(U), m, prec))
        return U

    def kmatvec_dev(self, V, U, prec: int = PREC_FP32, stream=None):
        m = 1 if V.dim() == 1 else V.shape[1]
        self._check(self._lib.kqr_kmatvec_dev(self._h, _tptr(V), _tptr(U), m, prec, _stream_ptr(stream)))
        return U

    def kmatvec_noalloc_dev(self, V, U, stream=None):
        """FP32 U = K V through the entry point that allocates no device memory
        (kqr_kmatvec_fp32_noalloc_dev); V, U contiguous CUDA float64 tensors."""
        m = 1 if V.dim() == 1 else V.shape[1]
        self._check(self._lib.kqr_kmatvec_fp32_noalloc_dev(self._h, _tptr(V), _tptr(U), m, _stream_ptr(stream)))
        return U

    def check_device(self) -> int:
        """kqr_check_device: OK, or DEVICE_WAIT_TIMEOUT if a kernel gave up a bounded wait."""
        return int(self._lib.kqr_check_device(self._h))

    def test_bounded_wait(self, max_polls: int):
        self._check(self._lib.kqr_test_bounded_wait(self._h, max_polls))

    def box_grad_dev(self, alpha, z, Kalpha, beta, sigma, tau, lam, eps, v=None, S=None, grad=None, Ldiag=None,
                     stream=None):
        g2 = ctypes.c_double()
        self._check(self._lib.kqr_box_grad_dev(self._h, _tptr(alpha), _tptr(z), _tptr(Kalpha), beta, sigma, tau, lam,
                                               eps, _tptr(v), _tptr(S), _tptr(grad), _tptr(Ldiag),
                                               ctypes.byref(g2), _stream_ptr(stream)))
        return g2.value

    def precond_apply_dev(self, Ldiag, gam, r, out, stream=None):
        self._check(self._lib.kqr_precond_apply_dev(self._h, _tptr(Ldiag), gam, _tptr(r), _tptr(out),
                                                    _stream_ptr(stream)))
        return out

    def pcg_dev(self, Ldiag, gam, b, x, tol, maxit=1000, stream=None):
        it = ctypes.c_int32()
        self._check(self._lib.kqr_pcg_dev(self._h, _tptr(Ldiag), gam, _tptr(b), _tptr(x), tol, maxit,
                                          ctypes.byref(it), _stream_ptr(stream)))
        return it.value

    def kkt(self, alpha, v, beta, z, tau, lam) -> dict:
        out = np.empty(7)
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        vv = np.ascontiguousarray(v, dtype=np.float64)
        zz = np.ascontiguousarray(z, dtype=np.float64)
        self._check(self._lib.kqr_kkt(self._h, _dptr(a), _dptr(vv), beta, _dptr(zz), tau, lam, _dptr(out)))
        return dict(zip(["eta_p", "eta_d", "eta_c", "eta_kkt", "eta_gap", "obj_p", "obj_d"], out.tolist()))

    def factor(self):
        rank = ctypes.c_int32()
        rank0 = ctypes.c_int32()
        self._check(self._lib.kqr_get_factor(self._h, None, None, ctypes.byref(rank), ctypes.byref(rank0)))
        F = np.empty(max(1, rank.value * self.n), dtype=np.float32)
        piv = np.empty(max(1, rank0.value), dtype=np.int64)
        self._check(self._lib.kqr_get_factor(self._h, F.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                             piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None, None))
        F = F[:rank.value * self.n].reshape(rank.value, self.n).T
        return F, piv[:rank0.value], rank.value, rank0.value

    def heldout_grad(self, Xh, yh, want_dX: bool = True):
        """Held-out check loss of the last solve and its gradient with respect to
        (log gamma, log lambda, X) (kqr_heldout_grad)."""
        Xh = np.ascontiguousarray(Xh, dtype=np.float64)
        yh = np.ascontiguousarray(yh, dtype=np.float64)
        loss, dg, dl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        dX = np.empty_like(self.X) if want_dX else None
        self._check(self._lib.kqr_heldout_grad(self._h, _dptr(self.X), _dptr(Xh), _dptr(yh), Xh.shape[0],
                                               ctypes.byref(loss), ctypes.byref(dg), ctypes.byref(dl),
                                               _dptr(dX) if want_dX else None))
        return loss.value, dg.value, dl.value, dX

    def refactor(self, pivot_uniforms=None):
        u = None
        if pivot_uniforms is not None:
            self._uniforms = np.ascontiguousarray(pivot_uniforms, dtype=np.float64)
            u = _dptr(self._uniforms)
        self._check(self._lib.kqr_refactor(self._h, u))

    def profile(self, enable: bool = True):
        self._check(self._lib.kqr_profile(self._h, 1 if enable else 0))

    def profile_read(self, kernel_id: int):
        cnt = ctypes.c_int64()
        ms = ctypes.c_double()
        self._check(self._lib.kqr_profile_read(self._h, kernel_id, ctypes.byref(cnt), ctypes.byref(ms)))
        return cnt.value, ms.value

    def set_stream(self, stream):
        self._check(self._lib.kqr_set_stream(self._h, _stream_ptr(stream)))

    @property
    def launches(self) -> int:
        return int(self._lib.kqr_launch_count(self._h))


class Batch:
    """B independent RBF problems (X_b n_b x p, gamma_b) for batched products
    U_b = K_b V_b with up to 64 right-hand sides (kqr_batch_create)."""

    def __init__(self, Xs, gammas, p_in_smem: bool = False):
        self._lib = lib()
        self.sizes = [int(x.shape[0]) for x in Xs]
        self.p = int(Xs[0].shape[1])
        self.X = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in Xs]))
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.gammas = np.ascontiguousarray(np.broadcast_to(np.asarray(gammas, dtype=np.float64), (len(Xs),)))
        h = ctypes.c_void_p()
        st = self._lib.kqr_batch_create(_dptr(self.X), self.offsets.ctypes.data_as(ctypes.POINTER(_I64)), len(Xs),
                                        self.p, _dptr(self.gammas), 1 if p_in_smem else 0, ctypes.byref(h))
        self._h = h
        if st != OK:
            msg = self._lib.kqr_last_error(h).decode() if h.value else ""
            self.close()
            raise KQRError(st, msg)
        self.n = int(self.offsets[-1])

    def _check(self, st: int):
        if st != OK:
            raise KQRError(st, self._lib.kqr_last_error(self._h).decode())

    def kmatmul(self, V) -> np.ndarray:
        """V: (sum n_b, m) host array, rows stacked like X; returns U of the same shape."""
        V = np.ascontiguousarray(V, dtype=np.float64)
        V2 = V.reshape(self.n, -1)
        U = np.empty_like(V2)
        self._check(self._lib.kqr_batch_kmatmul(self._h, _dptr(V2), _dptr(U), V2.shape[1]))
        return U.reshape(V.shape)

    def kmatmul_dev(self, V, U):
        m = 1 if V.dim() == 1 else V.shape[1]
        self._check(self._lib.kqr_batch_kmatmul_dev(self._h, _tptr(V), _tptr(U), m))
        return U

    def set_stream(self, stream):
        self._check(self._lib.kqr_set_stream(self._h, _stream_ptr(stream)))

    def profile(self, enable: bool):
        self._check(self._lib.kqr_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        cnt, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(self._lib.kqr_profile_read(self._h, 0, ctypes.byref(cnt), ctypes.byref(ms)))
        return cnt.value, ms.value

    @property
    def launches(self) -> int:
        return int(self._lib.kqr_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.kqr_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_torch_alloc_refs = None


def use_torch_allocator():
    """Routes the library's device allocations through torch's CUDA caching
    allocator (for handles created afterwards)."""
    global _torch_alloc_refs
    import torch

    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

    def _alloc(nbytes, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(ptr, _ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    _torch_alloc_refs = (ALLOC(_alloc), FREE(_free))
    lib().kqr_set_allocator(ctypes.cast(_torch_alloc_refs[0], ctypes.c_void_p),
                            ctypes.cast(_torch_alloc_refs[1], ctypes.c_void_p), None)


def use_cuda_allocator():
    lib().kqr_set_allocator(None, None, None)


def heldout_check_loss(X, y, Xh, yh, log_gamma, log_lambda, tau: float, tol: float = 1e-8, **opts):
    """Held-out check loss of the RBF kernel quantile regression fitted on
    (X, y) at exp(log_gamma), exp(log_lambda), as a torch autograd function of
    (X, log_gamma, log_lambda).  The forward pass is one kqr_solve and the
    backward pass uses the gradients kqr_heldout_grad returns with the loss;
    X, log_gamma and log_lambda are float64 CPU tensors (log_* 0-d)."""
    import torch

    class _HeldoutLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, Xt, lg, ll):
            with Problem(Xt.detach().numpy(), y, "rbf", float(torch.exp(lg)), **opts) as prob:
                prob.solve(tau, float(torch.exp(ll)), tol)
                loss, dg, dl, dX = prob.heldout_grad(Xh, yh, want_dX=Xt.requires_grad)
            ctx.save_for_backward(torch.from_numpy(dX) if dX is not None else torch.zeros(0, dtype=torch.float64),
                                  torch.tensor(dg, dtype=torch.float64), torch.tensor(dl, dtype=torch.float64))
            ctx.want_dX = dX is not None
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, go):
            dX, dg, dl = ctx.saved_tensors
            return (go * dX if ctx.want_dX else None), go * dg, go * dl

    return _HeldoutLoss.apply(X, log_gamma, log_lambda)


def solve_grid_batch(problems, taus, lambdas, tol: float = 1e-6, workers: int = 4):
    """kqr_solve_grid_batch over Problem objects with the same (tau, lambda)
    pairs.  Returns per problem (alpha n_b x m, beta m, kkt m, status m)."""
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
    m, B = taus.size, len(problems)
    sizes = [p.n for p in problems]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    alpha = np.empty(int(off[-1]) * m)
    beta, kkt = np.empty((B, m)), np.empty((B, m))
    status = np.empty((B, m), dtype=np.int32)
    hs = (_P * B)(*[p._h.value for p in problems])
    st = lib().kqr_solve_grid_batch(hs, B, m, _dptr(taus), _dptr(lambdas), tol, workers, _dptr(alpha),
                                    _dptr(beta), _dptr(kkt), status.ctypes.data_as(ctypes.POINTER(_I32)))
    if st != OK:
        msgs = [lib().kqr_last_error(p._h).decode() for p in problems]
        raise KQRError(st, "; ".join(x for x in msgs if x))
    out = []
    for b in range(B):
        a = alpha[off[b] * m:off[b + 1] * m].reshape(m, sizes[b]).T
        out.append((a, beta[b], kkt[b], status[b]))
    return out
