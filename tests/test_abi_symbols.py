"""The C-ABI library loads without a GPU and exports every symbol kqr.h
declares; the binding knows a signature for each one.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kqr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(kqr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib_path():
    import shutil

    from paper_2510_07929_gb300 import build

    if shutil.which("nvcc") is None and not os.path.exists(build.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kqr_create", "kqr_solve", "kqr_kmatvec", "kqr_kmatvec_dev", "kqr_destroy",
                     "kqr_last_error", "kqr_box_grad_dev", "kqr_precond_apply_dev", "kqr_pcg_dev", "kqr_kkt",
                     "kqr_get_factor"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in kqr.h but not exported"


def test_binding_covers_every_symbol(lib_path):
    from paper_2510_07929_gb300 import kqr

    assert set(declared_functions()) == set(kqr.SIGNATURES)
    lib = kqr.load_library(lib_path)
    o = kqr.Options()
    lib.kqr_default_options(ctypes.byref(o))          # host-only call
    assert o.admm_maxit == 100 and o.alm_maxit == 1000 and abs(o.admm_tol - 1e-3) < 1e-18
    assert lib.kqr_status_string(4) == b"not converged"
    assert lib.kqr_n(None) == 0


def test_options_struct_layout_matches_c(lib_path):
    """The ctypes mirror of kqr_options has the C layout: defaults written by C
    land in the right Python fields."""
    from paper_2510_07929_gb300 import kqr

    o = kqr.default_options()
    assert o.xi == 1e-10 and o.seed == 12345 and o.gamma_admm == 1.618 and o.sigma_factor == 10.0
    assert o.tau1 == 1e-2 and o.tau2 == 1e-1 and o.pcg_maxit == 1000 and o.verbose == 0 and o.sigma_alm_scale == 1.0
    assert o.core_reuse_rtol == 1e-2 and o.symmetric_gram == 1 and o.rbf_tensor_cores == 1 and o.cg_tf32 == 0
    assert o.cg_high == 2 and o.gram_store == 2
    assert o.admm_cg_rtol == 3e-4 and o.admm_maxit == 100 and o.precond == 0 and o.rank0 == 0
