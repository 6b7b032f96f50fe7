"""Loader for the oracle's plain-C FP64 kernel products (``kernel_native.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  ``build()`` compiles
the C file with gcc and OpenMP into ``oracle/_build/liboracle_native.so``;
``kmatvec`` and ``gram`` call it through ctypes.  Same definitions as
``kqr_oracle.kmatvec`` / ``kqr_oracle.gram`` (Sec. 1 kernel entries), pinned
against them by the CPU tests; the C form exists for the sizes numpy cannot
reach in seconds (a full K.v at n = 200000).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kernel_native.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle_native.so")
KINDS = {"rbf": 0, "laplacian": 1}

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"gcc failed on {SRC}:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        l = ctypes.CDLL(build())
        D, I64, P = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        l.oracle_kmatvec.restype = ctypes.c_int
        l.oracle_kmatvec.argtypes = [P, I64, I64, ctypes.c_int, D, P, I64, P, I64, P, ctypes.c_int]
        l.oracle_gram.restype = ctypes.c_int
        l.oracle_gram.argtypes = [P, I64, P, I64, I64, ctypes.c_int, D, P, ctypes.c_int]
        l.oracle_threads.restype = ctypes.c_int
        l.oracle_threads.argtypes = []
        _lib = l
    return _lib


def threads() -> int:
    """Threads the OpenMP regions use (all host cores unless OMP_NUM_THREADS says otherwise)."""
    return int(lib().oracle_threads())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def kmatvec(X, V, kind: str, gamma: float, rows=None, threads: int = 0) -> np.ndarray:
    """u = K[rows, :] @ V in FP64 with K from its definition (the C form of
    ``kqr_oracle.kmatvec``).  ``V`` is (n,) or (n, m)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    Vm = np.ascontiguousarray(V[:, None] if vec else V)
    n, p = X.shape
    idx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = n if idx is None else idx.size
    U = np.empty((nrows, Vm.shape[1]), dtype=np.float64)
    st = lib().oracle_kmatvec(_ptr(X), n, p, KINDS[kind], float(gamma), _ptr(Vm), Vm.shape[1],
                              None if idx is None else _ptr(idx), nrows, _ptr(U), int(threads))
    if st != 0:
        raise MemoryError("oracle_kmatvec: out of host memory")
    return U[:, 0] if vec else U


def gram(X, Z, kind: str, gamma: float, threads: int = 0) -> np.ndarray:
    """K[i, j] = k(x_i, z_j) in FP64 (the C form of ``kqr_oracle.gram``)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    G = np.empty((X.shape[0], Z.shape[0]), dtype=np.float64)
    st = lib().oracle_gram(_ptr(X), X.shape[0], _ptr(Z), Z.shape[0], X.shape[1], KINDS[kind], float(gamma),
                           _ptr(G), int(threads))
    if st != 0:
        raise MemoryError("oracle_gram: out of host memory")
    return G
