"""Seeded synthetic inputs for the kernel quantile regression workloads.

This module holds only data recipes (point clouds, responses, and the uniform
random numbers RPCholesky consumes); none of the method's arithmetic.  Both
the CUDA path and the CPU oracle are fed from it.

Workloads (shapes and distributions of the paper's synthetic experiments,
scaled to the sizes this library targets):

* ``rbf_small``  n=2000,  p=10, x ~ U[0,1]^p,
  y = sin(2 pi x_1) + 0.5 x_2 + (0.2 + 0.3 x_1) eps, eps ~ N(0,1);
  RBF gamma = 1/p, tau = 0.5, lambda = 1e-2.
* ``rbf_mid``    n=50000, p=20, x ~ N(0, I_p), y = ||x||_2 / sqrt(p) + t_3 noise;
  RBF gamma = 1/p, tau in {0.1, 0.5, 0.9}, lambda = 1e-3.
* ``lap_large``  n=200000, p=50, x ~ U[-1,1]^p,
  y = sum_j sin(x_j) / sqrt(p) + (0.5 + |x_1|) N(0,1);
  Laplacian gamma = 1/p, tau = 0.25, lambda = 1e-4.
* ``yuan2006``   the p=2 generator of the paper's Sec. 4.1 (context runs).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray          # (n, p) float64, row-major
    y: np.ndarray          # (n,) float64
    kind: str              # "rbf" or "laplacian"
    gamma: float
    tau: float
    lam: float

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def p(self) -> int:
        return self.X.shape[1]


def rbf_small(n: int = 2000, p: int = 10, seed: int = 0, tau: float = 0.5, lam: float = 1e-2) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.random((n, p))
    eps = rng.standard_normal(n)
    y = np.sin(2.0 * np.pi * X[:, 0]) + 0.5 * X[:, 1] + (0.2 + 0.3 * X[:, 0]) * eps
    return Workload("rbf_small", X, y, "rbf", 1.0 / p, tau, lam)


def rbf_mid(n: int = 50000, p: int = 20, seed: int = 0, tau: float = 0.5, lam: float = 1e-3) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    y = np.linalg.norm(X, axis=1) / np.sqrt(p) + rng.standard_t(3, size=n)
    return Workload("rbf_mid", X, y, "rbf", 1.0 / p, tau, lam)


def lap_large(n: int = 200000, p: int = 50, seed: int = 0, tau: float = 0.25, lam: float = 1e-4) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(n, p))
    y = np.sin(X).sum(axis=1) / np.sqrt(p) + (0.5 + np.abs(X[:, 0])) * rng.standard_normal(n)
    return Workload("lap_large", X, y, "laplacian", 1.0 / p, tau, lam)


def yuan2006(n: int = 5000, seed: int = 0, gamma: float = 0.1, tau: float = 0.5, lam: float = 0.1) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.random((n, 2))
    a = 8.0 * ((X[:, 0] - 0.5) ** 2 + (X[:, 1] - 0.5) ** 2)
    b = 8.0 * ((X[:, 0] - 0.2) ** 2 + (X[:, 1] - 0.7) ** 2)
    c = 8.0 * ((X[:, 0] - 0.7) ** 2 + (X[:, 1] - 0.2) ** 2)
    y = 40.0 * np.exp(a) / (np.exp(b) + np.exp(c)) + rng.standard_normal(n)
    return Workload("yuan2006", X, y, "rbf", gamma, tau, lam)


GENERATORS = {"rbf_small": rbf_small, "rbf_mid": rbf_mid, "lap_large": lap_large, "yuan2006": yuan2006}


def pivot_uniforms(count: int, seed: int = 12345) -> np.ndarray:
    """Uniform [0,1) numbers consumed one per RPCholesky pivot step."""
    return np.random.default_rng(seed).random(count)


def random_vectors(n: int, m: int = 1, seed: int = 7) -> np.ndarray:
    """Standard normal test vectors for Gram-product parity, shape (n,) or (n, m)."""
    v = np.random.default_rng(seed).standard_normal((n, m))
    return v[:, 0] if m == 1 else v
