"""FP64 CPU oracle for PALM-KQR (Deng, Li, Zhang, arxiv 2510.07929).

TEST INFRASTRUCTURE ONLY.  This module states, plainly and slowly, in float64
numpy, what the GPU path computes.  It shares no code with the CUDA library and
does not import it; the library does not import this.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import it.

Each function cites the part of the paper it follows.  Where the paper leaves
a constant or a rule open, the reading taken is stated at that function and in
``Options``.  Every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, brute-force active-set enumeration,
the large-lambda LP limit, a dense inverse, finite differences, weak duality,
exact invariances, or a library QP routine on tiny inputs).

Notation follows the paper: n points x_i in R^p, responses y, quantile level
tau, regularisation lambda (``lam``), kernel scale gamma, dual variable alpha,
consensus copy v, multipliers (beta, z), ALM/ADMM penalty sigma.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as _sla

RBF = "rbf"
LAPLACIAN = "laplacian"


# ---------------------------------------------------------------------------
# Kernel entries (Section 1, text after eq. (1.1)):
#   RBF        k(x, x') = exp(-gamma * ||x - x'||_2^2)
#   Laplacian  k(x, x') = exp(-gamma * ||x - x'||_1)
# ---------------------------------------------------------------------------
def _chunk_rows(n_rows: int, n_cols: int, p: int, max_elems: int) -> int:
    return max(1, min(n_rows, max_elems // max(1, n_cols * p)))


def gram(X, Z, kind: str, gamma: float, max_elems: int = 1 << 25) -> np.ndarray:
    """Kernel matrix block K[i, j] = k(x_i, z_j), from its definition (Sec. 1)."""
    X = np.asarray(X, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    if kind not in (RBF, LAPLACIAN):
        raise ValueError(f"unknown kernel {kind!r}")
    out = np.empty((X.shape[0], Z.shape[0]), dtype=np.float64)
    step = _chunk_rows(X.shape[0], Z.shape[0], X.shape[1], max_elems)
    for i0 in range(0, X.shape[0], step):
        diff = X[i0:i0 + step, None, :] - Z[None, :, :]
        if kind == RBF:
            dist = np.sum(diff * diff, axis=2)
        else:
            dist = np.sum(np.abs(diff), axis=2)
        out[i0:i0 + step] = np.exp(-gamma * dist)
    return out


def kmatvec(X, V, kind: str, gamma: float, rows=None, max_elems: int = 1 << 25) -> np.ndarray:
    """u = K[rows, :] @ V with K formed from its definition, a block of rows at
    a time (the K.v / K.V product that dominates the method, Sec. 1 and Sec. 3).
    ``V`` may be a vector (n,) or a matrix (n, m)."""
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    idx = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    vec = V.ndim == 1
    Vm = V[:, None] if vec else V
    out = np.empty((idx.size, Vm.shape[1]), dtype=np.float64)
    step = _chunk_rows(idx.size, X.shape[0], X.shape[1], max_elems)
    for a in range(0, idx.size, step):
        out[a:a + step] = gram(X[idx[a:a + step]], X, kind, gamma, max_elems) @ Vm
    return out[:, 0] if vec else out


def predict(X, alpha, beta: float, Xnew, kind: str, gamma: float, lam: float) -> np.ndarray:
    """Representer form f(x) = beta + (1/lambda) sum_j alpha_j k(x_j, x) (Sec. 1)."""
    return beta + gram(Xnew, X, kind, gamma) @ np.asarray(alpha, dtype=np.float64) / lam


# ---------------------------------------------------------------------------
# Check loss, its conjugate's box, projection and Clarke Jacobian
# ---------------------------------------------------------------------------
def check_loss(z, tau: float) -> float:
    """rho_tau(z) = sum_i (tau z_i if z_i > 0 else -(1 - tau) z_i)  (Sec. 1)."""
    z = np.asarray(z, dtype=np.float64)
    return float(np.sum(np.where(z > 0, tau * z, -(1.0 - tau) * z)))


def proj_box(w, tau: float) -> np.ndarray:
    """Euclidean projection onto B = [tau - 1, tau]^n (Sec. 2.1)."""
    return np.clip(np.asarray(w, dtype=np.float64), tau - 1.0, tau)


def jacobian_diag(w, tau: float) -> np.ndarray:
    """Diagonal of one element S of the Clarke Jacobian of Pi_B at w (Sec. 2.2):
    1 strictly inside (tau - 1, tau), 0 strictly outside.  On the boundary the
    Jacobian is the whole interval [0, 1]; this oracle takes 0 there."""
    w = np.asarray(w, dtype=np.float64)
    return ((w > tau - 1.0) & (w < tau)).astype(np.float64)


# ---------------------------------------------------------------------------
# Objectives and the relative KKT residuals / duality gap (Sec. 4)
# ---------------------------------------------------------------------------
def dual_objective(alpha, Kalpha, y, lam: float) -> float:
    """obj_D = -alpha^T K alpha / (2 lambda) + y^T alpha  (eq. (1.3))."""
    alpha = np.asarray(alpha, dtype=np.float64)
    return float(-alpha @ Kalpha / (2.0 * lam) + np.asarray(y) @ alpha)


def kkt_residuals(alpha, v, beta: float, z, y, Kalpha, tau: float, lam: float) -> dict:
    """eta_p, eta_d, eta_c, eta_kkt = max of the three, and eta_gap (Sec. 4).

    ``Kalpha`` is K @ alpha.  obj_P = rho_tau(z) + alpha^T K alpha / (2 lambda)
    uses the multiplier z, as in Sec. 4."""
    alpha = np.asarray(alpha, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    Kalpha = np.asarray(Kalpha, dtype=np.float64)
    eta_p = np.linalg.norm(z - y + beta + Kalpha / lam) / (1.0 + np.linalg.norm(y))
    eta_d = math.sqrt(alpha.sum() ** 2 + np.sum((alpha - v) ** 2)) / (1.0 + np.linalg.norm(alpha))
    eta_c = np.linalg.norm(v - proj_box(z + v, tau)) / (1.0 + np.linalg.norm(v))
    quad = float(alpha @ Kalpha) / (2.0 * lam)
    obj_p = check_loss(z, tau) + quad
    obj_d = -quad + float(y @ alpha)
    eta_gap = abs(obj_p - obj_d) / (1.0 + abs(obj_p) + abs(obj_d))
    return dict(eta_p=float(eta_p), eta_d=float(eta_d), eta_c=float(eta_c),
                eta_kkt=float(max(eta_p, eta_d, eta_c)), eta_gap=float(eta_gap),
                obj_p=obj_p, obj_d=obj_d)


# ---------------------------------------------------------------------------
# The reduced ALM subproblem phi_k (eq. (2.2)) and its gradient (eq. (2.3))
# ---------------------------------------------------------------------------
def moreau_box(w, tau: float, sigma: float) -> float:
    """Moreau envelope of delta_B with parameter sigma (Appendix A):
    min_u delta_B(u) + sigma/2 ||u - w||^2 = sigma/2 ||w - Pi_B(w)||^2."""
    w = np.asarray(w, dtype=np.float64)
    return 0.5 * sigma * float(np.sum((w - proj_box(w, tau)) ** 2))


def phi(alpha, Kalpha, y, beta: float, z, sigma: float, tau: float, lam: float) -> float:
    """phi_k(alpha) of eq. (2.2)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    s = alpha.sum() + beta / sigma
    return (float(alpha @ Kalpha) / (2.0 * lam) - float(np.asarray(y) @ alpha)
            + 0.5 * sigma * s * s + moreau_box(alpha + np.asarray(z) / sigma, tau, sigma))


def grad_phi(alpha, Kalpha, y, beta: float, z, sigma: float, tau: float, lam: float) -> np.ndarray:
    """grad phi_k(alpha) = K alpha / lambda - y + beta 1 + sigma 1 1^T alpha
    + sigma (w - Pi_B(w)),  w = alpha + z / sigma  (eq. (2.3))."""
    alpha = np.asarray(alpha, dtype=np.float64)
    w = alpha + np.asarray(z) / sigma
    return (np.asarray(Kalpha) / lam - np.asarray(y) + beta + sigma * alpha.sum()
            + sigma * (w - proj_box(w, tau)))


def newton_diag(w, tau: float, sigma: float, lam: float, eps: float) -> np.ndarray:
    """Diagonal L of the scaled Newton system (eq. (3.1)):
    L = lambda sigma (I - S) + lambda eps I, S from ``jacobian_diag``."""
    return lam * sigma * (1.0 - jacobian_diag(w, tau)) + lam * eps


# ---------------------------------------------------------------------------
# Low-rank preconditioner (Sec. 3): RPCholesky, rank heuristic, Lemma 1, PCG
# ---------------------------------------------------------------------------
def rpcholesky(column, diag, r: int, uniforms):
    """Randomly pivoted Cholesky, F = RPCholesky(K, r) with K ~= F F^T (Sec. 3,
    after Chen, Epperly, Tropp and Webber 2023).

    ``column(s)`` returns column s of K; ``diag`` is diag(K).  Step t draws the
    pivot s with probability d_s / sum(d), d the residual diagonal, by inverting
    the cumulative sum at ``uniforms[t] * sum(d)`` (the smallest s whose running
    sum exceeds it); the random numbers are inputs so that another
    implementation can draw the same pivots.  A chosen pivot's residual becomes
    0, so columns are sampled without replacement.  Stops early when the
    residual diagonal is exhausted.  Returns (F, pivots)."""
    d = np.array(diag, dtype=np.float64)
    n = d.size
    F = np.zeros((n, r), dtype=np.float64)
    piv = []
    for t in range(r):
        total = d.sum()
        if not total > 0.0:
            break
        s = int(np.searchsorted(np.cumsum(d), uniforms[t] * total, side="right"))
        s = min(s, n - 1)
        g = np.asarray(column(s), dtype=np.float64) - F[:, :t] @ F[s, :t]
        if not g[s] > 0.0:
            break
        F[:, t] = g / math.sqrt(g[s])
        d = np.maximum(d - F[:, t] ** 2, 0.0)
        piv.append(s)
    return F[:, :len(piv)], np.array(piv, dtype=np.int64)


def rank_from_spectrum(F0, xi: float) -> int:
    """Rank heuristic of Sec. 3: with lambda_1 >= ... the eigenvalues of
    F0^T F0 (equal to the nonzero eigenvalues of F0 F0^T), r is the smallest
    index with xi * lambda_1 >= lambda_r; if no index satisfies it, r = r0."""
    F0 = np.asarray(F0, dtype=np.float64)
    lam = np.sort(np.linalg.eigvalsh(F0.T @ F0))[::-1]
    for i, li in enumerate(lam):
        if xi * lam[0] >= li:
            return i + 1
    return lam.size


def woodbury_apply(F, Ldiag, gam: float, rvec) -> np.ndarray:
    """P^{-1} r for P = F F^T + gam 1 1^T + diag(L), by Lemma 1:
    P^{-1} = L^{-1} - L^{-1} U (C + U^T L^{-1} U)^{-1} U^T L^{-1},
    U = [F 1], C = diag(I_r, 1/gam)."""
    F = np.asarray(F, dtype=np.float64)
    Ldiag = np.asarray(Ldiag, dtype=np.float64)
    n, r = F.shape
    U = np.hstack([F, np.ones((n, 1))])
    C = np.diag(np.concatenate([np.ones(r), [1.0 / gam]]))
    Linv_r = np.asarray(rvec, dtype=np.float64) / Ldiag
    G = C + U.T @ (U / Ldiag[:, None])
    t = np.linalg.solve(G, U.T @ Linv_r)
    return Linv_r - (U @ t) / Ldiag


def pcg(Aop, b, Pinv, tol: float, maxit: int, x0=None):
    """Left-preconditioned conjugate gradients (Sec. 3; Saad, Alg. 9.1) for
    A x = b, stopping when the recursive residual satisfies ||r|| <= tol.
    Returns (x, iterations, ||r||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - Aop(x) if x0 is not None else b.copy()
    it = 0
    rn = float(np.linalg.norm(r))
    if rn <= tol:
        return x, it, rn
    zz = Pinv(r)
    p = zz.copy()
    rz = float(r @ zz)
    while it < maxit:
        Ap = Aop(p)
        a = rz / float(p @ Ap)
        x = x + a * p
        r = r - a * Ap
        it += 1
        rn = float(np.linalg.norm(r))
        if rn <= tol:
            break
        zz = Pinv(r)
        rz_new = float(r @ zz)
        p = zz + (rz_new / rz) * p
        rz = rz_new
    return x, it, rn


# ---------------------------------------------------------------------------
# Algorithm constants.  The paper leaves these open; the values are the
# readings this oracle takes (the GPU library takes the same ones).
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    sigma0: float = 1.0          # ADMM penalty sigma (Alg. 1 input)
    gamma_admm: float = 1.618    # ADMM step length in (0, (1 + sqrt 5) / 2) (Alg. 1)
    admm_tol: float = 1e-3       # Phase I stop: max(eta_kkt, eta_gap) <= 1e-3 (Sec. 4)
    admm_maxit: int = 100        # ... or 100 iterations (Sec. 4)
    balance_every: int = 5       # ADMM residual balancing period (reading)
    balance_ratio: float = 5.0   # rebalance when eta_p / eta_d leaves [1/5, 5]
    balance_factor: float = 1.5  # sigma multiplied or divided by this
    alm_maxit: int = 1000        # Phase II stop: 1000 iterations (Sec. 4)
    sigma_alm_scale: float = 1.0 # ALM sigma_0 = max(final ADMM sigma, sigma_alm_scale / lambda) (reading)
    sigma_factor: float = 10.0   # ALM "sigma_{k+1} >= sigma_k" rule (reading)
    sigma_max: float = 1e8
    eta_bar: float = 0.5         # Alg. 3 constants (reading)
    iota: float = 0.5
    mu: float = 1e-4
    r_ls: float = 0.5
    tau1: float = 1e-2
    tau2: float = 1e-1
    ssn_maxit: int = 50
    ls_maxit: int = 40


def _admm_sigma_update(sigma: float, k: int, res: dict, o: Options) -> float:
    """Residual balancing between eta_p (stationarity) and eta_d (consensus
    feasibility), every ``balance_every`` iterations (reading of Alg. 1's
    free sigma); ``balance_every <= 0`` keeps sigma fixed."""
    if o.balance_every <= 0 or (k + 1) % o.balance_every != 0:
        return sigma
    if res["eta_d"] > o.balance_ratio * res["eta_p"]:
        return sigma * o.balance_factor
    if res["eta_p"] > o.balance_ratio * res["eta_d"]:
        return sigma / o.balance_factor
    return sigma


def admm(K, y, tau: float, lam: float, o: Options, beta: float = 0.0, z=None, v=None):
    """Phase I, Algorithm 1 (inexact ADMM on (1.4)); the alpha-system
    M alpha = b_k is solved exactly here (Cholesky factor of the SPD M, reused
    while sigma is unchanged), which satisfies every inexactness bound
    eps_k >= 0.  Starts from beta = 0, z = v = 0 unless given.
    Stops when max(eta_kkt, eta_gap) <= admm_tol or after admm_maxit (Sec. 4)."""
    n = y.size
    z = np.zeros(n) if z is None else np.array(z, dtype=np.float64)
    v = np.zeros(n) if v is None else np.array(v, dtype=np.float64)
    sigma = o.sigma0
    ones = np.ones(n)
    chol = None
    res = None
    alpha = np.zeros(n)
    k = 0
    for k in range(o.admm_maxit):
        if chol is None:
            M = K + lam * sigma * (np.eye(n) + np.outer(ones, ones))
            chol = _sla.cho_factor(M, lower=True)
        b = lam * (y - beta * ones - z + sigma * v)
        alpha = _sla.cho_solve(chol, b)
        v = proj_box(alpha + z / sigma, tau)
        beta = beta + o.gamma_admm * sigma * alpha.sum()
        z = z + o.gamma_admm * sigma * (alpha - v)
        res = kkt_residuals(alpha, v, beta, z, y, K @ alpha, tau, lam)
        if max(res["eta_kkt"], res["eta_gap"]) <= o.admm_tol:
            break
        new_sigma = _admm_sigma_update(sigma, k, res, o)
        if new_sigma != sigma:
            sigma, chol = new_sigma, None
    return dict(alpha=alpha, v=v, beta=beta, z=z, sigma=sigma, iters=k + 1, kkt=res)


def ssn(K, y, tau: float, lam: float, beta: float, z, sigma: float, alpha0, o: Options, tol_grad: float):
    """Algorithm 3 (semismooth Newton on phi_k) with Armijo backtracking.  The
    regularised Newton system (H_t + eps_t I) d = -grad is solved exactly
    (Cholesky: every generalized Hessian is positive definite), which meets
    the PCG accuracy bound of Alg. 3.  Stops when ||grad phi_k|| <= tol_grad
    or after ssn_maxit steps.  The Armijo test
    phi(alpha + c d) <= phi(alpha) + mu c <grad, d> is evaluated on the
    difference phi(alpha + c d) - phi(alpha), term by term."""
    n = y.size
    alpha = np.array(alpha0, dtype=np.float64)
    Kalpha = K @ alpha
    ones = np.ones(n)
    steps = 0
    for _ in range(o.ssn_maxit):
        w = alpha + z / sigma
        g = grad_phi(alpha, Kalpha, y, beta, z, sigma, tau, lam)
        ng = float(np.linalg.norm(g))
        if ng <= tol_grad:
            break
        eps = o.tau1 * min(o.tau2, ng)
        S = jacobian_diag(w, tau)
        H = K / lam + sigma * (np.outer(ones, ones) + np.diag(1.0 - S)) + eps * np.eye(n)
        d = _sla.cho_solve(_sla.cho_factor(H, lower=True), -g)
        Kd = K @ d
        gd = float(g @ d)
        s0 = alpha.sum() + beta / sigma
        sd = d.sum()
        m0 = moreau_box(w, tau, sigma)
        c = 1.0
        for _ls in range(o.ls_maxit):
            dphi = ((c * float(Kalpha @ d) + 0.5 * c * c * float(d @ Kd)) / lam
                    - c * float(y @ d)
                    + 0.5 * sigma * ((s0 + c * sd) ** 2 - s0 ** 2)
                    + moreau_box(w + c * d, tau, sigma) - m0)
            if dphi <= o.mu * c * gd:
                break
            c *= o.r_ls
        alpha = alpha + c * d
        Kalpha = Kalpha + c * Kd
        steps += 1
    v = proj_box(alpha + z / sigma, tau)
    return alpha, v, Kalpha, steps


def alm(K, y, tau: float, lam: float, o: Options, tol: float, start: dict):
    """Phase II, Algorithm 2 (SSN-ALM), from the Phase I iterate.  Multiplier
    updates beta += sigma 1^T alpha, z += sigma (alpha - v).  Stops when
    max(eta_kkt, eta_gap) <= tol or after alm_maxit iterations (Sec. 4).

    Readings: sigma_0 = max(Phase I's final sigma, sigma_alm_scale / lambda)
    (the multiplier of 1^T alpha = 0 contracts by about 1 / (1 + lambda sigma
    1^T K^-1 1) per iteration, so sigma is put on the 1/lambda scale); sigma is multiplied by
    sigma_factor (capped at sigma_max) whenever eta_d fails to halve; the SSN
    inner tolerance is max(0.1 tol (1 + ||y||), g0 0.2^(k+1)), g0 the gradient
    norm at the first ALM iterate."""
    alpha = np.array(start["alpha"], dtype=np.float64)
    beta = float(start["beta"])
    z = np.array(start["z"], dtype=np.float64)
    sigma = max(float(start["sigma"]), o.sigma_alm_scale / lam)
    ny = float(np.linalg.norm(y))
    g0 = None
    prev_eta_d = None
    res = start.get("kkt")
    newton = 0
    k = 0
    for k in range(o.alm_maxit):
        if g0 is None:
            g0 = float(np.linalg.norm(grad_phi(alpha, K @ alpha, y, beta, z, sigma, tau, lam)))
        tol_grad = max(0.1 * tol * (1.0 + ny), g0 * 0.2 ** (k + 1))
        alpha, v, Kalpha, steps = ssn(K, y, tau, lam, beta, z, sigma, alpha, o, tol_grad)
        newton += steps
        beta = beta + sigma * alpha.sum()
        z = z + sigma * (alpha - v)
        res = kkt_residuals(alpha, v, beta, z, y, K @ alpha, tau, lam)
        if max(res["eta_kkt"], res["eta_gap"]) <= tol:
            break
        if prev_eta_d is not None and res["eta_d"] > 0.5 * prev_eta_d:
            sigma = min(o.sigma_max, sigma * o.sigma_factor)
        prev_eta_d = res["eta_d"]
    return dict(alpha=alpha, v=v, beta=beta, z=z, sigma=sigma, iters=k + 1,
                newton=newton, kkt=res)


def solve_dense(K, y, tau: float, lam: float, tol: float = 1e-6, o: Options | None = None) -> dict:
    """Two-phase PALM-KQR (Alg. 1 then Alg. 2/3) on an explicit FP64 kernel
    matrix.  Returns alpha, beta, v, z, the Sec. 4 residuals and iteration
    counts."""
    o = o or Options()
    y = np.asarray(y, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    p1 = admm(K, y, tau, lam, o)
    out = dict(phase1_iters=p1["iters"], phase1_kkt=p1["kkt"])
    if max(p1["kkt"]["eta_kkt"], p1["kkt"]["eta_gap"]) <= tol:
        out.update(alpha=p1["alpha"], v=p1["v"], beta=p1["beta"], z=p1["z"], kkt=p1["kkt"],
                   phase2_iters=0, newton=0)
        return out
    p2 = alm(K, y, tau, lam, o, tol, p1)
    out.update(alpha=p2["alpha"], v=p2["v"], beta=p2["beta"], z=p2["z"], kkt=p2["kkt"],
               phase2_iters=p2["iters"], newton=p2["newton"])
    return out


def solve(X, y, kind: str, gamma: float, tau: float, lam: float, tol: float = 1e-6,
          o: Options | None = None) -> dict:
    """Forms K from its definition, then runs ``solve_dense``."""
    return solve_dense(gram(X, X, kind, gamma), y, tau, lam, tol, o)


# ---------------------------------------------------------------------------
# Certificate independent of any algorithm (weak duality between (1.2) and (1.3))
# ---------------------------------------------------------------------------
def project_feasible(alpha, tau: float, iters: int = 200) -> np.ndarray:
    """Projection onto {alpha in B : 1^T alpha = 0}: Pi_B(alpha - t 1) with the
    scalar t found by bisection so that the sum vanishes."""
    alpha = np.asarray(alpha, dtype=np.float64)
    lo, hi = float(alpha.min()) - 1.0, float(alpha.max()) + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if proj_box(alpha - mid, tau).sum() > 0.0:
            lo = mid
        else:
            hi = mid
    return proj_box(alpha - 0.5 * (lo + hi), tau)


def quantile_intercept(r, tau: float) -> float:
    """argmin_beta rho_tau(r - beta 1): a sample tau-quantile of r.  The
    objective is convex and piecewise linear with kinks at the r_i, so the
    minimum is at an order statistic; the ones around ceil(n tau) are tried."""
    rs = np.sort(np.asarray(r, dtype=np.float64))
    k = int(math.ceil(rs.size * tau))
    cand = rs[max(0, k - 3):min(rs.size, k + 3)]
    vals = [check_loss(rs - b, tau) for b in cand]
    return float(cand[int(np.argmin(vals))])


def certified_gap(alpha, K, y, tau: float, lam: float, theta=None) -> dict:
    """Relative duality gap between the primal (1.2) at theta (default: alpha
    as given), beta = the tau-quantile of y - K theta / lambda, and the dual
    (1.3) at a = the feasible projection of alpha.  Weak duality gives P >= D
    for every theta and every feasible a (rho_tau(u) >= a^T u on the box, and
    (theta - a)^T K (theta - a) >= 0), so the gap bounds how far both are from
    the optimum.  Leaving theta unprojected keeps the 1/lambda factor of the
    primal residual away from the projection step."""
    theta = np.asarray(alpha if theta is None else theta, dtype=np.float64)
    a = project_feasible(alpha, tau)
    return certified_gap_from_products(theta, a, K @ theta, K @ a, y, tau, lam)


def certified_gap_from_products(theta, a, Ktheta, Ka, y, tau: float, lam: float) -> dict:
    """The weak-duality certificate of ``certified_gap`` from the products
    K theta and K a (for sizes where K cannot be formed); ``a`` must be the
    feasible projection of alpha (``project_feasible``)."""
    y = np.asarray(y, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    r = y - np.asarray(Ktheta) / lam
    beta = quantile_intercept(r, tau)
    P = check_loss(r - beta, tau) + float(theta @ Ktheta) / (2.0 * lam)
    D = -float(a @ Ka) / (2.0 * lam) + float(y @ a)
    return dict(gap=(P - D) / (1.0 + abs(P) + abs(D)), P=P, D=D, beta=beta, alpha=a)


# ---------------------------------------------------------------------------
# Held-out check loss and its gradient by implicit differentiation (an
# extension of the method: the paper has no counterpart; built on eq. (1.3),
# the representer form of Sec. 1 and the Sec. 4 KKT conditions).
#
# With E = {i : tau - 1 < alpha_i < tau} (the elbow set) fixed, the KKT
# conditions read F(alpha_E, beta; theta) = 0 with
#   F_E = (K alpha)_E / lambda + beta - y_E,   F_last = 1^T alpha,
# and alpha_i fixed at its bound off E.  The held-out loss is
#   l = sum_h rho_tau(y_h - f(x_h)),  f(x) = beta + (1/lambda) sum_j alpha_j k(x_j, x).
# With g_h = d rho_tau / d f (= -tau when y_h > f_h, 1 - tau when y_h < f_h),
# a = [K_{E,h} g / lambda ; sum_h g_h] and J = [[K_EE / lambda, 1], [1^T, 0]],
# solve J w = a; then for each parameter theta
#   dl/dtheta = g^T (df_h/dtheta at fixed alpha, beta) - w^T (dF/dtheta at fixed alpha, beta).
# ---------------------------------------------------------------------------
def _sq_dists(X, Z):
    diff = np.asarray(X, dtype=np.float64)[:, None, :] - np.asarray(Z, dtype=np.float64)[None, :, :]
    return np.sum(diff * diff, axis=2)


def heldout_loss(X, y, Xh, yh, gamma: float, tau: float, lam: float, tol: float = 1e-12,
                 o: Options | None = None) -> dict:
    """Solves the RBF problem on (X, y) and evaluates the held-out check loss
    sum_h rho_tau(y_h - f(x_h)) of the representer-form predictor (Sec. 1)."""
    K = gram(X, X, RBF, gamma)
    res = solve_dense(K, y, tau, lam, tol, o)
    f = predict(X, res["alpha"], res["beta"], Xh, RBF, gamma, lam)
    return dict(loss=check_loss(np.asarray(yh) - f, tau), alpha=res["alpha"], beta=res["beta"], f=f, K=K, kkt=res["kkt"])


def heldout_grad(X, y, Xh, yh, gamma: float, tau: float, lam: float, tol: float = 1e-12, edge: float = 1e-7,
                 want_dX: bool = True) -> dict:
    """Gradient of the held-out check loss with respect to log gamma, log
    lambda and the training inputs X, by the implicit-function formula above,
    with every partial derivative formed densely from its definition."""
    X = np.asarray(X, dtype=np.float64)
    Xh = np.asarray(Xh, dtype=np.float64)
    yh = np.asarray(yh, dtype=np.float64)
    n, p = X.shape
    st = heldout_loss(X, y, Xh, yh, gamma, tau, lam, tol)
    alpha, beta, f, K = st["alpha"], st["beta"], st["f"], st["K"]
    Kh = gram(Xh, X, RBF, gamma)
    D = _sq_dists(X, X)
    Dh = _sq_dists(Xh, X)
    r = yh - f
    g = np.where(r > 0, -tau, 1.0 - tau)
    E = np.flatnonzero((alpha > tau - 1.0 + edge) & (alpha < tau - edge))
    m = E.size
    J = np.zeros((m + 1, m + 1))
    J[:m, :m] = K[np.ix_(E, E)] / lam
    J[:m, m] = 1.0
    J[m, :m] = 1.0
    a = np.concatenate([Kh[:, E].T @ g / lam, [g.sum()]])
    w = np.linalg.solve(J, a)
    u = w[:m]

    def total(dK, dKh, dlam_scale=None):
        # explicit derivatives of f_h and F for a derivative dK of K (and dKh of Kh)
        dfh = dKh @ alpha / lam
        dFE = (dK @ alpha)[E] / lam
        return float(g @ dfh - u @ dFE)

    d_loglam = float(g @ (-(Kh @ alpha) / lam) - u @ (-(K @ alpha)[E] / lam))
    d_loggam = total(-gamma * D * K, -gamma * Dh * Kh)
    dX = np.zeros((n, p)) if want_dX else None
    for k in range(n if want_dX else 0):
        for c in range(p):
            # d K_ij / d X_kc: row and column k of K, column k of Kh
            dK = np.zeros((n, n))
            col = -2.0 * gamma * (X[k, c] - X[:, c]) * K[k, :]
            dK[k, :] = col
            dK[:, k] = col
            dK[k, k] = 0.0
            dKh = np.zeros_like(Kh)
            dKh[:, k] = -2.0 * gamma * (X[k, c] - Xh[:, c]) * Kh[:, k]
            dX[k, c] = total(dK, dKh)
    return dict(loss=st["loss"], d_loggamma=d_loggam, d_loglambda=d_loglam, dX=dX, elbow=E, g=g, w=w,
                alpha=alpha, beta=beta)
