"""Row-block partition of the preconditioned CG of Sec. 3 over several ranks.

The linear systems of the method, (2.1) and (3.1), have the form
A x = b with A = K + gam 1 1^T + diag(L) and the preconditioner of Lemma 1,
P = F F^T + gam 1 1^T + diag(Lp), applied through the Woodbury identity with
U = [F 1].  When the n rows are split into contiguous blocks I_g, one per
rank, every step of CG needs only these exchanges:

* the search direction p is allgathered (each rank needs all of p to form
  (K p)_{I_g} = K_{I_g,:} p);
* the scalars 1^T p, p^T A p and r^T z are allreduced;
* the Woodbury apply allreduces the (r+1)-vector U^T Lp^{-1} r (each rank
  holds its rows of U), and the set-up allreduces the (r+1)^2 core
  C + U^T Lp^{-1} U once per system.

This module holds that host logic: the split, the per-rank pieces and the
collectives, over ``torch.distributed`` (any backend).  The rank-local Gram
product is a callable ``kmat_rows(row0, row1, p_full) -> (K p)[row0:row1]``,
on a GPU the library's tiled product restricted to a row range; the tests
drive it with a dense stand-in.  Arithmetic is float64 (the reductions),
matching the single-rank CG of the library.
"""
from __future__ import annotations

import numpy as np

TILE = 128


def row_ranges(n: int, world: int, align: int = TILE) -> list[tuple[int, int]]:
    """Contiguous row blocks [start, stop) covering 0..n, one per rank, with
    every boundary a multiple of ``align`` (the Gram kernels' row tile) and
    block sizes differing by at most one tile.  Ranks beyond the number of
    tiles get empty blocks."""
    if n < 0 or world < 1 or align < 1:
        raise ValueError("need n >= 0, world >= 1, align >= 1")
    tiles = (n + align - 1) // align
    base, extra = divmod(tiles, world)
    out, t = [], 0
    for g in range(world):
        cnt = base + (1 if g < extra else 0)
        start, stop = min(n, t * align), min(n, (t + cnt) * align)
        out.append((start, stop))
        t += cnt
    return out


class RowComm:
    """The collectives the partitioned CG uses, over torch.distributed."""

    def __init__(self, dist=None, ranges=None):
        self.dist = dist
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0
        self.ranges = ranges

    def allreduce(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        if self.dist is None:
            return x.copy()
        import torch

        t = torch.from_numpy(x.copy())
        self.dist.all_reduce(t)
        return t.numpy()

    def allgather_rows(self, local: np.ndarray, n: int) -> np.ndarray:
        """Concatenate every rank's block (rank order = row order) into length n."""
        local = np.ascontiguousarray(local, dtype=np.float64)
        if self.dist is None:
            return local.copy()
        import torch

        width = max(b - a for a, b in self.ranges)
        buf = torch.zeros(width, dtype=torch.float64)
        buf[:local.size] = torch.from_numpy(local)
        parts = [torch.zeros(width, dtype=torch.float64) for _ in range(self.world)]
        self.dist.all_gather(parts, buf)
        out = np.empty(n)
        for (a, b), part in zip(self.ranges, parts):
            out[a:b] = part.numpy()[:b - a]
        return out


def woodbury_core(F_rows: np.ndarray, Lp_rows: np.ndarray, gam: float, comm: RowComm) -> np.ndarray:
    """The (r+1)^2 core C + U^T Lp^{-1} U of Lemma 1, U = [F 1], C = diag(I_r, 1/gam):
    each rank adds its rows' share, then one allreduce."""
    n_loc, r = F_rows.shape
    U = np.hstack([F_rows, np.ones((n_loc, 1))])
    G = comm.allreduce(U.T @ (U / Lp_rows[:, None]))
    G[np.arange(r), np.arange(r)] += 1.0
    G[r, r] += 1.0 / gam
    return G


def woodbury_apply_rows(F_rows, Lp_rows, G_chol, r_rows, comm: RowComm) -> np.ndarray:
    """Rows of P^{-1} r by Lemma 1: t = U^T Lp^{-1} r (allreduced), t2 = G^{-1} t
    (replicated), z_I = Lp_I^{-1} (r_I - U_I t2)."""
    n_loc = F_rows.shape[0]
    U = np.hstack([F_rows, np.ones((n_loc, 1))])
    w = r_rows / Lp_rows
    t = comm.allreduce(U.T @ w)
    t2 = _chol_solve(G_chol, t)
    return w - (U @ t2) / Lp_rows


def _chol_solve(Lc: np.ndarray, b: np.ndarray) -> np.ndarray:
    import scipy.linalg as sla

    return sla.cho_solve((Lc, True), b)


def pcg_rows(kmat_rows, n: int, b_rows, L_rows, Lp_rows, gam: float, F_rows, tol: float, maxit: int,
             comm: RowComm, row0: int, row1: int):
    """Left-preconditioned CG for (K + gam 1 1^T + diag(L)) x = b with this
    rank's rows [row0, row1) of every vector, from x = 0, until the recursive
    residual satisfies ||r|| <= tol or maxit iterations.  ``kmat_rows(row0,
    row1, p)`` returns rows [row0, row1) of K p for a full-length p.  Returns
    (x_rows, iterations, ||r||)."""
    import scipy.linalg as sla

    G = woodbury_core(F_rows, Lp_rows, gam, comm)
    G_chol = sla.cholesky(G, lower=True)
    x = np.zeros(row1 - row0)
    r = np.array(b_rows, dtype=np.float64)
    rn = float(np.sqrt(comm.allreduce(np.array([r @ r]))[0]))
    it = 0
    if rn <= tol:
        return x, it, rn
    z = woodbury_apply_rows(F_rows, Lp_rows, G_chol, r, comm)
    p = z.copy()
    rz = float(comm.allreduce(np.array([r @ z]))[0])
    while it < maxit:
        p_full = comm.allgather_rows(p, n)
        sum_p = float(p_full.sum())
        q = kmat_rows(row0, row1, p_full) + gam * sum_p + L_rows * p
        pAp = float(comm.allreduce(np.array([p @ q]))[0])
        a = rz / pAp
        x += a * p
        r -= a * q
        it += 1
        rn = float(np.sqrt(comm.allreduce(np.array([r @ r]))[0]))
        if rn <= tol:
            break
        z = woodbury_apply_rows(F_rows, Lp_rows, G_chol, r, comm)
        rz_new = float(comm.allreduce(np.array([r @ z]))[0])
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rn
