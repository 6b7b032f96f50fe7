"""Row-block partition of the preconditioned CG (paper_2510_07929_gb300/partition.py),
run as 2 and 4 gloo ranks on the CPU: the split, the allgather of the search
direction, the allreduced scalars and the allreduced Woodbury vector and core
must reproduce the one-rank CG to rounding.  The operator is a dense stand-in
the test builds itself (no GPU); this checks the partition logic only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2510_07929_gb300 import partition as PT  # noqa: E402


def test_row_ranges_cover_aligned_and_balanced():
    for n in (1, 127, 128, 129, 1000, 20000, 200000):
        for world in (1, 2, 3, 4, 8):
            rr = PT.row_ranges(n, world)
            assert len(rr) == world and rr[0][0] == 0 and rr[-1][1] == n
            assert all(a <= b for a, b in rr) and all(rr[g][1] == rr[g + 1][0] for g in range(world - 1))
            assert all(a % PT.TILE == 0 or a == n for a, _ in rr)
            sizes = [(b - a + PT.TILE - 1) // PT.TILE for a, b in rr]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        PT.row_ranges(10, 0)


def _problem(n=700, r=60, seed=0):
    """Dense stand-in: an RBF-like SPD K, its leading r pivoted-Cholesky columns
    as F, a two-level diagonal L and a right-hand side."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, 3))
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    K = np.exp(-2.0 * d2)
    F = np.linalg.cholesky(K + 1e-8 * np.eye(n))[:, :r]
    L = np.where(rng.random(n) < 0.5, 1e-3, 5e-2)
    Lp = L + 0.01
    b = rng.standard_normal(n)
    return K, F, L, Lp, b


def _solve_rows(world, rank, dist=None):
    K, F, L, Lp, b = _problem()
    n = K.shape[0]
    ranges = PT.row_ranges(n, world)
    comm = PT.RowComm(dist, ranges)
    a, c = ranges[rank]
    kmat_rows = lambda r0, r1, p: K[r0:r1] @ p
    x, it, rn = PT.pcg_rows(kmat_rows, n, b[a:c], L[a:c], Lp[a:c], 0.05, F[a:c], 1e-9 * np.linalg.norm(b), 500,
                            comm, a, c)
    return comm.allgather_rows(x, n) if dist is not None else x, it, rn


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import test_row_partition_gloo as T
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
x, it, rn = T._solve_rows(world, rank, dist)
if rank == 0:
    print(json.dumps({"x": x.tolist(), "it": it, "rn": rn}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
def test_partitioned_pcg_reproduces_single_rank(world):
    x1, it1, rn1 = _solve_rows(1, 0)
    K, F, L, Lp, b = _problem()
    A = K + 0.05 * np.ones_like(K) + np.diag(L)
    np.testing.assert_allclose(x1, np.linalg.solve(A, b), rtol=1e-6, atol=1e-8 * np.abs(x1).max())
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(out)
    d = json.loads(outs[0].strip().splitlines()[-1])
    # the allreduced dots are summed in another order than on one rank: the runs agree
    # to rounding amplified by CG, i.e. to well inside CG's own tolerance
    assert abs(d["it"] - it1) <= 1
    np.testing.assert_allclose(d["x"], x1, rtol=0, atol=1e-7 * np.abs(x1).max())
    assert d["rn"] <= 1e-9 * np.linalg.norm(b)


def test_woodbury_pieces_sum_to_the_full_reduction():
    """Per-rank shares of U^T Lp^-1 r and of the core add up to the one-rank values."""
    K, F, L, Lp, b = _problem(n=515, r=7, seed=3)
    n = b.size
    one = PT.RowComm(None)
    G_full = PT.woodbury_core(F, Lp, 0.2, one)
    U = np.hstack([F, np.ones((n, 1))])
    parts = [U[a:c].T @ (U[a:c] / Lp[a:c, None]) for a, c in PT.row_ranges(n, 3)]
    G_sum = sum(parts)
    G_sum[np.arange(7), np.arange(7)] += 1.0
    G_sum[7, 7] += 1.0 / 0.2
    np.testing.assert_allclose(G_sum, G_full, rtol=1e-12)
    P = F @ F.T + 0.2 * np.ones((n, n)) + np.diag(Lp)
    import scipy.linalg as sla

    z = PT.woodbury_apply_rows(F, Lp, sla.cholesky(G_full, lower=True), b, one)
    np.testing.assert_allclose(z, np.linalg.solve(P, b), rtol=1e-8, atol=1e-10 * np.abs(z).max())
