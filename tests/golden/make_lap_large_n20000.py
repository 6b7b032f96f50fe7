"""Writes lap_large_n20000.json: the FP64 oracle's solution summary for the
Laplacian workload's generator at n = 20000 (x ~ U[-1,1]^50,
y = sum_j sin(x_j)/sqrt(50) + (0.5 + |x_1|) N(0,1), seed 0, gamma = 1/50,
tau = 0.25, lambda = 1e-4).

Calls only the oracle: K from its definition in FP64 (oracle.native.gram),
the two-phase method of Alg. 1 and Alg. 2/3 with exact dense solves
(oracle.kqr_oracle.solve_dense) to max(eta_kkt, eta_gap) <= 1e-10, then the
weak-duality certificate of the result.  The dual optimum D* = obj_D at the
feasible projection of alpha is what the GPU parity test compares against
(relative objective gap <= 1e-6).  Run: python tests/golden/make_lap_large_n20000.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import kqr_oracle as O  # noqa: E402
from oracle import native as N  # noqa: E402
from paper_2510_07929_gb300 import workloads as W  # noqa: E402


def main():
    wl = W.lap_large(n=20000, seed=0)
    t0 = time.time()
    K = N.gram(wl.X, wl.X, wl.kind, wl.gamma)
    t_gram = time.time() - t0
    res = O.solve_dense(K, wl.y, wl.tau, wl.lam, tol=1e-10)
    t_solve = time.time() - t0 - t_gram
    a = O.project_feasible(res["alpha"], wl.tau)
    Ka = K @ a
    cert = O.certified_gap(res["alpha"], K, wl.y, wl.tau, wl.lam)
    out = {
        "what": "FP64 oracle solution summary, lap_large generator at n = 20000 (seed 0), Laplacian gamma = 1/50, "
                "tau = 0.25, lambda = 1e-4, solved to max(eta_kkt, eta_gap) <= 1e-10 by Alg. 1 then Alg. 2/3 "
                "with exact dense solves; written by tests/golden/make_lap_large_n20000.py (oracle only)",
        "n": wl.n, "p": wl.p, "kind": wl.kind, "gamma": wl.gamma, "tau": wl.tau, "lam": wl.lam, "seed": 0,
        "obj_d_star": O.dual_objective(a, Ka, wl.y, wl.lam),
        "certified_gap": cert["gap"], "certificate_P": cert["P"], "certificate_D": cert["D"],
        "beta": res["beta"], "kkt": res["kkt"], "phase1_iters": res["phase1_iters"],
        "phase2_iters": res["phase2_iters"], "newton_steps": res["newton"],
        "alpha_sum": float(res["alpha"].sum()), "alpha_norm": float(np.linalg.norm(res["alpha"])),
        "elbow_count": int(np.sum((a > wl.tau - 1 + 1e-9) & (a < wl.tau - 1e-9))),
        "seconds": {"gram": t_gram, "solve": t_solve},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lap_large_n20000.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
