#!/usr/bin/env python
"""Benchmark: kernel quantile regression solve seconds to KKT <= 1e-6.

Workload (default): n = 200000, p = 50, x ~ U[-1,1]^p,
y = sum_j sin(x_j)/sqrt(p) + (0.5 + |x_1|) N(0,1), Laplacian kernel gamma = 1/p,
tau = 0.25, lambda = 1e-4, on-the-fly Gram tiles.

One step = RPCholesky set-up on the device-resident X (Sec. 3) + a full
two-phase solve (Alg. 1, then Alg. 2/3) to max(eta_kkt, eta_gap) <= 1e-6.
Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KQR solve sec to KKT≤1e-6 at n=200k; fused K·V TFLOP/s and % of roofline"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# Gram products (FP32 + FP64-class) of one solve of the default workload with
# the library's default constants; the reference arm, which cannot run the
# solver, scales the oracle's per-product time by it.
REF_PRODUCTS_PER_SOLVE = 330


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lap_large")
    ap.add_argument("--n", type=int, default=0, help="override n (testing only)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--rank0", type=int, default=1024, help="initial RPCholesky rank (library default: ceil(sqrt n))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "gram"],
                    help="gram: time --matvecs FP32 and FP64-class Gram products only (kernel profiling)")
    ap.add_argument("--matvecs", type=int, default=3)
    return ap.parse_args()


def workload(args, seed=0):
    from paper_2510_07929_gb300 import workloads as W

    gen = W.GENERATORS[args.workload]
    return gen(n=args.n, seed=seed) if args.n else gen(seed=seed)


def describe(wl, args):
    return (f"{wl.name} n={wl.n} p={wl.p} {wl.kind} gamma={wl.gamma:g} tau={wl.tau:g} lambda={wl.lam:g} "
            f"tol={args.tol:g}")


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[2:6]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing
def oracle_matvec_seconds(wl, rows: int = 96, seed: int = 0):
    """Seconds for one full FP64 oracle K.v on this workload, from a timed
    sample of ``rows`` rows scaled by n / rows."""
    from oracle import kqr_oracle as O

    rng = np.random.default_rng(seed)
    idx = rng.choice(wl.n, size=min(rows, wl.n), replace=False)
    v = rng.standard_normal(wl.n)
    t0 = time.perf_counter()
    O.kmatvec(wl.X, v, wl.kind, wl.gamma, rows=idx)
    dt = time.perf_counter() - t0
    return dt * wl.n / idx.size, idx.size, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args)
    times = []
    rows = 64 if wl.n >= 100000 else max(8, min(wl.n, 2000))
    for i in range(args.warmup + args.steps):
        per_mv, nrows, dt = oracle_matvec_seconds(wl, rows=rows, seed=i)
        est = per_mv * REF_PRODUCTS_PER_SOLVE
        if i >= args.warmup:
            times.append(est)
    value = statistics.mean(times)
    sample = (f"FP64 numpy oracle K.v on {rows} random rows of the workload per step, scaled by n/rows to one "
              f"product and by {REF_PRODUCTS_PER_SOLVE} Gram products per solve")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(wl, args)},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    wl = workload(args, seed=rank)
    opts = dict(rank0=args.rank0, verbose=1 if args.verbose else 0)
    prob = kqr.Problem(wl.X, wl.y, wl.kind, wl.gamma, **opts)
    stream = torch.cuda.Stream()
    prob.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        prob.refactor()
        return prob.solve(wl.tau, wl.lam, args.tol)

    infos = []
    for _ in range(args.warmup):
        _, _, kkt, info = step()
        infos.append(info)
    barrier()
    prob.profile(True)
    launches0 = prob.launches
    clocks = ClockSampler(local)
    clocks.start()
    step_ms = []
    setup_ms = []
    kkts = []
    barrier()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(float(len(step_ms)))              # L2 flush outside the step's events
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        em = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.refactor()
        em.record(stream)
        _, _, kkt, info = prob.solve(wl.tau, wl.lam, args.tol)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        setup_ms.append(e0.elapsed_time(em))
        kkts.append(kkt)
        infos.append(info)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = prob.launches - launches0
    n32, ms32 = prob.profile_read(0)
    nhp, mshp = prob.profile_read(1)
    prob.profile(False)
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = world * args.steps
    value = total_ms / 1e3 / units                    # seconds per solve, whole job

    # e2e through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Xp = torch.empty(wl.X.shape, dtype=torch.float64, pin_memory=True)
        yp = torch.empty(wl.y.shape, dtype=torch.float64, pin_memory=True)
        Xp.numpy()[:] = wl.X
        yp.numpy()[:] = wl.y
        e2e_s = []
        barrier()
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with kqr.Problem(Xp.numpy(), yp.numpy(), wl.kind, wl.gamma, rank0=args.rank0) as p2:
                alpha, beta, kkt2, _ = p2.solve(wl.tau, wl.lam, args.tol)
            torch.cuda.synchronize()
            e2e_s.append(time.perf_counter() - t0)
        barrier()
        tot = sum(e2e_s)
        if dist is not None:
            t = torch.tensor([tot], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        e2e = {"value": tot / units, "unit": "s", "h2d_bytes_per_step": int(wl.X.nbytes + wl.y.nbytes),
               "d2h_bytes_per_step": int(wl.n * 8 + 16)}

    last = infos[-1]
    n, p = wl.n, wl.p
    # the single-vector products form each off-diagonal tile once: n(n+1)/2 entries,
    # each with two FFMAs (row and column sums)
    entries = float(n) * float(n + 1) / 2.0
    sym_extra = 1
    roofline = None
    if n32 > 0:
        avg_s = ms32 / n32 / 1e3
        if wl.kind == "laplacian":
            ops_per_entry = 2 * p + 1 + sym_extra   # FADD + FADD|.| per feature; FFMA with v_j (and v_i)
            flops_per_entry = 3 * p + 4             # sub, abs, add per feature; scale, exp, multiply, add
        else:
            ops_per_entry = p + 3 + sym_extra
            flops_per_entry = 2 * p + 5
        peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12   # Top/s, FP32 pipe lane-ops
        achieved = entries * ops_per_entry / avg_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                    "traffic": None, "kernel": "gram_f32_sym_kernel (FP32 Gram tiles, symmetric)",
                    "launches": n32, "avg_ms": ms32 / n32, "entries_per_launch": entries,
                    "kv_tflops_effective": float(n) * n * flops_per_entry / avg_s / 1e12,
                    "peak_basis": "152 SM x 128 FP32 lanes x 2070 MHz (derived, not measured)"}
    hp = {"launches": nhp, "avg_ms": (mshp / nhp) if nhp else None}

    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32,f64", "data": "synthetic",
            "config": {"workload": describe(wl, args), "n": n, "p": p, "kernel": wl.kind, "rank0": args.rank0,
                       "xi": 1e-6, "preconditioner": "RPCholesky + floored residual diagonal (Woodbury)",
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1gpu"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
            "high_precision_gram": hp,
            "solve": {"kkt": max(kkts), "phase1_iters": last["phase1_iters"], "alm_iters": last["phase2_iters"],
                      "newton_steps": last["newton_steps"], "cg_iters": last["pcg_iters"],
                      "gram_fp32": last["matvecs_fp32"], "gram_high": last["matvecs_high"], "rank": last["rank"],
                      "core_builds": last["core_builds"],
                      "eta_gap": last["eta_gap"], "wall_s": t_wall, "setup_s": sum(setup_ms) / 1e3 / args.steps}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_mv, nrows, dt = oracle_matvec_seconds(wl, rows=96 if n >= 100000 else min(n, 2000))
        products = last["matvecs_fp32"] + last["matvecs_high"]
        line["cpu_baseline"] = {
            "value": per_mv * products, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 numpy oracle K.v on {nrows} random rows ({dt:.1f} s), scaled by n/rows to one product "
                       f"and by the {products} Gram products this solve used; set-up and O(n) work not counted")}
    prob.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_gram(args):
    """Kernel-only timing of the Gram products on the resident problem."""
    import torch

    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    wl = workload(args)
    prob = kqr.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=args.rank0)
    V = torch.from_numpy(np.random.default_rng(0).standard_normal(wl.n)).cuda()
    U = torch.empty_like(V)
    out = {"mode": "gram", "config": {"workload": describe(wl, args)}}
    for name, prec in (("fp32", kqr.PREC_FP32), ("high", kqr.PREC_HIGH)):
        prob.kmatvec_dev(V, U, prec)
        torch.cuda.synchronize()
        prob.profile(True)
        for _ in range(args.matvecs):
            prob.kmatvec_dev(V, U, prec)
        cnt, ms = prob.profile_read(0 if prec == kqr.PREC_FP32 else 1)
        prob.profile(False)
        out[name] = {"launches": cnt, "avg_ms": ms / max(cnt, 1)}
    prob.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "gram":
        return run_gram(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
