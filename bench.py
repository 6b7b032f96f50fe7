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
FP32_LANES_PER_SM = 128          # FP32 FFMA/FADD lanes per SM (measured unit rate, see the design notes)
XU_LANES_PER_SM = 32             # MUFU ex2 per SM and clock (microbenchmark; ncu's XU-pipe counter agrees)
TF32_PER_BF16 = 1.1 / 2.25       # nominal dense TF32 / bf16 tensor rate
SM_COUNT_FALLBACK = 152          # used only when the device cannot be queried
SM_MAX_MHZ_FALLBACK = 2070.0     # used only when nvidia-smi gives no maximum clock
# DRAM bytes (read + write) per launch of gram_f32_sym_kernel on the n = 200000, p = 50
# Laplacian workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum).
SYM_LAPLACIAN_TRAFFIC = {(200000, 50): 42469632 + 8192}
# Rows of the workload the oracle's full reference solve uses (dense FP64, Alg. 1
# then Alg. 2/3): the full n = 200000 problem is far beyond it in a bench run.
REF_SUBSAMPLE_ROWS = 2000
# Seconds of multi-core oracle K.v work that the CPU baseline's projection samples.
CPU_SAMPLE_SECONDS = 15.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lap_large")
    ap.add_argument("--n", type=int, default=0, help="override n (testing only)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--tau", type=float, default=0.0, help="override the workload's tau")
    ap.add_argument("--rank0", type=int, default=1024, help="initial RPCholesky rank (library default: ceil(sqrt n))")
    ap.add_argument("--gram-store", type=int, default=0,
                    help="CG products from a stored K: 0 on the fly (the headline workload's stated form), "
                         "1 always, 2 when it fits (library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "gram", "precision", "path", "grad", "batch", "grid"],
                    help="gram: time --matvecs FP32 and FP64-class Gram products only (kernel profiling)")
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--ncu-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--path-gamma", type=float, default=0.1)
    ap.add_argument("--path-tau", type=float, default=0.5)
    ap.add_argument("--path-lambdas", type=int, default=50)
    ap.add_argument("--path-precond", type=int, default=0, help="0 Nystrom+diag, 1 paper, 2 none (NALM)")
    ap.add_argument("--path-kernel", default="rbf", choices=["rbf", "laplacian"])
    ap.add_argument("--path-first", type=int, nargs=2, default=None, metavar=("START", "STOP"),
                    help="--mode path: solve only lambdas[START:STOP] of the grid")
    ap.add_argument("--path-cg-high", type=int, default=2,
                    help="--mode path: CG products 0 FP32, 1 FP64-class, 2 FP64-class when K is numerically low-rank")
    ap.add_argument("--prec-taus", default="0.5", help="comma-separated tau values for --mode precision")
    ap.add_argument("--batch-p-in-smem", action="store_true",
                    help="--mode batch: stage the Gram tile through shared memory instead of tensor memory")
    ap.add_argument("--time-limit", type=float, default=600.0, help="per-solve wall-clock limit (s) in the study modes")
    ap.add_argument("--grid-problems", type=int, default=64, help="--mode grid: number of problems")
    ap.add_argument("--grid-nmax", type=int, default=20000, help="--mode grid: n_b ~ U{1000..nmax}")
    ap.add_argument("--grid-side", type=int, default=8, help="--mode grid: taus x lambdas = side x side pairs")
    ap.add_argument("--grid-workers", type=int, default=4, help="--mode grid: problems solved at a time")
    ap.add_argument("--grid-lmin", type=float, default=1e-5, help="--mode grid: smallest lambda of the grid")
    ap.add_argument("--grid-nl", type=int, default=0, help="--mode grid: number of lambdas (0: --grid-side)")
    ap.add_argument("--grid-seq-sample", type=int, default=32,
                    help="--mode grid: pairs solved one at a time through kqr_solve for the comparison")
    return ap.parse_args()


def workload(args, seed=0):
    from paper_2510_07929_gb300 import workloads as W

    gen = W.GENERATORS[args.workload]
    kw = {"tau": args.tau} if getattr(args, "tau", 0.0) else {}
    return gen(n=args.n, seed=seed, **kw) if args.n else gen(seed=seed, **kw)


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
def oracle_matvec_seconds(wl, budget_s: float = CPU_SAMPLE_SECONDS, seed: int = 0):
    """Seconds for one full FP64 oracle K.v on this workload, projected from a
    timed multi-core run of the oracle's C product (all host cores) over a
    random row sample sized to about ``budget_s``.  Returns (seconds per full
    product, rows sampled, seconds measured, threads)."""
    from oracle import native as N

    rng = np.random.default_rng(seed)
    v = rng.standard_normal(wl.n)
    probe = rng.choice(wl.n, size=min(wl.n, 64 * N.threads()), replace=False)
    t0 = time.perf_counter()
    N.kmatvec(wl.X, v, wl.kind, wl.gamma, rows=probe)
    per_row = (time.perf_counter() - t0) / probe.size
    rows = int(min(wl.n, max(probe.size, budget_s / max(per_row, 1e-12))))
    idx = rng.choice(wl.n, size=rows, replace=False)
    t0 = time.perf_counter()
    N.kmatvec(wl.X, v, wl.kind, wl.gamma, rows=idx)
    dt = time.perf_counter() - t0
    return dt * wl.n / rows, rows, dt, N.threads()


def oracle_subsample_solve(wl, rows: int, tol: float, seed: int = 0):
    """The oracle's full two-phase solve (Alg. 1 then Alg. 2/3, exact dense
    FP64 solves) of the problem restricted to a random subsample of ``rows``
    points of the workload.  Returns (seconds, eta_kkt reached, rows)."""
    from oracle import kqr_oracle as O
    from oracle import native as N

    idx = np.sort(np.random.default_rng(seed).choice(wl.n, size=min(rows, wl.n), replace=False))
    X, y = wl.X[idx], wl.y[idx]
    t0 = time.perf_counter()
    K = N.gram(X, X, wl.kind, wl.gamma)
    res = O.solve_dense(K, y, wl.tau, wl.lam, tol=tol)
    return time.perf_counter() - t0, max(res["kkt"]["eta_kkt"], res["kkt"]["eta_gap"]), idx.size


def device_sm_count() -> int:
    try:
        import torch

        return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        return SM_COUNT_FALLBACK


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (the job finishes when every replica has)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput_value(total_ms: float, world: int, steps: int) -> float:
    """Seconds per solve over the whole job: every rank solves one replica per step."""
    return total_ms / 1e3 / (world * steps)


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def stored_k_roofline(n: int, launches: int, ms: float) -> dict:
    """The stored-K product reads every stored 128 x 128 FP32 tile once per launch."""
    t = (n + 127) // 128
    nbytes = t * (t + 1) // 2 * 128 * 128 * 4 + 8 * n
    peak = measured_peaks().get("hbm_gbs")
    basis = "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    if not peak:
        peak, basis = 6800.0, "fallback 6.8 TB/s"
    achieved = nbytes / (ms / launches / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "kstore_gemv_kernel (stored K, symmetric)", "launches": launches,
            "avg_ms": ms / launches, "bytes_per_launch": nbytes,
            "work_per_entry": "4 bytes per stored entry (upper-triangle tiles) + v and u", "peak_basis": basis}


def rbf_tc_roofline(n: int, p: int, launches: int, ms: float, sm_count: int, sm_mhz: float, f16: bool) -> dict:
    """The symmetric tcgen05 RBF tiles: per entry one exp2 on the MUFU (XU) pipe, three
    FFMAs (exponent, row and column products) and 2p tensor flops per product term (three
    terms for FP32 accuracy: fp16 parts when the row factors fold and 3p <= 128, else TF32
    parts); n(n+1)/2 entries per launch."""
    entries = float(n) * float(n + 1) / 2.0
    avg_s = ms / launches / 1e3
    xu_peak = sm_count * XU_LANES_PER_SM * sm_mhz * 1e6 / 1e12          # T exp2/s
    xu = entries / avg_s / 1e12
    fma_peak = sm_count * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    fma = 3.0 * entries / avg_s / 1e12
    bf16 = measured_peaks().get("bf16_tflops")
    ratio = 1.0 if f16 else TF32_PER_BF16
    tc_peak = (bf16 if bf16 else 1900.0) * ratio
    tc = 6.0 * p * entries / avg_s / 1e12
    return {"bound": "alu", "achieved": xu, "peak": xu_peak, "unit": "T exp2/s", "frac": xu / xu_peak,
            "traffic": None, "kernel": "gram_rbf_tc_sym_kernel (tcgen05 RBF tiles, symmetric)",
            "launches": launches, "avg_ms": ms / launches, "entries_per_launch": entries,
            "work_per_entry": "1 exp2 (MUFU) + 3 FFMA; 6p tensor flops (three terms, "
                              + ("fp16 parts concatenated along K)" if f16 else "TF32 parts)"),
            "peak_basis": f"{sm_count} SMs x {XU_LANES_PER_SM} ex2 per SM and clock x {sm_mhz:g} MHz (ex2 rate from "
                          f"a microbenchmark, consistent with ncu's XU-pipe utilisation of this kernel)",
            "fma_convention": {"achieved": fma, "peak": fma_peak, "unit": "Top/s", "frac": fma / fma_peak},
            "tensor_convention": {"achieved": tc, "peak": tc_peak, "unit": "TFLOP/s", "frac": tc / tc_peak,
                                  "peak_basis": ("measured bf16 dense (fp16 runs at the bf16 rate)" if f16 else
                                                 "measured bf16 dense x nominal TF32/bf16 ratio 1.1/2.25")
                                  + ("" if bf16 else " (fallback 1.9 PFLOP/s bf16)")}}


def bench_config(wl, args, world: int) -> dict:
    """The bench line's config, shared by both arms."""
    return {"workload": describe(wl, args), "n": wl.n, "p": wl.p, "kernel": wl.kind, "rank0": args.rank0,
            "xi": 1e-10, "preconditioner": "RPCholesky + floored residual diagonal (Woodbury)",
            "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1gpu"}


def run_reference(args):
    """The oracle as it stands on the host cores.  Each step is a bounded
    sample of the workload that the oracle completes: its full two-phase solve
    (Alg. 1, Alg. 2/3, dense FP64) of the problem on a random subsample of
    REF_SUBSAMPLE_ROWS points.  ``value`` is the measured seconds of one such
    solve; the projection of one full-size solve's Gram products is reported
    beside it, labelled as a projection."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import native as N

    wl = workload(args)
    times, reached = [], []
    for i in range(args.warmup + args.steps):
        dt, kkt, rows = oracle_subsample_solve(wl, REF_SUBSAMPLE_ROWS, args.tol, seed=i)
        if i >= args.warmup:
            times.append(dt)
            reached.append(kkt)
    value = statistics.mean(times)
    per_mv, nrows, dt_mv, threads = oracle_matvec_seconds(wl, budget_s=min(CPU_SAMPLE_SECONDS, 5.0))
    sample = (f"oracle full solve (Alg. 1 then Alg. 2/3, exact dense FP64 solves, K from its definition) of the "
              f"problem on a random {rows}-point subsample of the workload, to max(eta_kkt, eta_gap) <= {args.tol:g} "
              f"(reached {max(reached):.1e}); {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(wl, args, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "full_size_projection": {
                "kind": "projection", "unit": "s per FP64 K.v at full size", "value": per_mv,
                "sample": f"oracle C K.v on {nrows} random rows ({dt_mv:.1f} s, {threads} threads), scaled by n/rows"}}
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
    opts = dict(rank0=args.rank0, verbose=1 if args.verbose else 0, gram_store=args.gram_store)
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
    # kernel timing (CUDA events around every Gram launch) is kept off for small
    # problems: it disables the CUDA graphs of the CG iterations there
    profiled = wl.n > 32768
    if profiled:
        prob.profile(True)
    launches0 = prob.launches
    clocks = ClockSampler(local)
    clocks.start()
    step_ms = []
    setup_ms = []
    kkts = []
    barrier()
    if args.ncu_window:
        torch.cuda.profiler.start()
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
    if args.ncu_window:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    launches = prob.launches - launches0
    n32, ms32 = prob.profile_read(0)
    nhp, mshp = prob.profile_read(1)
    nks, msks = prob.profile_read(2)
    prob.profile(False)
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    units = world * args.steps
    value = job_throughput_value(total_ms, world, args.steps)

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
            with kqr.Problem(Xp.numpy(), yp.numpy(), wl.kind, wl.gamma, rank0=args.rank0,
                             gram_store=args.gram_store) as p2:
                alpha, beta, kkt2, _ = p2.solve(wl.tau, wl.lam, args.tol)
            torch.cuda.synchronize()
            e2e_s.append(time.perf_counter() - t0)
        barrier()
        tot = max_over_ranks(sum(e2e_s), dist, "cuda")
        e2e = {"value": tot / units, "unit": "s", "h2d_bytes_per_step": int(wl.X.nbytes + wl.y.nbytes),
               "d2h_bytes_per_step": int(wl.n * 8 + 16)}

    last = infos[-1]
    n, p = wl.n, wl.p
    # the single-vector products form each off-diagonal tile once: n(n+1)/2 entries,
    # each with two FFMAs (row and column sums)
    entries = float(n) * float(n + 1) / 2.0
    sm_count = device_sm_count()
    sm_mhz = clk.get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK
    roofline = None
    if nks > n32:
        roofline = stored_k_roofline(n, nks, msks)
    elif n32 > 0 and wl.kind == "rbf":
        # the library folds the row factors when every gamma log2(e) |x_i - mean|^2 < 60
        xc = wl.X - wl.X.mean(axis=0)
        fold = float(wl.gamma * np.log2(np.e) * np.max(np.sum(xc * xc, axis=1))) < 60.0
        roofline = rbf_tc_roofline(n, p, n32, ms32, sm_count, sm_mhz, f16=fold and 3 * p <= 128)
    elif n32 > 0:
        avg_s = ms32 / n32 / 1e3
        ops_per_entry = 2 * p + 2               # FADD + FADD|.| per feature; FFMA with v_j and with v_i
        flops_per_entry = 3 * p + 4             # sub, abs, add per feature; scale, exp, multiply, add
        peak = sm_count * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12         # Top/s, FP32 pipe lane operations
        achieved = entries * ops_per_entry / avg_s / 1e12
        flop_peak = 2.0 * peak                                               # FFMA = 2 flops per lane and clock
        flop_achieved = entries * flops_per_entry / avg_s / 1e12
        traffic = SYM_LAPLACIAN_TRAFFIC.get((n, p))
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                    "traffic": traffic, "traffic_unit": "bytes per launch",
                    "kernel": "gram_f32_sym_kernel (FP32 Gram tiles, symmetric)",
                    "launches": n32, "avg_ms": ms32 / n32, "entries_per_launch": entries,
                    "work_per_entry": f"{ops_per_entry} FP32-pipe lane operations (FADD, FADD|.| per feature; "
                                      f"two FFMAs for the row and column sums)",
                    "peak_basis": f"{sm_count} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:g} MHz "
                                  f"(max SM clock sampled by nvidia-smi); derived from unit counts and clocks",
                    "flop_convention": {
                        "achieved": flop_achieved, "peak": flop_peak, "unit": "TFLOP/s", "frac": flop_achieved / flop_peak,
                        "flops_per_entry": flops_per_entry, "entries": "n(n+1)/2 formed per launch",
                        "peak_basis": "SMs x 128 lanes x 2 flops (FFMA) x clock"}}
    hp = {"launches": nhp, "avg_ms": (mshp / nhp) if nhp else None}

    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32,f64", "data": "synthetic",
            "config": bench_config(wl, args, world),
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
            "high_precision_gram": hp,
            "solve": {"kkt": max(kkts), "phase1_iters": last["phase1_iters"], "alm_iters": last["phase2_iters"],
                      "newton_steps": last["newton_steps"], "cg_iters": last["pcg_iters"],
                      "gram_fp32": last["matvecs_fp32"], "gram_high": last["matvecs_high"], "rank": last["rank"],
                      "core_builds": last["core_builds"],
                      "eta_gap": last["eta_gap"], "wall_s": t_wall, "setup_s": sum(setup_ms) / 1e3 / args.steps}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_mv, nrows, dt, threads = oracle_matvec_seconds(wl)
        products = last["matvecs_fp32"] + last["matvecs_high"]
        line["cpu_baseline"] = {
            "value": per_mv * products, "unit": "s", "cores": threads, "kind": "projection", "source": "oracle",
            "sample": (f"oracle C FP64 K.v (OpenMP, {threads} threads) on {nrows} random rows, {dt:.1f} s measured, "
                       f"scaled by n/rows to one product ({per_mv:.1f} s) and by the {products} Gram products this "
                       f"solve used; set-up and O(n) work not counted, so a lower bound on the oracle's solve")}
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
    t0 = time.perf_counter()
    prob = kqr.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=args.rank0, gram_store=args.gram_store)
    create_s = time.perf_counter() - t0
    V = torch.from_numpy(np.random.default_rng(0).standard_normal(wl.n)).cuda()
    U = torch.empty_like(V)
    out = {"mode": "gram", "config": {"workload": describe(wl, args), "gram_store": args.gram_store},
           "create_s": create_s}
    for name, prec in (("fp32", kqr.PREC_FP32), ("high", kqr.PREC_HIGH)):
        prob.kmatvec_dev(V, U, prec)
        torch.cuda.synchronize()
        prob.profile(True)
        for _ in range(args.matvecs):
            prob.kmatvec_dev(V, U, prec)
        cnt, ms = prob.profile_read(0 if prec == kqr.PREC_FP32 else 1)
        if prec == kqr.PREC_FP32 and cnt == 0:
            cnt, ms = prob.profile_read(2)
            name = "fp32_stored"
            stored_bytes = (wl.n + 127) // 128 * ((wl.n + 127) // 128 + 1) // 2 * 65536
            out["stored_bytes"] = stored_bytes
            out["stored_gbs"] = stored_bytes / (ms / max(cnt, 1) / 1e3) / 1e9
        prob.profile(False)
        out[name] = {"launches": cnt, "avg_ms": ms / max(cnt, 1)}
    prob.close()
    print(json.dumps(out), flush=True)
    return 0


def run_precision(args):
    """Mixed-precision comparison on the RBF workload (n = 50000, p = 20,
    lambda = 1e-3): solve seconds to the same KKT tolerance with (a) FP32
    CUDA-core Gram products, (b) FP32 products with the cross term on tcgen05
    (three TF32 terms), (c) TF32 tensor-core products inside CG refined against
    FP32 residuals.  One JSON line per run, then a summary line."""
    import torch

    from paper_2510_07929_gb300 import build, workloads as W

    build.build()
    from paper_2510_07929_gb300 import kqr

    n = args.n or 50000
    configs = {"fp32_cuda_cores": dict(rbf_tensor_cores=0), "fp32_tcgen05": dict(rbf_tensor_cores=1),
               "tf32_tcgen05_refined": dict(rbf_tensor_cores=1, cg_tf32=1)}
    taus = [float(t) for t in args.prec_taus.split(",")]
    runs = []
    for tau in taus:
        wl = W.rbf_mid(n=n, tau=tau)
        for name, cfg in configs.items():
            with kqr.Problem(wl.X, wl.y, wl.kind, wl.gamma, rank0=args.rank0, time_limit_s=args.time_limit,
                             **cfg) as prob:
                if args.warmup > 0:
                    prob.solve(wl.tau, wl.lam, args.tol, allow_not_converged=True)
                torch.cuda.synchronize()
                prob.profile(True)
                t0 = time.perf_counter()
                _, _, kkt, info = prob.solve(wl.tau, wl.lam, args.tol, allow_not_converged=True)
                dt = time.perf_counter() - t0
                n_cg, ms_cg = prob.profile_read(0)             # CG Gram products (FP32 or TF32 tiles)
                n_hp, ms_hp = prob.profile_read(1)             # FP64-class products
                prob.profile(False)
            run = {"tau": tau, "config": name, "status": info["status"], "seconds": dt,
                   "cg_gram_seconds": ms_cg / 1e3, "high_gram_seconds": ms_hp / 1e3, "kkt": kkt,
                   "eta_gap": info["eta_gap"], "gram_fp32": info["matvecs_fp32"], "gram_tf32": info["matvecs_low"],
                   "gram_high": info["matvecs_high"], "cg_iters": info["pcg_iters"],
                   "newton_steps": info["newton_steps"], "cg_truncations": info["cg_truncations"]}
            runs.append(run)
            print(json.dumps(dict(mode="precision_run", n=n, **run)), flush=True)
    out = {"mode": "precision", "workload": f"rbf_mid n={n} p=20 gamma=1/p lambda=1e-3 tol={args.tol:g}"}
    for tau in taus:
        for key in ("seconds", "cg_gram_seconds"):
            r = {x["config"]: x[key] for x in runs if x["tau"] == tau}
            out[f"speedup_{key}_tau{tau}"] = {
                "tcgen05_fp32_vs_cuda_fp32": r["fp32_cuda_cores"] / r["fp32_tcgen05"],
                "mixed_vs_cuda_fp32": r["fp32_cuda_cores"] / r["tf32_tcgen05_refined"],
                "mixed_vs_tcgen05_fp32": r["fp32_tcgen05"] / r["tf32_tcgen05_refined"]}
    print(json.dumps(out), flush=True)
    return 0


# Total seconds of a 50-lambda path in the paper's Table 1 (MATLAB, Intel Xeon Platinum
# 8375C, 128 cores; RBF kernel, p = 2 generator of Sec. 4.1, tolerance 1e-8), keyed by
# (n, gamma, tau).  Context only: another machine, language and tolerance handling.
PAPER_TABLE1_S = {
    (5000, 0.1, 0.1): 45, (5000, 0.1, 0.5): 34, (5000, 0.1, 0.9): 36,
    (10000, 0.1, 0.1): 146, (10000, 0.1, 0.5): 152, (10000, 0.1, 0.9): 161,
    (20000, 0.1, 0.1): 881, (20000, 0.1, 0.5): 863, (20000, 0.1, 0.9): 801,
    (5000, 0.01, 0.1): 40, (5000, 0.01, 0.5): 35, (5000, 0.01, 0.9): 35,
    (10000, 0.01, 0.1): 121, (10000, 0.01, 0.5): 132, (10000, 0.01, 0.9): 144,
    (20000, 0.01, 0.1): 763, (20000, 0.01, 0.5): 763, (20000, 0.01, 0.9): 765,
    (5000, 0.001, 0.1): 28, (5000, 0.001, 0.5): 29, (5000, 0.001, 0.9): 31,
    (10000, 0.001, 0.1): 83, (10000, 0.001, 0.5): 97, (10000, 0.001, 0.9): 111,
    (20000, 0.001, 0.1): 501, (20000, 0.001, 0.5): 512, (20000, 0.001, 0.9): 514,
}


# Total seconds of a 50-lambda path in the paper's Table 2 (Laplacian kernel, gamma = 0.1,
# same generator, machine and tolerance as Table 1), keyed by (n, tau).  Context only.
PAPER_TABLE2_S = {
    (5000, 0.1): 139, (5000, 0.5): 143, (5000, 0.9): 141,
    (10000, 0.1): 316, (10000, 0.5): 323, (10000, 0.9): 322,
    (20000, 0.1): 1907, (20000, 0.5): 1899, (20000, 0.9): 1898,
}


def run_path(args):
    """A 50-lambda regularisation path (lambda log-spaced in [1e-2, 1]) on the
    paper's p = 2 generator (Sec. 4.1), RBF or Laplacian kernel (--path-kernel),
    tolerance 1e-8 per solve, one handle (the RPCholesky factor is built once,
    as in Sec. 3), no warm start across lambda.  One JSON line per lambda, then
    a summary line."""
    import torch

    from paper_2510_07929_gb300 import build, workloads as W

    build.build()
    from paper_2510_07929_gb300 import kqr

    n = args.n or 5000
    tol = 1e-8
    wl = W.yuan2006(n=n, gamma=args.path_gamma, tau=args.path_tau)
    kind = args.path_kernel
    lams = np.logspace(-2, 0, args.path_lambdas)
    if args.path_first:
        lams = lams[args.path_first[0]:args.path_first[1]]
    name = f"yuan2006 n={n} p=2 {kind} gamma={args.path_gamma:g} tau={args.path_tau:g}"
    t0 = time.perf_counter()
    prob = kqr.Problem(wl.X, wl.y, kind, wl.gamma, precond=args.path_precond, time_limit_s=args.time_limit,
                       cg_high=args.path_cg_high)
    t_setup = time.perf_counter() - t0
    per, worst, unsolved, products = [], 0.0, 0, 0
    for lam in lams:
        t1 = time.perf_counter()
        _, _, kkt, info = prob.solve(wl.tau, float(lam), tol, allow_not_converged=True)
        torch.cuda.synchronize()
        per.append(time.perf_counter() - t1)
        worst = max(worst, max(kkt, info["eta_gap"]))
        unsolved += int(info["status"] != kqr.OK)
        products += info["matvecs_fp32"] + info["matvecs_high"]
        print(json.dumps({"mode": "path_lambda", "workload": name, "lambda": float(lam), "status": info["status"],
                          "kkt": kkt, "eta_gap": info["eta_gap"], "seconds": per[-1], "cg_iters": info["pcg_iters"],
                          "newton_steps": info["newton_steps"], "alm_iters": info["phase2_iters"],
                          "cg_truncations": info["cg_truncations"], "gram_fp32": info["matvecs_fp32"],
                          "gram_high": info["matvecs_high"], "cg_high_used": info["cg_high_used"],
                          "rank": info["rank"]}), flush=True)
    prob.close()
    total = t_setup + sum(per)
    paper = (PAPER_TABLE1_S.get((n, args.path_gamma, args.path_tau)) if kind == "rbf"
             else PAPER_TABLE2_S.get((n, args.path_tau)) if args.path_gamma == 0.1 else None)
    out = {"mode": "path", "workload": name,
           "lambdas": len(lams), "tol": tol, "precond": ["nystrom_diag", "paper", "none"][args.path_precond],
           "cg_products": ["fp32", "fp64-class", "auto"][args.path_cg_high],
           "total_s": total, "setup_s": t_setup, "median_solve_s": float(np.median(per)), "max_solve_s": max(per),
           "worst_kkt_or_gap": worst, "not_converged": unsolved, "gram_products": products,
           "time_limit_s_per_lambda": args.time_limit,
           "paper_total_s": paper, "paper_hardware": "MATLAB, Xeon Platinum 8375C, 128 cores (tables 1-2)"}
    print(json.dumps(out), flush=True)
    return 0


def run_grad(args):
    """Held-out loss gradient on the n = 20000 (+ 5000 held-out) p = 16 RBF
    workload (x ~ U[0,1]^16, gamma = 0.25, lambda = 0.1, tau = 0.5): seconds of
    the forward solve and of kqr_heldout_grad, with a central-difference check
    of the log-lambda and log-gamma derivatives from four more solves."""
    import torch

    from paper_2510_07929_gb300 import build, workloads as W

    build.build()
    from paper_2510_07929_gb300 import kqr

    n = args.n or 20000
    nh = max(1, n // 4)
    tau, lam, tol = 0.5, 0.1, 1e-8
    tr = W.rbf_small(n=n, p=16, seed=0, tau=tau, lam=lam)
    ho = W.rbf_small(n=nh, p=16, seed=1000, tau=tau, lam=lam)
    gamma = 0.25

    def fwd(gm, lm, grad=True):
        with kqr.Problem(tr.X, tr.y, "rbf", gm) as prob:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, kkt, info = prob.solve(tau, lm, tol)
            t1 = time.perf_counter()
            res = prob.heldout_grad(ho.X, ho.y, want_dX=grad)
            t2 = time.perf_counter()
        return res, t1 - t0, t2 - t1, kkt, info

    fwd(gamma, lam)                                   # warm-up (build, allocator)
    (loss, dg, dl, dX), t_solve, t_grad, kkt, info = fwd(gamma, lam)
    h = 1e-4
    fl = [fwd(gamma, lam * np.exp(s * h), False)[0][0] for s in (1, -1)]
    fg = [fwd(gamma * np.exp(s * h), lam, False)[0][0] for s in (1, -1)]
    out = {"mode": "grad", "workload": f"rbf n={n} + {nh} held-out, p=16, gamma={gamma:g}, lambda={lam:g}, tau={tau:g}",
           "solve_s": t_solve, "grad_s": t_grad, "kkt": kkt, "loss": loss, "d_loglambda": dl, "d_loggamma": dg,
           "dX_max_abs": float(np.abs(dX).max()),
           "fd_d_loglambda": (fl[0] - fl[1]) / (2 * h), "fd_d_loggamma": (fg[0] - fg[1]) / (2 * h),
           "fd_step_log": h}
    print(json.dumps(out), flush=True)
    return 0


def batch_workload(seed: int = 0):
    """64 problems, n_b ~ U{1000..20000}, x ~ U[0,1]^8, RBF gamma = 1/8, and 64
    right-hand sides per problem (one per (tau, lambda) pair of an 8 x 8 grid)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1000, 20001, size=64)
    Xs = [rng.random((int(n), 8)) for n in sizes]
    V = rng.standard_normal((int(sizes.sum()), 64))
    return Xs, V


def run_batch(args):
    """Batched multi-RHS products U_b = K_b V_b on the tensor cores: seconds per
    batched product (all 64 problems, 64 right-hand sides), TFLOP/s at 2p + 2m
    = 144 tensor flops per Gram entry, against the measured bf16 dense peak
    scaled by the nominal TF32/bf16 ratio (1.1 / 2.25)."""
    import torch

    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    Xs, V = batch_workload()
    sizes = [x.shape[0] for x in Xs]
    entries = float(sum(n * n for n in sizes))
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    bf16 = peaks.get("bf16_tflops", 1900.0)
    peak = bf16 * 1.1 / 2.25
    with kqr.Batch(Xs, 0.125, p_in_smem=args.batch_p_in_smem) as bt:
        stream = torch.cuda.Stream()
        bt.set_stream(stream)
        Vd = torch.tensor(V, device="cuda")
        Ud = torch.empty_like(Vd)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for _ in range(max(3, args.warmup)):
            bt.kmatmul_dev(Vd, Ud)
        torch.cuda.synchronize()
        steps = max(args.steps, 10)
        bt.profile(True)
        times = []
        clocks = ClockSampler(0)
        clocks.start()
        for k in range(steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.kmatmul_dev(Vd, Ud)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        clk = clocks.stop()
        nk, ms_k = bt.profile_read()
        bt.profile(False)
        # e2e: host V in pinned memory, host U, copies inside the timed region
        Vh = torch.empty(V.shape, dtype=torch.float64, pin_memory=True)
        Vh.numpy()[:] = V
        t0 = time.perf_counter()
        U = bt.kmatmul(Vh.numpy())
        e2e_s = time.perf_counter() - t0
    ms = statistics.median(times)
    kern_ms = ms_k / max(nk, 1)
    flops = entries * (2 * 8 + 2 * 64)
    out = {"mode": "batch", "workload": "64 RBF problems, n_b ~ U{1000..20000} (seed 0), p=8, gamma=1/8, m=64",
           "gram_tile": "shared memory" if args.batch_p_in_smem else "tensor memory",
           "sum_n": int(sum(sizes)), "entries": entries, "ms_per_product": ms, "kernel_ms": kern_ms,
           "tflops": flops / (kern_ms * 1e-3) / 1e12,
           "roofline": {"bound": "tensor", "achieved": flops / (kern_ms * 1e-3) / 1e12, "peak": peak,
                        "unit": "TFLOP/s", "frac": flops / (kern_ms * 1e-3) / 1e12 / peak,
                        "peak_basis": "measured bf16 dense x 1.1/2.25 (nominal TF32/bf16)"},
           "e2e_s": e2e_s, "clocks": clk, "u_checksum": float(np.abs(U).sum())}
    print(json.dumps(out), flush=True)
    return 0


def grid_workload(problems: int, nmax: int, side: int, seed: int = 0, lmin: float = 1e-5, nl: int = 0):
    """The batched workload: problems with n_b ~ U{1000..nmax} (seed 0), each the
    rbf_small recipe at p = 8 from seed 1000 + b (x ~ U[0,1]^8, RBF gamma = 1/8),
    and side taus in [0.05, 0.95] x (nl or side) lambdas log-spaced in [lmin, 1e-1]."""
    from paper_2510_07929_gb300 import workloads as W

    rng = np.random.default_rng(seed)
    sizes = rng.integers(1000, nmax + 1, size=problems)
    wls = [W.rbf_small(n=int(n), p=8, seed=1000 + b) for b, n in enumerate(sizes)]
    taus, lams = np.meshgrid(np.linspace(0.05, 0.95, side), np.logspace(np.log10(lmin), -1, nl or side),
                             indexing="ij")
    return wls, taus.ravel(), lams.ravel()


def run_grid(args):
    """Grid solves on the batched workload: every problem's (tau, lambda) pairs
    through kqr_solve_grid_batch (the pairs of a problem share their Gram
    products), against the same pairs solved one at a time through kqr_solve on
    the same handles (all of them when --grid-seq-sample covers the grid, else a
    random sample of pairs, whose mean time is scaled to the grid and labelled a
    projection).  CG products: FP64-class where the kernel is numerically
    low-rank at FP32 resolution (options.cg_high = 2), as on this smooth kernel."""
    import torch

    from paper_2510_07929_gb300 import build

    build.build()
    from paper_2510_07929_gb300 import kqr

    wls, taus, lams = grid_workload(args.grid_problems, args.grid_nmax, args.grid_side, lmin=args.grid_lmin,
                                    nl=args.grid_nl)
    tol = args.tol
    t0 = time.perf_counter()
    probs = [kqr.Problem(wl.X, wl.y, wl.kind, wl.gamma, cg_high=2, time_limit_s=args.time_limit) for wl in wls]
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    out = kqr.solve_grid_batch(probs, taus, lams, tol=tol, workers=args.grid_workers)
    t_grid = time.perf_counter() - t0
    statuses = np.concatenate([o[3] for o in out])
    worst = float(max(np.max(o[2]) for o in out))
    pairs = len(wls) * taus.size
    rng = np.random.default_rng(1)
    sample = [(int(b), int(c)) for b, c in zip(rng.integers(0, len(wls), size=pairs),
                                                rng.integers(0, taus.size, size=pairs))]
    full = args.grid_seq_sample >= pairs
    if full:
        sample = [(b, c) for b in range(len(wls)) for c in range(taus.size)]
    else:
        sample = sample[:args.grid_seq_sample]
    seq, seq_status = [], []
    for b, c in sample:
        t1 = time.perf_counter()
        _, _, kkt, info = probs[b].solve(float(taus[c]), float(lams[c]), tol, allow_not_converged=True)
        seq.append(time.perf_counter() - t1)
        seq_status.append(int(info["status"]))
    grid_sample_status = [int(out[b][3][c]) for b, c in sample]
    t_seq = sum(seq) if full else float(np.mean(seq)) * pairs
    for p in probs:
        p.close()
    res = {"mode": "grid",
           "workload": f"{len(wls)} RBF problems, n_b ~ U{{1000..{args.grid_nmax}}} (seed 0), p=8, gamma=1/8, "
                       f"{args.grid_side} taus in [0.05, 0.95] x {args.grid_nl or args.grid_side} lambdas log-spaced in "
                       f"[{args.grid_lmin:g}, 1e-1], tol {tol:g}",
           "sum_n": int(sum(w.n for w in wls)), "pairs": pairs, "create_s": t_create, "grid_s": t_grid,
           "grid_status_counts": {str(k): int(v) for k, v in zip(*np.unique(statuses, return_counts=True))},
           "grid_worst_kkt": worst,
           "sequential": {"kind": "measured" if full else "projection", "pairs_timed": len(seq),
                          "seconds": t_seq, "mean_s_per_pair": float(np.mean(seq)),
                          "status_counts": {str(k): int(v) for k, v in zip(*np.unique(seq_status, return_counts=True))},
                          "grid_status_counts_same_pairs": {str(k): int(v) for k, v in
                                                            zip(*np.unique(grid_sample_status, return_counts=True))}},
           "time_limit_s_per_pair": args.time_limit,
           "speedup": t_seq / t_grid}
    print(json.dumps(res), flush=True)
    return 0


def main():
    args = parse()
    if args.mode == "grid":
        return run_grid(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "grad":
        return run_grad(args)
    if args.mode == "path":
        return run_path(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "gram":
        return run_gram(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
