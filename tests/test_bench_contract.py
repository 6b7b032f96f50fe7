"""The bench's JSON line, checked on the CPU through its reference arm (the
oracle's timed sample): one line, the contract's keys, and a config equal to the
one the GPU arm reports for the same workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "rbf_small", "--n", "600", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload, n, tol, rank0 = "rbf_small", 600, 1e-6, 1024

    assert d["config"] == bench.bench_config(bench.workload(A), A, 1)


def test_roofline_helpers():
    """The stored-K roofline counts the packed upper triangle of 128 x 128 FP32 tiles
    plus v and u; the RBF roofline's fractions are achieved / peak on each unit, with
    n(n+1)/2 entries per launch."""
    sys.path.insert(0, ROOT)
    import bench

    n = 50000
    t = (n + 127) // 128
    r = bench.stored_k_roofline(n, launches=4, ms=4.0)
    assert r["bound"] == "hbm" and r["bytes_per_launch"] == t * (t + 1) // 2 * 65536 + 8 * n
    assert abs(r["achieved"] - r["bytes_per_launch"] / 1e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    entries = n * (n + 1) / 2
    for f16 in (True, False):
        q = bench.rbf_tc_roofline(n, 20, launches=2, ms=1.0, sm_count=152, sm_mhz=2000.0, f16=f16)
        assert q["bound"] == "alu"
        assert abs(q["achieved"] - entries / 0.5e-3 / 1e12) < 1e-9
        assert abs(q["peak"] - 152 * bench.XU_LANES_PER_SM * 2000e6 / 1e12) < 1e-9
        assert abs(q["fma_convention"]["achieved"] - 3 * entries / 0.5e-3 / 1e12) < 1e-9
        tc = q["tensor_convention"]
        assert abs(tc["achieved"] - 6 * 20 * entries / 0.5e-3 / 1e12) < 1e-9
        assert abs(tc["frac"] - tc["achieved"] / tc["peak"]) < 1e-12
    assert (bench.rbf_tc_roofline(n, 20, 2, 1.0, 152, 2000.0, True)["tensor_convention"]["peak"] >
            bench.rbf_tc_roofline(n, 20, 2, 1.0, 152, 2000.0, False)["tensor_convention"]["peak"])
