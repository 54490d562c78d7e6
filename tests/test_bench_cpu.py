"""bench.py on the CPU: the reference arm's JSON line, and the GPU arm's helpers.

The reference arm times the FP64 oracle on the host (the one other place the
benchmark runs the oracle); its line must keep the benchmark contract.  The
GPU arm cannot run here; its pure helpers are checked, and every function the
GPU arm calls must exist.
"""
import ast
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1", "--ref-step-seconds", "0.3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["cores"] <= (os.cpu_count() or 1)
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]


def test_gpu_arm_calls_only_defined_functions():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    defined = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    called = {n.func.id for n in ast.walk(tree)
              if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    import builtins as b
    builtins = set(dir(b))
    local = set()
    for n in ast.walk(tree):   # names bound by assignment or arguments (closures, lambdas)
        if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store):
            local.add(n.id)
        if isinstance(n, ast.arg):
            local.add(n.arg)
    missing = called - defined - builtins - local
    assert not missing, missing


def test_throughput_and_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2, 10, 30, 1, 1000.0) == 2 * 10 * 30 / 1.0
    N, n = 65536, 13107
    assert bench.algorithmic_bytes("col_pass", N, n, 4) == 16 * N + 12 * n + N / 8
    assert bench.algorithmic_bytes("fft_rows", N, n, 4) == 16 * N
    assert bench.algorithmic_bytes("sure", N, n, 4) == 8 * N
    assert bench.algorithmic_bytes("idwt", N, n, 4) == sum(16 * N / 4 ** j for j in range(4)) / 4
    assert len(bench.source_hash()) == 16


def test_iteration_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    # F_alg per slice-iteration: about 24 MFLOP at 256x256 db4 s=4, 38.6 at 320x320 s=5
    assert abs(bench.iteration_flops(256, 256, 4, 8) / 1e6 - 24.2) < 0.2
    assert abs(bench.iteration_flops(320, 320, 5, 8) / 1e6 - 38.6) < 0.2
    N, n = 65536, 13107
    r = bench.iteration_roofline(10e-6, 256, 256, n, 4, 8, 6800.0, 80.0)
    b, f = 16 * N + 12 * n + N / 8, bench.iteration_flops(256, 256, 4, 8)
    assert r["bytes_per_slice_iter"] == b
    assert abs(r["hbm_frac"] - b / 6.8e12 / 10e-6) < 1e-12
    assert abs(r["alu_frac"] - f / 80e12 / 10e-6) < 1e-12
    assert r["bound"] == ("alu" if f / 80e12 > b / 6.8e12 else "hbm")
    assert r["frac"] == max(r["hbm_frac"], r["alu_frac"])
    assert bench.bound_of(100.0, 1.0, 6800.0, 80.0) == "hbm"
    assert bench.bound_of(1.0, 1e6, 6800.0, 80.0) == "alu"
