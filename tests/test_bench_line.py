"""The benchmark's JSON line: the keys and types a reader of bench.py's
output relies on, for the timed CUDA arm (GPU) and the oracle arm (CPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def _common(d, steps):
    assert d["metric"] and d["unit"] == "steps/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    assert d["e2e"]["value"] > 0 and d["e2e"]["unit"] == d["unit"]


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    _common(d, 1)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_cuda_arm_line():
    """The default line: the 512000-ion 256^3 box with FP64 state and the
    integer V-cycle (multigrid); beside it the same box with the all-FP64
    V-cycle and in mixed precision."""
    steps = 8
    d = _run("--steps", str(steps), "--warmup", "3", timeout=1200)
    _common(d, steps)
    assert "impl" not in d and d["dtype"] == "f64+i64+f32x2" and d["config"]["grid"] == 256
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["peak"] > 0 and r["achieved"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] is None or r["traffic"] > 0
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 48 * 512000 and e["d2h_bytes_per_step"] > 48 * 512000
    assert d["gpu_launches"] == 9 * steps          # move, 3 cell-list kernels, pairs, spread, solve, gather, finish
    assert d["clocks"]["sm_mhz"] > 0 and isinstance(d["clocks"]["reasons"], list)
    assert d["force_error"] < 1e-7                 # FP64 at tol 1e-10 (the solver tolerance dominates)
    assert d["ms_per_step"] > 0 and d["p99_us"] >= d["p50_us"] > 0
    fr = d["full_run"]                             # the configuration's 200 steps from the start
    assert fr["steps"] == 200 and fr["steps_per_s"] > 0 and fr["iters_per_step"] >= 4.0
    sr = d["serial"]
    assert sr["iters_per_step"] == d["iters_per_step"] and sr["roofline"]["bound"] == "hbm"
    assert sr["gpu_launches"] == 8 * steps
    f = d["fp64"]
    assert f["dtype"] == "f64+f32x2" and f["iters_per_step"] == d["iters_per_step"]
    assert abs(f["force_error"] - d["force_error"]) < 1e-9
    assert {f["roofline"]["bound"], f["roofline_other"]["bound"]} == {"hbm", "alu"}
    m = d["mixed"]
    assert m["steps_per_s"] > d["value"] and m["force_error"] < 1e-5
    assert m["roofline"]["bound"] == "hbm" and m["gpu_launches"] == 8 * steps
    assert d["cpu_baseline_all_cores"]["cores"] >= 1
