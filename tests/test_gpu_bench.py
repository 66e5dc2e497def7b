"""The benchmark's output contract on a small run (the 256^3 m^2 phi^2 workload):
one JSON line with the metric, the roofline object (bound, achieved, peak, unit,
frac, traffic), the end-to-end object, the launch count, the clock summary and the
autotuner's choice; and the same for the z-slab mode. Run as subprocesses, as the
benchmark is run."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _common(d, steps):
    assert d["unit"] == "site-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == steps and d["value"] > 0 and d["ms_per_step"] > 0
    n = d["config"]["n"]
    assert abs(d["value"] - d["n_gpus"] * n ** 3 / (d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]
    ro = d["roofline"]
    assert ro["bound"] == "hbm" and ro["unit"] == "GB/s" and ro["peak"] > 0
    assert abs(ro["frac"] - ro["achieved"] / ro["peak"]) <= 1e-9
    # 32 B per site-update (FP32) over the step time, per GPU
    assert abs(ro["achieved"] - 32 * n ** 3 / d["n_gpus"] / (d["ms_per_step"] / 1e3) / 1e9) <= 1e-6 * ro["achieved"]
    assert "traffic" in ro
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= steps
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]


def test_bench_line_contract():
    d = _run("--workload", "m2phi2_256_fp32", "--steps", "40", "--warmup", "3", "--no-cpu-baseline", "--no-extras",
             "--e2e-steps", "2")
    _common(d, 40)
    assert d["scaling"] == "weak" and d["n_gpus"] == 1
    assert d["config"]["workload"] == "m2phi2_256_fp32"
    assert d["gpu_launches"] == 40          # one fused kernel per step
    t = d["tune"]
    assert t["candidates"] >= 2 and t["best_ms"] <= t["slowest_ms"]
    assert f"variant {t['chosen']['variant']}" in d["roofline"]["kernel"]


def test_bench_slab_line_contract():
    d = _run("--workload", "m2phi2_256_fp32", "--slabs", "2", "--steps", "20", "--warmup", "2", "--e2e-steps", "2")
    _common(d, 20)
    assert d["scaling"] == "strong"
    assert d["slabs"]["count"] == 2 and sum(d["slabs"]["planes"]) == 256
    assert d["config"]["parallelism"].startswith("zslab2")
