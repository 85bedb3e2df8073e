"""bench.py's JSON line on the GPU (the 24-sphere profiling case, one timed step): the keys of the
benchmark contract, a roofline of the dominant kernel, the CPU baseline, the end-to-end leg through
host buffers and the sampled clocks."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_keys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--small", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, check=True, cwd=ROOT, timeout=900)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 3 and line["value"] > 0
    r = line["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and 0.0 < r["frac"] < 1.05
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] > 0
    e = line["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] > 0
    assert "sm_mhz" in line["clocks"] and "reasons" in line["clocks"]
