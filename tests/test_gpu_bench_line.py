"""The benchmark's GPU arm prints one JSON line with every key the
measurement contract names (a short run of the headline configuration)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_headline_json_line():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                          "--cpu-seconds", "0.5"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks", "fp32_mixed", "errors_vs_oracle"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    r = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r, key
    assert 0.0 < r["frac"] < 1.5
    assert r["executed"] is None or r["executed"]["frac"] > 0
    assert r["peak_source"].startswith("measured")
    pk = d["alu_peaks_measured"]
    assert pk["dfma"]["tflops"] > 0.5 and max(pk["ffma"]["tflops"], pk["ffma2"]["tflops"]) > 30
    assert d["fp32_mixed"]["roofline"]["frac"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["single_core"]["cores"] == 1
    assert d["gpu_launches"] > 0 and "workload" in d["config"]
    assert d["errors_vs_oracle"]["fp64"]["single"] <= 1e-12 and d["errors_vs_oracle"]["fp32"]["single"] <= 1e-5
    # the clock record covers both precision arms
    wins = d["clocks"]["windows"]
    assert any(k.startswith("fp64") for k in wins) and any(k.startswith("fp32") for k in wins)
    eq = d["speedup_at_equal_accuracy"]
    assert eq["speedup"] > 1 and len(eq["by_distance"]) == 3
