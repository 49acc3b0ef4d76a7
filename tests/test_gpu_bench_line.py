"""The benchmark line's contract on a short run: one JSON line with the
headline metric, the roofline of the dominant kernel, the end-to-end figure
through the C ABI, the clocks, the launch count and the legs of the other
workloads (ensemble, Eq. 13 detection, capillary-wave slab, serving)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_short_bench_line_has_every_key():
    cmd = [sys.executable, "bench.py", "--steps", "6", "--warmup", "3", "--no-cpu-baseline",
           "--no-tune", "--list-lanes", "8", "--ens-steps", "2", "--seg-steps", "2",
           "--e2e-steps", "2", "--wavy-steps", "2", "--serve-requests", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks", "latency_ms"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 6 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["gpu_launches"] > 0
    roof = d["roofline"]
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert 0 < roof["frac"] < 1 and abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    cfg = d["config"]
    assert cfg["fp64_gpu_path"]["value"] > 0
    assert cfg["mixed_vs_fp64_forces"]["max_err_over_bar"] <= 1.0
    assert cfg["ensemble_vs_fp64"]["speedup"] > 1
    assert cfg["segmentation_eq13"]["eq13"]["detect_ms_per_detection"] > 0
    assert cfg["wavy_slab"]["value"] > 0 and cfg["wavy_slab"]["n"] == 2097152
    assert cfg["serving"]["done"] == 2 and cfg["serving"]["atom_steps_per_s"] > 0
