"""bench.py's GPU arm on the headline workload prints one JSON line with the
contract's keys: a whole-job value consistent with its step time, the
convolution's roofline against the ALU peak, the end-to-end figure with the
host bytes it moved, the launches of the library's kernels and the SM clocks
sampled in the timed region."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_headline_line_keeps_the_contract():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3", "--no-cpu-baseline"],
                       cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["n_gpus"] == 1 and d["steps"] == 3
    assert d["warmup"] >= 3 and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert abs(d["value"] - bench.EVALS_PER_STEP / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    assert "workload" in d["config"]
    rf = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rf, key
    assert rf["bound"] == "alu" and rf["unit"] == "TFLOP/s" and 0.0 < rf["frac"] < 1.2
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) <= 1e-9
    e = d["e2e"]
    assert 0.0 < e["value"] <= d["value"] * 1.05
    assert e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == bench.NX * bench.N ** 3 * 8
    assert d["gpu_launches"] > 0
    c = d["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list)
