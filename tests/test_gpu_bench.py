"""bench.py's JSON line on a small workload (R-MAT 20, 64 seeds): every key of the line's
contract is present and consistent: the roofline of the round kernel, the end-to-end
figure through host pointers, the kernel-launch count, the clocks and the random-access
calibration."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--graph", "rmat20", "--seeds", "64", "--steps", "3",
           "--warmup", "3", "--no-plain", "--no-cpu", "--no-autotune", "--serve-seconds", "0", "--no-gd",
           "--no-kinds", "--no-c2", "--no-c3", "--probe-gb", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["unit"] == "seeds/s" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] == pytest.approx(64 * 3 / (d["ms_per_step"] * 3 / 1e3), rel=1e-6)
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0 and rf["achieved"] > 0
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-9)
    assert rf["traffic"] is None  # DRAM bytes are recorded for the full workload only
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == "seeds/s"
    assert e2e["h2d_bytes_per_step"] == 4 * 64 and e2e["d2h_bytes_per_step"] == 8 * 64 * 64
    assert d["gpu_launches"] == 3 * 3  # seed, round kernel and top-k per step
    assert "reasons" in d["clocks"]
    ra = d["random_access"]
    assert ra["load_gaccess_per_s"] > 0 and ra["load_atomic_gaccess_per_s"] > 0
    assert ra["round_kernel_inserts_gaccess_per_s"] > 0
