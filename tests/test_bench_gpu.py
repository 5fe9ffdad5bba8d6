"""The benchmark's own JSON line on the GPU (the 64x64 workload, a short run):
every key the line must carry, measured values that are consistent with each
other, and the GPU result checked against the oracle inside the run."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--config", "1",
                          "--steps", "3", "--warmup", "3", "--reps", "4", "--cpu-budget", "0.5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.strip()][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks", "modelled_comm"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] >= 3 and d["value"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["gpu_vs_oracle_relerr"] <= 1e-13
    assert d["e2e"]["h2d_bytes_per_step"] == 8 * 4096 and d["e2e"]["value"] > 0
    # 4 chained applies per step, at least one SpMV launch each
    assert d["gpu_launches"] >= 3 * 4
