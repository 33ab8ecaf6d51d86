"""The benchmark's one-line JSON contract on a small block: the keys the
round-end reader takes, their units, and their consistency (launch count, the
roofline's own arithmetic, end-to-end below the device rate)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "block_h8_32", "--steps", "20",
           "--warmup", "3", "--no-cpu-baseline", "--no-planning", "--no-precision"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 20 and d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "block_h8_32" and d["config"]["elements"] == 32 ** 3
    # value = element-steps per second of the timed region
    assert abs(d["value"] - 32 ** 3 / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert abs(rf["achieved"] - rf["algorithmic_bytes_per_step"] / (rf["kernel_ms_per_step"] * 1e-3) / 1e9) \
        <= 1e-6 * rf["achieved"]
    assert rf["traffic"] is None  # no committed capture of this workload
    e = d["e2e"]
    assert e["unit"] == d["unit"] and 0 < e["value"] < d["value"] * 1.05
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    # streamed: a tile and a shared-node kernel per step and a clock bump per graph (20 = 16 + 4);
    # the (grid-)resident modes: one step kernel and a clock bump per graph
    mode = d["plan"]["kernels"].split(" ")[0]
    assert mode in ("streamed", "resident", "grid-resident")
    assert d["gpu_launches"] == (20 * 2 + 2 if mode == "streamed" else 2 * 2)
    assert d["clocks"]["sm_mhz"] > 0 and isinstance(d["clocks"]["reasons"], list)
