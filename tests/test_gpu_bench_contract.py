"""bench.py's JSON line on a GPU: one line with every field of the contract, consistent.

Runs a short bench (four timed steps, no serving leg, no CPU baseline) as a subprocess
and checks the keys, the units and the relations between them.
"""
import json
import subprocess
import sys
from pathlib import Path

import pytest

from gpu_util import need_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = Path(__file__).resolve().parent.parent


def test_bench_line_has_the_contract_fields():
    need_gpu()
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--steps", "4", "--warmup", "3", "--no-serving",
                        "--no-cpu-baseline", "--host-depth", "2"], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["metric"] == "HE-MatMul plaintext MACs/s" and d["unit"] == "MAC/s" and d["higher_is_better"]
    assert d["n_gpus"] == 1 and d["steps"] == 4 and d["warmup"] == 3 and d["scaling"] == "weak"
    assert d["value"] > 0 and d["vs_baseline"] is None and d["data"] == "synthetic"
    macs = d["config"]["plain_macs_per_step"]
    assert abs(d["value"] - macs / (d["ms_per_step"] / 1e3)) / d["value"] < 1e-6
    rf = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rf, key
    assert rf["bound"] in ("alu", "hbm", "tensor") and 0 < rf["frac"] < 1.5
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-3
    e = d["e2e"]
    assert e["unit"] == "MAC/s" and e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= d["steps"]
    assert d["clocks"] is None or {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    bt = d["batched_requests"]  # mixed requests: one launch and one call per request agree bit for bit
    assert bt["outputs_identical"] and bt["requests"] == 64 and 16 <= bt["m_min"] <= bt["m_max"] <= 512
    assert bt["one_launch"]["ms"] > 0 and bt["per_request"]["ms"] > 0
