"""The JSON line bench.py prints: the keys and shapes the benchmark contract fixes.
The reference arm (the CPU oracle) runs on CPU; the own arm needs a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = ["metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline",
          "dtype", "data", "config", "e2e", "cpu_baseline"]


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"], timeout=300)
    for k in COMMON + ["impl"]:
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GLUPS"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # ms_per_step is the measured step of the sampled box; the 512^3 figure is labelled as implied
    assert abs(d["ms_per_step"] - 64 ** 3 / (d["value"] * 1e9) * 1e3) < 1e-6 * d["ms_per_step"]
    assert d["implied_ms_per_step_512"] > d["ms_per_step"]


@pytest.mark.gpu
def test_own_arm_line_small():
    d = _run(["--n", "64", "--steps", "3", "--warmup", "3", "--variants", "0", "--no-cpu"], timeout=600)
    for k in COMMON + ["ms_per_step", "roofline", "gpu_launches", "clocks"]:
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["scaling"] == "weak"
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 2 * d["steps"]
    assert sum(d["runs"]["steps"]) == d["steps"] and d["runs"]["median_GLUPS"] > 0
    assert d["config"]["workload"].startswith("kh64")
    dev = d["developed"]
    assert dev["GLUPS"] > 0 and dev["after_steps"] >= 2000
