"""The benchmark's reference arm (the CPU oracle timed on the host cores)
runs without a GPU and prints one JSON line with the contract's keys; the
benchmark's --launch option is parsed on the host."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "256",
                        "--ref-rows", "8", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "cell-stage/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["cells"] == 256 * 8


def test_launch_option_parsing():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_launch("32x32:160", 2) == ((32, 32, 1), 160, 0)
    assert bench.parse_launch("32x8:256", 2) == ((32, 8, 1), 256, 0)
    assert bench.parse_launch("8x8x8:192", 3) == ((8, 8, 8), 192, 0)
    assert bench.parse_launch("16x15x32:256:march", 3) == ((16, 15, 32), 256, 1)
    for bad, dim in [("32x32", 2), ("32:160", 2), ("8x8x8:192", 2), ("32x32:160:march", 2), ("8x8:1:box", 3)]:
        with pytest.raises(ValueError):
            bench.parse_launch(bad, dim)
