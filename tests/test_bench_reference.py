"""The reference arm of bench.py (the CPU oracle timed on the host's cores, no GPU): it prints
one JSON line with the benchmark's metric, unit and direction, the arm's own cpu_baseline and
e2e objects, and a positive rate; under a multi-process launch only rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip().startswith("{")]


@pytest.mark.slow
def test_reference_arm_json_line():
    lines = _run({"WORLD_SIZE": "1", "RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "unknowns/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("laplace_batched")
    # ms_per_step is the measured sample time; the full-factor figure is named as extrapolated
    ex = d["extrapolation"]
    assert abs(d["ms_per_step"] - ex["sample_ms_per_step"]) <= 1e-9 * d["ms_per_step"]
    assert ex["extrapolated_ms_full_factor"] > d["ms_per_step"] and 0 < ex["flop_share"] < 1
    assert abs(d["value"] * ex["extrapolated_ms_full_factor"] * 1e-3 - d["config"]["N"]) <= 1e-6 * d["config"]["N"]


def test_reference_arm_other_ranks_are_silent():
    assert _run({"WORLD_SIZE": "2", "RANK": "1"}) == []
