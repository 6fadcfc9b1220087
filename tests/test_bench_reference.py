"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
keeps the result-line contract on a CPU-only machine: one JSON line with the
metric, value, unit, the oracle as cpu_baseline and a zero-copy e2e entry,
also appended to a JSON-lines run log."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line(tmp_path):
    log = tmp_path / "runs.jsonl"
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--jsonl", str(log)], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    wall_s = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "grid3d_256"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the step time is the measured time of the sample each step evaluates, so
    # the timed steps fit inside the run; the full-size time is only extrapolated
    assert 0 < d["sampled_cells"] <= d["config"]["cells"]
    assert d["ms_per_step"] * (d["steps"] + d["warmup"]) / 1e3 < wall_s
    assert d["value"] == pytest.approx(d["sampled_cells"] * d["config"]["modes"] / (d["ms_per_step"] * 1e-3) / 1e9,
                                       rel=1e-9)
    assert d["extrapolated_ms_full_size"] == pytest.approx(d["ms_per_step"] * d["config"]["cells"] /
                                                           d["sampled_cells"], rel=1e-9)
    logged = [json.loads(x) for x in log.read_text().splitlines()]
    assert len(logged) == 1 and logged[0]["value"] == d["value"] and "logged_utc" in logged[0]
