"""Host-side checks of bench.py: the JSON line of the reference arm (the oracle on the host
cores) and the rule that a committed ncu traffic figure is reported only for the kernel source it
was measured on.  No GPU is needed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_records_follow_the_kernel_source(tmp_path, monkeypatch):
    import bench
    h = bench.collide_source_hash()
    assert len(h) == 16
    rec = tmp_path / "profiles"
    rec.mkdir()
    body = "# a record\nsource_hash={}\ndram_bytes_per_launch_full_size=123456\n"
    (rec / "k_collide_x_traffic.txt").write_text(body.format(h))
    (rec / "k_collide_y_traffic.txt").write_text(body.format("0" * 16))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "collide_source_hash", lambda: h)
    assert bench.recorded_traffic("x") == 123456.0
    assert bench.recorded_traffic("y") is None        # measured on another source
    assert bench.recorded_traffic("z") is None        # no record


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints one JSON line with
    the contract's keys, its cpu_baseline describing the run and an e2e of the same value."""
    pytest.importorskip("numpy")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
