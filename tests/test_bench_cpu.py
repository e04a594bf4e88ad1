"""bench.py's reference arm (the FP64 oracle on the host cores) on CPU: the JSON line carries the
contract's keys, and a rank other than 0 exits without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_json_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "2D symbols/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] >= 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_recorded_counters_follow_the_kernel_source_hash(tmp_path, monkeypatch):
    """roofline.traffic and roofline.ncu come from the committed capture only while the kernel
    sources still hash to the value recorded with it."""
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "traffic.txt"
    body = ("source_hash: {h}\ndram_bytes_per_full_launch: 123\nfma_pipe_pct: 50.5\n"
            "issue_active_pct: 60.0\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    f.write_text(body.format(h=bench.kernel_source_hash()))
    assert bench.recorded_traffic() == 123.0
    assert bench.recorded_ncu_counters() == {"fma_pipe_pct": 50.5, "issue_active_pct": 60.0}
    f.write_text(body.format(h="0" * 16))
    assert bench.recorded_traffic() is None and bench.recorded_ncu_counters() is None
