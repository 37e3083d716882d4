"""The reference arm of bench.py (the CPU oracle, no GPU): one JSON line with the
same metric, unit and config as the native arm, a cpu_baseline describing the run,
and an e2e entry with no host-device traffic; ranks other than 0 print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--scale", "12", "--batch", "4096", "--ref-batch", "1024",
        "--steps", "3", "--warmup", "3"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + ARGS, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_line_matches_native_config():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench

    class A:
        scale, batch = 12, 4096
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    # the config names the batch the oracle actually ran (1024), not the native arm's
    want = bench.plain_config(A, 1 << 12, d["config"]["m"], 1, batch=1024)
    cfg = dict(d["config"])
    assert cfg.pop("native_arm_batch") == 4096
    cfg.pop("stream")
    want.pop("stream")
    assert cfg == want and cfg["batch"] == 1024 and "B1e3" in cfg["workload"]
    assert d["config"]["m"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] > 0 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_ranks_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
