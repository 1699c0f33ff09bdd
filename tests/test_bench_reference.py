"""The bench's reference arm (the FP64 CPU oracle timed on the host) prints the
one JSON line of the bench contract: same metric and unit as the GPU arm, the
oracle's rate as `value`, a `cpu_baseline` describing the run and an `e2e` with no
host-device bytes.  Runs on CPU in about ten seconds (one bounded step)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    import bench
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["higher_is_better"] is True and out["value"] > 0
    assert out["steps"] == 1 and out["warmup"] == 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["sample"]
    # the oracle runs on every host core, one worker process each, and says which CPU
    assert cb["cores"] == cb["nproc"] == (os.cpu_count() or 1) and cb["cpu_model"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["n_det"] == 1024 and out["config"]["n_samp"] == 1 << 20


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle and prints; the others exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
