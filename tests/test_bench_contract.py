"""bench.py's output contract, checked on the CPU through its reference arm
(the FP64 oracle timed on the host cores): one JSON line with the keys the
benchmark line carries, and, under a multi-rank launch, silence and exit 0
on every rank but 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    env.pop("SCAL3R_TTT_LIBRARY", None)
    return subprocess.run([sys.executable, BENCH, "--impl", "reference", *args], env=env, capture_output=True,
                          text=True, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_complete_line():
    r = _run({}, "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert d["config"]["workload"] == "bf16_vggt64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--gpus", "2", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip() == ""
