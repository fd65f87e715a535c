"""The benchmark's reference arm (the CPU oracle) prints the JSON contract line (CPU).

`bench.py --impl reference` times the oracle on a bounded sample of the workload and prints one
JSON line with the same metric, unit and config as the GPU arm, plus `impl`, `cpu_baseline` and an
`e2e` object without host copies; under a multi-process launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    return r.returncode, r.stdout


def test_reference_line_carries_the_contract():
    rc, out = run(["--impl", "reference", "--workload", "c1", "--steps", "2", "--warmup", "1"])
    assert rc == 0
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert isinstance(d["metric"], str) and d["metric"]
    assert d["unit"] == "entries/s" and d["value"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    cfg = d["config"]
    assert cfg["workload"].startswith("c1") and cfg["entries_per_step"] == 4 * 64 * 64
    assert "fit in L2" in cfg["l2"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and isinstance(cb["sample"], str)
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_only_on_rank_0():
    rc, out = run(["--impl", "reference", "--workload", "c1", "--steps", "1", "--warmup", "0"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert rc == 0
    assert not [l for l in out.splitlines() if l.startswith("{")]
