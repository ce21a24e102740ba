"""bench.py's reference arm on the CPU (the oracle timed on host cores): the
JSON line's contract keys, and the multi-rank launch where only rank 0
works and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env, *args):
    env = dict(os.environ, **extra_env)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    lines = run_bench({}, "--workload", "tiny_closed", "--steps", "2", "--warmup", "1", "--oracle-spectra", "6")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tiny_closed: 500 proteins")


def test_reference_arm_other_ranks_are_silent():
    assert run_bench({"RANK": "1", "WORLD_SIZE": "2"}, "--workload", "tiny_closed", "--steps", "1") == []


def test_reference_arm_with_a_json_workload(tmp_path):
    from paper_2102_02286_gb300 import configs
    w = configs.TINY_CLOSED.with_proteins(60)
    w = configs.workload_from_json(configs.workload_to_json(w).replace('"tiny_closed"', '"my_workload"'))
    cfg = tmp_path / "w.json"
    cfg.write_text(configs.workload_to_json(w))
    lines = run_bench({}, "--config", str(cfg), "--steps", "1", "--warmup", "0", "--oracle-spectra", "3")
    d = json.loads(lines[0])
    assert d["config"]["workload"].startswith("my_workload")
