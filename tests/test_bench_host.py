"""bench.py's reference arm on the CPU: the oracle, as it stands, timed on
one host core on a bounded sample of the benchmark workload.  Its JSON line
carries the same metric, unit, direction and workload as the GPU arm, a
cpu_baseline describing the run and an e2e entry with no host-device bytes;
under a multi-rank launch only rank 0 runs and prints."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("elsr_bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _run(args, **env):
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, capture_output=True,
                          text=True, timeout=300, env=dict(os.environ, **env))


def test_reference_arm_json_line():
    b = _bench_module()
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "3", "--ref-iters", "4"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == (b.METRIC, b.UNIT, True)
    assert d["config"]["workload"] == b.WORKLOAD["workload"]
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 3, 1)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "first 4 of" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-iters", "2"],
             RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
