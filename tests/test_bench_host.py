"""bench.py host logic on the CPU.

* The reference arm: the oracle, as it stands, timed on one host core on a
  bounded sample of the benchmark workload.  Its JSON line carries the same
  metric, unit, direction and workload as the GPU arm, a cpu_baseline
  describing the run and an e2e entry with no host-device bytes; under a
  multi-rank launch only rank 0 runs and prints.
* The clock record: sampled nvidia-smi lines summarised into the line's
  `clocks` entry (median SM clock, maximum, throttle reasons seen)."""
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


def test_clock_summary_parses_throttle_reasons(tmp_path):
    """The sampled nvidia-smi lines become the line's `clocks` entry: median
    SM clock under load, the maximum clock, and every throttle reason seen
    active at any sample."""
    b = _bench_module()
    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1500, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = b.ClockSampler(0)
    s.proc, s.path = object(), str(csv)
    out = s.summary()
    assert out["samples"] == 4 and out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2025.0                       # median of 2070, 1980, 2070, 1500
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not os.path.exists(csv)                       # the sample file is removed
    empty = b.ClockSampler(0)
    assert empty.summary()["reasons"] == ["unsampled"]   # nvidia-smi could not start


def test_cpu_baseline_pool_reports_all_cores_and_one_core():
    """The batched workloads' CPU baseline: independent oracle runs on every
    host core (spawned workers, so the module runs as `bench`), reported as
    the whole pool's rate and as the one-core rate of the same runs (their
    moves over the sum of their own run times)."""
    code = ("import json, bench; print(json.dumps(bench.cpu_baseline_pool("
            "[('batch', i, i, 3) for i in range(4)], 'four small runs')))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    cb = json.loads(r.stdout.strip().splitlines()[-1])
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["instances_per_s"] > 0
    one = cb["one_core"]
    assert one["unit"] == cb["unit"] and one["value"] > 0 and one["instances_per_s"] > 0
    assert "four small runs (4 runs" in cb["sample"]


def test_full_workload_extrapolation():
    """The oracle's full-workload time is the runs times the iteration scale
    over the sample's runs per second."""
    b = _bench_module()
    cb = {"instances_per_s": 8.0}
    out = b.extrapolate_full(cb, 4096, 5.0, "note")
    assert out is cb and cb["full_workload_s_extrapolated"] == 4096 * 5.0 / 8.0
    assert cb["extrapolation"] == "note"
