"""bench.py's reference arm (the oracle timed on the host) keeps the output
contract: one JSON line with the metric, value, unit, timing keys, the
configuration, a cpu_baseline describing the run and an e2e with no host
transfers; ranks other than 0 exit 0 without output.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, **env):
    e = dict(os.environ, **env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=e, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "cell-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"], RANK="1", WORLD_SIZE="2",
            LOCAL_RANK="1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


class _FakeSmi:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_keeps_the_timed_window_and_its_throttle_reasons():
    """The nvidia-smi samples inside the timed window give the median SM
    clock, the maximum and every throttle reason seen active; malformed lines
    are skipped; with no sample inside the window all samples are used."""
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.proc = _FakeSmi()
    s.lines = [(0.0, "1400, 2070, Not Active, Not Active, Not Active, Not Active"),   # before the window
               (1.0, "2070, 2070, Not Active, Not Active, Not Active, Active"),
               (1.2, "[N/A], 2070, Not Active, Not Active, Not Active, Not Active"),  # malformed
               (1.5, "2055, 2070, Not Active, Not Active, Not Active, Not Active"),
               (2.0, "2070, 2070, Active, Not Active, Not Active, Not Active"),
               (3.0, "1000, 2070, Not Active, Not Active, Active, Not Active")]     # after it
    out = s.stop(window=(0.5, 2.5))
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["samples"] == 3 and out["samples_in_timed_region"] == 4
    s2 = bench.ClockSampler(0)
    s2.proc = _FakeSmi()
    s2.lines = [(0.0, "1980, 2070, Not Active, Not Active, Not Active, Not Active")]
    out2 = s2.stop(window=(5.0, 6.0))
    assert out2["sm_mhz"] == 1980.0 and out2["samples_in_timed_region"] == 0
