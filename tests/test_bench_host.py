"""bench.py's host logic (no GPU): workload defaults, the published rates
vs_baseline divides by, the gate on measured DRAM traffic, the clock
sampler's timestamp parsing, and the reference arm (the CPU oracle)."""
import argparse
import os
import sys

import pytest

import bench
from tests.paper_values import GOLDEN


def parse(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_workload_defaults():
    a = parse()
    assert (a.workload, a.histories, a.batches, a.steps, a.warmup) == ("ct256_imrt7", 1e8, 100, 10, 3)
    a = parse("--workload", "paper_slab_6MV_lung")
    assert (a.histories, a.batches) == (2.5e8, 10)
    a = parse("--workload", "water64_e15", "--histories", "2e5")
    assert (a.histories, a.batches) == (2e5, 10)
    assert set(bench.DEFAULT_SIZE) <= set(bench.WORKLOADS) and set(bench.PAPER_RATE) <= set(bench.WORKLOADS)


def test_published_rates_come_from_the_paper():
    """vs_baseline divides by histories / T_GPU as the paper prints them
    (fixture tests/golden/paper_gpu_times.txt: Table 2 and Sec. 4)."""
    rows = {}
    for line in open(os.path.join(GOLDEN, "paper_gpu_times.txt")):
        if line.strip() and not line.startswith("#"):
            name, n, t = line.split()
            rows[name] = (float(n), float(t))
    assert set(rows) == set(bench.PAPER_RATE)
    for name, (n, t) in rows.items():
        assert bench.PAPER_RATE[name] == pytest.approx(n / t, rel=1e-12)
        assert bench.DEFAULT_SIZE[name][0] == n            # the paper's history count


def test_traffic_is_scaled_per_history_and_gated_on_the_sources(monkeypatch):
    """The ncu bytes per history of a capture, times the step's histories,
    over the step's launches of that kernel; None for another workload, tally
    mode or kernel, or once the kernel sources no longer hash to the
    capture's value."""
    cap = {"tally": "fp64", "sha1": bench.sources_sha1(),
           "bytes_per_history": {"electron phase": 120.0, "photon phase": 180.0}}
    monkeypatch.setitem(bench.TRAFFIC, "ct256_imrt7", cap)
    ns = argparse.Namespace(workload="ct256_imrt7", histories=1e8, batches=100, tally="fp64")
    assert bench.measured_traffic(ns, "electron phase", 8.0) == pytest.approx(120.0 * 1e8 / 8.0)
    assert bench.measured_traffic(argparse.Namespace(**{**vars(ns), "histories": 1e7}),
                                  "photon phase", 2.0) == pytest.approx(180.0 * 1e7 / 2.0)
    for change in (dict(tally="fp32pair"), dict(workload="slab128_e20MeV")):
        assert bench.measured_traffic(argparse.Namespace(**{**vars(ns), **change}), "electron phase", 8.0) is None
    assert bench.measured_traffic(ns, "batch fold", 1.0) is None
    monkeypatch.setitem(bench.TRAFFIC, "ct256_imrt7", dict(cap, sha1="0" * 40))
    assert bench.measured_traffic(ns, "electron phase", 8.0) is None


def test_nominal_and_detailed_op_counts():
    """frac takes the nominal per-unit work of the method's steps (30 per
    Woodcock flight, 60 per Klein-Nishina interaction, 100 per electron
    step); the detailed counts only add work (random numbers, crossings)."""
    assert bench.NOMINAL_OPS == {"ph_flights": 30, "compton": 60, "el_steps": 100}
    for k, v in bench.NOMINAL_OPS.items():
        assert bench.OPS[k] >= v


def test_clock_sampler_reads_nvidia_smi_timestamps():
    import datetime
    t = bench.Clocks._stamp("2026/12/03 12:34:56.789")
    assert t == pytest.approx(datetime.datetime(2026, 12, 3, 12, 34, 56, 789000).timestamp())
    assert bench.Clocks._stamp("not a time") is None


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` times the CPU oracle (no GPU, no torch on
    its path) and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "water32_1MeV_pencil", "--steps", "1", "--warmup", "3",
                          "--cpu-seconds", "1"], cwd=here, capture_output=True, text=True,
                         timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "histories/s" and d["unit"] == "histories/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == "water32_1MeV_pencil"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "histories/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; the others exit 0
    without output or work."""
    import subprocess
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], cwd=here, capture_output=True,
                         text=True, timeout=120, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
