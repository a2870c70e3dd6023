"""The benchmark's JSON line on the host: the reference arm (the oracle on
the CPU) prints the contract's keys, and its `config` is the one the GPU
arm prints for the same workload and launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line(orc):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "plain_fp64_4096", "--precision", "0", "--steps", "3", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 3 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]

    sys.path.insert(0, ROOT)
    import argparse

    import bench
    _, desc = bench.make_workload("plain_fp64_4096", 0, 0)
    args = argparse.Namespace(settle=line["config"]["settle_iterations"])
    own = bench.arm_config(desc, bench.parallelism_of("plain_fp64_4096", 1), bench.precision_of(0), args)
    ref = line["config"]
    # the same workload; parallelism and precision name what each arm runs
    assert {k: v for k, v in ref.items() if k not in ("parallelism", "precision")} == \
        {k: v for k, v in own.items() if k not in ("parallelism", "precision")}
    assert ref["precision"] == "fp64 (the oracle)" and "host core" in ref["parallelism"]
    cb = line["cpu_baseline"]
    assert cb["nproc"] >= 1 and cb["cpu_model"]


def test_settle_defaults():
    sys.path.insert(0, ROOT)
    import bench
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--workload", "growth_division_65536"]
        assert bench.parse().settle == 65
        sys.argv = ["bench.py"]
        assert bench.parse().settle == 50
    finally:
        sys.argv = argv


def test_clock_summary():
    sys.path.insert(0, ROOT)
    import bench
    lines = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1995, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage", ""]
    out = bench.ClockSampler.summarize(lines)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.summarize(["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
