"""The kernels' float-float and bit-construction arithmetic
(csrc/ffmath.cuh), compiled for the host with the same rounding as the
device intrinsics and checked against IEEE arithmetic: box indices from the
float-float quotient against IEEE floor((x - o) / L) on grids up to 2M boxes
wide (§4.4.3), the double -> float-float split, the exact bit-built
conversions, the error-free transformations, and the float-float update of
box-relative offsets by FP32 displacements (incremental grid)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2503_10796_gb300", "csrc")


def test_ffmath_on_the_host(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "ffmath_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "host", "ffmath_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    lines = [ln.split() for ln in out.stdout.splitlines() if not ln.startswith(" ")]
    results = {ln[0]: (int(ln[1]), int(ln[2])) for ln in lines if len(ln) == 3 and ln[1].isdigit()}
    names = ["split_ff", "bit_construction", "error_free_transformations", "ff_add_float"]
    for grid in ("box_coord_narrow", "box_coord_wide", "box_coord_2M"):
        names += [grid, grid + "_random_fallback_over_1pct"]
    for name in names:
        cases, failures = results[name]
        assert cases > 0 and failures == 0, (name, out.stdout)
    assert out.returncode == 0, out.stdout
