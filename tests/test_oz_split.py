"""The BF16 slicing of the tensor-core form (csrc/oz_split.h) on the CPU:
slices exact in BF16, multiples of 2^(-7 s) within their bounds, and the
representation error within 2^-29 + 2^-37 of |H + L| <= 2^7 -- the facts the
exact level-0/1 sums and the stated error of the tensor-core form rest on."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent


def test_slicing_bounds(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "oz_split_check"
    # no fast-math and no FMA contraction: the split relies on IEEE FP32 adds
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", str(HERE / "oz_split_check.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), "2000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "violations 0" in r.stdout
