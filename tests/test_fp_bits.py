"""The integer-bit FP64 <-> double-FP32 conversions of the tensor-core form
(csrc/fp_bits.h) against their plain FP64 counterparts, bit for bit, compiled
as host C++ with g++.  CPU only."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent


def test_conversions_match_fp64_route(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "fp_bits_check"
    # no fast-math: the reference side relies on IEEE rounding of casts
    subprocess.run([gxx, "-std=c++17", "-O2", str(HERE / "fp_bits_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), "3000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "split_mismatch 0 scale_mismatch 0" in r.stdout
