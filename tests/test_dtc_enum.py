"""Host logic: the enumeration of the direct form on the tensor cores
(csrc/dtc_enum.h) -- l1 runs of the (l2, l3) pairs, the batches cut from the
device cursor, the GEMM items -- compiled with g++ and checked against a
brute-force list of the sorted triples on sparse, dense and small grids in
both weight modes (tests/dtc_enum_check.cpp).  CPU only."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent


def test_dtc_enumeration(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "dtc_enum_check"
    subprocess.run([gxx, "-std=c++17", "-O2", str(HERE / "dtc_enum_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip().endswith("0 violations")
