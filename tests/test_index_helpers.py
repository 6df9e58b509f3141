"""Host logic: the pair index and the triple-product table layout of
csrc/common.cuh, with the checked index that MODAL_DEBUG builds use in the
gather and scatter kernels, compiled with g++ and checked exhaustively on
small layouts (tests/index_check.cpp).  CPU only."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent


def test_index_helpers(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    inc = "/usr/local/cuda/include"
    if not Path(inc, "cuda_runtime.h").exists():
        pytest.skip("CUDA headers not available")
    exe = tmp_path / "index_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, str(HERE / "index_check.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip().endswith("0 violations")
