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


def test_double_fp32_running_sum(tmp_path):
    """df_add, the running sums of the GEMM drains, against the exact sum
    (rational arithmetic) of n double-FP32 terms: same-sign terms over eight
    decades and cancelling terms; the error stays within n 2^-46 of the sum
    of magnitudes (a first-order bound of about n u^2 for this pair
    arithmetic, u = 2^-24; measured: 3e-16 .. 2e-14 of that sum), and at least a
    thousand times below plain FP32 summation of the same terms."""
    from fractions import Fraction

    import numpy as np

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "df_sum_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", str(HERE / "df_sum_check.cpp"),
                    "-o", str(exe)], check=True)
    rng = np.random.default_rng(7)
    for case in range(6):
        n = 4000
        mag = 10.0 ** rng.uniform(-4, 4, n)
        sign = np.ones(n) if case % 2 == 0 else rng.choice([-1.0, 1.0], n)
        x = sign * mag
        bh = x.astype(np.float32)
        bl = (x - bh.astype(np.float64)).astype(np.float32)
        inp = f"{n}\n" + "".join(f"{float(h).hex()} {float(l).hex()}\n" for h, l in zip(bh, bl))
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        hi, lo = float.fromhex(out[0]), float.fromhex(out[1])
        exact = sum(Fraction(float(h)) + Fraction(float(l)) for h, l in zip(bh, bl))
        got = Fraction(hi) + Fraction(lo)
        scale = sum(abs(Fraction(float(h)) + Fraction(float(l))) for h, l in zip(bh, bl))
        assert abs(got - exact) <= Fraction(n, 2 ** 46) * scale
        # and the compensation shows: >= 1000x below FP32 (pairwise) summation
        f32 = Fraction(float(np.sum(bh, dtype=np.float32)))
        assert abs(got - exact) * 1000 <= abs(f32 - exact)
