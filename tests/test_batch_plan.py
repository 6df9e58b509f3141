"""Host logic of the batched entry point: problems spread over concurrent
streams by longest-processing-time-first (csrc/batch_plan.h), compiled with
g++ and checked against its rule, Graham's 4/3 - 1/(3S) bound (brute force
on small batches) and the per-stream scratch blocks.  CPU only."""
from __future__ import annotations

import itertools
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

HERE = Path(__file__).resolve().parent


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("batch") / "check"
    subprocess.run([gxx, "-std=c++17", "-O1", str(HERE / "batch_plan_check.cpp"), "-o", str(exe)], check=True)

    def run(cost, nbytes, ns):
        inp = f"{len(cost)} {ns}\n" + "".join(f"{c!r} {b}\n" for c, b in zip(cost, nbytes))
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
        lines = out.split("\n")
        stream_of = [int(v) for v in lines[0].split()]
        return stream_of, [int(v) for v in lines[1].split()]
    return run


def lpt_reference(cost, ns):
    order = sorted(range(len(cost)), key=lambda i: -cost[i])   # stable: ties keep index order
    load, out = [0.0] * ns, [0] * len(cost)
    for i in order:
        k = min(range(ns), key=lambda s: (load[s], s))
        out[i] = k
        load[k] += cost[i]
    return out


def check_offsets(stream_of, off, nbytes, ns):
    assert len(off) == ns + 1 and off[0] == 0
    for k in range(ns):
        size = off[k + 1] - off[k]
        assert size % 256 == 0 and off[k] % 256 == 0
        need = max([nbytes[i] for i in range(len(nbytes)) if stream_of[i] == k], default=0)
        assert size >= max(need, 256)


@pytest.mark.parametrize("seed", range(8))
def test_random_batches(layout, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 70))
    cost = [float(c) for c in rng.lognormal(20, 1.5, n)]
    nbytes = [int(b) for b in rng.integers(1, 1 << 30, n)]
    for ns in (1, 2, 3, 4, 8):
        stream_of, off = layout(cost, nbytes, ns)
        assert stream_of == lpt_reference(cost, ns)
        check_offsets(stream_of, off, nbytes, ns)


def test_graham_bound_small_batches(layout):
    rng = np.random.default_rng(11)
    for _ in range(30):
        n, ns = int(rng.integers(2, 8)), int(rng.integers(2, 4))
        cost = [float(c) for c in rng.integers(1, 100, n)]
        stream_of, _ = layout(cost, [1] * n, ns)
        make = max(sum(c for c, s in zip(cost, stream_of) if s == k) for k in range(ns))
        opt = min(max(sum(c for c, s in zip(cost, assign) if s == k) for k in range(ns))
                  for assign in itertools.product(range(ns), repeat=n))
        assert make <= (4.0 / 3.0 - 1.0 / (3 * ns)) * opt + 1e-9


def test_empty_and_single(layout):
    stream_of, off = layout([], [], 4)
    assert stream_of == [] and off == [0, 256, 512, 768, 1024]
    stream_of, off = layout([5.0], [1000], 2)
    assert stream_of == [0] and off == [0, 1024, 1280]
