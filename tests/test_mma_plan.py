"""Host logic of the tensor-core form: the schedules of the 15 slice products
(s + t <= 4) as tcgen05 MMA runs (csrc/mma_plan.h), compiled with g++ and
checked against the rules the GEMM kernel relies on.  CPU only."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
SLICES, MAXLEV = 5, 4


@pytest.fixture(scope="module")
def schedules(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("plan") / "dump"
    subprocess.run([gxx, "-std=c++17", "-O1", str(HERE / "mma_plan_dump.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rows = []
    for line in out.split("\n"):
        if line.strip():
            f = line.split()
            rows.append((int(f[0]), int(f[1], 16), [int(x, 16) for x in f[2:]]))
    return rows


def decode(r):
    return r & 15, (r >> 4) & 15, (r >> 8) & 15, (r >> 12) & 15, bool((r >> 16) & 1)


def check(w, header, runs):
    nruns, used = header & 0xFF, (header >> 8) & 0xFF
    assert nruns == len(runs) and 1 <= nruns <= 16
    assert 4 <= used <= 5                               # the drain reads accumulators 0..3 (and 4)
    seen, fresh = set(), set(range(16))
    touched = set()
    for r in runs:
        sa, sb, n, a0, is_fresh = decode(r)
        assert n >= 1 and n * w <= 256                  # MMA N = n w
        assert (a0 + n) * w <= 512 and a0 + n <= used   # TMEM columns
        accs = set(range(a0, a0 + n))
        # a run is all first touches (overwrite) or all accumulations
        assert (accs <= fresh) if is_fresh else not (accs & fresh)
        fresh -= accs
        touched |= accs
        for t in range(n):
            a, lv = a0 + t, sa + sb + t
            assert (sa, sb + t) not in seen
            seen.add((sa, sb + t))
            assert lv <= MAXLEV and sa < SLICES
            assert a == lv if lv < 2 else a >= 2        # levels 0, 1 exact on their own accumulators
    assert seen == {(s, t) for s in range(SLICES) for t in range(SLICES) if s + t <= MAXLEV}
    assert touched == set(range(used))                  # every accumulator the drain reads is written


def test_searched_schedules(schedules):
    widths = [w for w, _, _ in schedules if w > 0]
    assert widths == list(range(16, 129, 16))
    for w, header, runs in schedules:
        if w > 0:
            check(w, header, runs)


def test_merged_runs_beat_singles(schedules):
    """The searched schedules cost no more than one MMA per product under the
    issue model (max(80, N/2) clocks per MMA), and strictly less where runs
    can merge at all (w <= 128)."""
    cost = lambda w, runs: sum(max(80.0, decode(r)[2] * w / 2.0) for r in runs)
    for w, _, runs in schedules:
        if w > 0:
            assert cost(w, runs) < 15 * max(80.0, w / 2.0)


def test_singles_fallback_is_valid(schedules):
    for w, header, runs in schedules:
        if w < 0:
            check(-w, header, runs)
            assert all(decode(r)[2] == 1 for r in runs)


def test_pair_schedule(schedules):
    """The 2-SM schedule: runs of exactly two B slots with N = 2w, where the
    odd CTA's slot j holds B slice j + 1 (slot 4: zeros, i.e. slice 5 out of
    range).  Every product with sa + sb <= 4 is issued exactly once; levels 0
    and 1 stay alone on accumulators 0 and 1; anything else (levels 2 .. 5,
    the zero slot) lands on accumulators 2 and 3; fresh runs touch only
    untouched accumulators and all four are written."""
    (header, runs), = [(h, r) for w, h, r in schedules if w == 0]
    assert header & 0xFF == len(runs) == 9 and (header >> 8) & 0xFF == 4
    wanted = {(s, t) for s in range(SLICES) for t in range(SLICES) if s + t <= MAXLEV}
    seen, fresh = [], set(range(4))
    for r in runs:
        sa, j, n, a0, is_fresh = decode(r)
        assert n == 2 and 0 <= j < SLICES and a0 + 2 <= 4
        accs = {a0, a0 + 1}
        assert (accs <= fresh) if is_fresh else not (accs & fresh)
        fresh -= accs
        for t, sb in enumerate((j, j + 1)):      # even CTA: slice j; odd CTA: slice j + 1
            a, lv = a0 + t, sa + sb
            if sb >= SLICES:                     # the zero slot of the odd CTA
                assert a >= 2
                continue
            seen.append((sa, sb))
            assert a == lv if lv < 2 else a >= 2
    assert not fresh
    assert len(seen) == len(set(seen))
    assert wanted <= set(seen)
    assert all(s + t <= MAXLEV + 1 for s, t in set(seen) - wanted)  # extras: level 5 only
