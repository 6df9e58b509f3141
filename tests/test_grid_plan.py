"""Host logic of the dense-output GEMM grids and of the tensor-core adjoint's
radial chunk (csrc/grid_plan.h), compiled with g++: the rows-per-CTA rule
covers every row tile once, the wave count matches a simulated dispatch of
the CTAs on the SMs, and the chosen chunk is the cheapest of its range (at
the gradient workload: 25 radial points, 48 waves, against 52 for the 29
that memory allows).  CPU only."""
from __future__ import annotations

import random
import shutil
import subprocess
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
TILE = 128


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("gridp") / "check"
    subprocess.run([gxx, "-std=c++17", "-O1", str(HERE / "grid_plan_check.cpp"), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="".join(l + "\n" for l in lines), capture_output=True, text=True,
                             check=True).stdout
        return [[int(v) for v in l.split()] for l in out.strip().split("\n")]
    return run


def cdiv(a, b):
    return -(-a // b)


def rows_per_cta(rows, cols):
    return max(1, min(4, cdiv(rows, TILE) * cdiv(cols, TILE) // (4 * 152)))


def uniform(rows, cols):
    return cdiv(rows, TILE) % rows_per_cta(rows, cols) == 0


def simulated_makespan(rows, cols, rpc, sms):
    """CTAs in launch order onto the first free SM, each lasting its number
    of row tiles (the last CTA of a column may hold fewer)."""
    nrt, nct = cdiv(rows, TILE), cdiv(cols, TILE)
    durations = [min(rpc, nrt - y * rpc) for y in range(cdiv(nrt, rpc)) for _ in range(nct)]
    free = [0] * sms
    for d in durations:
        k = min(range(sms), key=lambda i: free[i])
        free[k] += d
    return max(free)


def test_rows_per_cta_covers_every_tile(plan):
    rng = random.Random(5)
    cases = [(rng.randint(1, 400_000), rng.randint(1, 1200)) for _ in range(200)] + [(128, 128), (1, 1)]
    got = plan([f"c {r} {c}" for r, c in cases])
    for (rows, cols), (rpc, ctas) in zip(cases, got):
        nrt, nct = cdiv(rows, TILE), cdiv(cols, TILE)
        assert 1 <= rpc <= 4
        # the rule: about four waves of 152 SMs before a CTA takes several row tiles
        assert rpc == max(1, min(4, nrt * nct // (4 * 152)))
        # the kernel's assignment: CTA row y runs row tiles y*rpc .. y*rpc + rpc - 1 (clipped)
        covered = sorted(y * rpc + i for y in range(cdiv(nrt, rpc)) for i in range(min(rpc, nrt - y * rpc)))
        assert covered == list(range(nrt))
        assert ctas == nct * cdiv(nrt, rpc)


def test_waves_match_simulated_dispatch(plan):
    rng = random.Random(7)
    cases = []
    for _ in range(120):
        sms = rng.choice([4, 16, 152])
        cases.append((rng.randint(1, 60_000 if sms > 16 else 6_000), rng.randint(1, 600), sms))
    got = plan([f"w {r} {c} {s}" for r, c, s in cases])
    for (rows, cols, sms), (w,) in zip(cases, got):
        nrt = cdiv(rows, TILE)
        rpc = rows_per_cta(rows, cols)
        sim = simulated_makespan(rows, cols, rpc, sms)
        assert w >= sim                      # never optimistic
        if nrt % rpc == 0:
            assert w == sim                  # exact when every CTA holds rpc row tiles


def test_chunk_is_cheapest_of_its_range(plan):
    rng = random.Random(11)
    cases = [(300, 1501, 256, 29, 152)]
    for _ in range(60):
        cases.append((rng.randint(1, 700), rng.choice([73, 751, 1501, 3001]), rng.choice([25, 256, 400, 1024]),
                      rng.randint(1, 32), rng.choice([8, 148, 152])))
    got = plan([f"k {' '.join(map(str, c))}" for c in cases])
    for (n_x, n_mu, cols, cmax, sms), row in zip(cases, got):
        c, costs = row[0], row[1:]
        assert len(costs) == cmax
        lo = cdiv(cmax, 2)
        assert lo <= c <= cmax
        # the cost of a chunk, recomputed from simulated dispatches where every
        # CTA holds the same number of row tiles: waves of its full and ragged
        # launches (tenths) plus one tenth per launch
        for cc in {c, cmax, lo}:
            full, rest = divmod(n_x, cc)
            sizes = [cc * n_mu] * full + ([rest * n_mu] if rest else [])
            if all(uniform(rows, cols) for rows in sizes):
                exp = sum(10 * simulated_makespan(rows, cols, rows_per_cta(rows, cols), sms) + 1 for rows in sizes)
                assert costs[cc - 1] == exp
        best = min(costs[lo - 1:])
        assert costs[c - 1] == best
        assert all(costs[k - 1] > best for k in range(c + 1, cmax + 1))   # ties go to the larger chunk


def test_gradient_workload_chunk(plan):
    # l_max 1000, 16 functions: 1501 GL nodes, 256 entries (x, y), 29 radial
    # points by memory, 300 in all, 152 SMs
    (row,) = plan(["k 300 1501 256 29 152"])
    c, costs = row[0], row[1:]
    assert c == 25
    assert costs[25 - 1] == 12 * (10 * 4 + 1)          # twelve launches of 3.87 waves -> 4
    assert costs[29 - 1] == 10 * (10 * 5 + 1) + (10 * 2 + 1)   # ten of 4.49 -> 5, one of 1.55 -> 2
