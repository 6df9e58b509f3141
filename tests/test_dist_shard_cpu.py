"""Slice sharding of one projection (paper_1503_08809_gb300/shard.py) on CPU:
the radial partition, and two gloo ranks that each project their radial
range (with the full grid's radial weights) and sum Gamma' by all-reduce --
against the single-rank result.  The per-rank projection here is the FP64
oracle (the device path is covered by tests/test_gpu_shard.py); what is
under test is the partition and the reduction."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1503_08809_gb300.shard import x_ranges


def test_x_ranges_cover_and_balance():
    for n_x in (0, 1, 2, 7, 24, 500):
        for world in (1, 2, 3, 8):
            rs = x_ranges(n_x, world)
            assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == n_x
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))          # contiguous, in order
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    assert x_ranges(2, 3) == [(0, 1), (1, 2), (2, 2)]                    # an empty range
    with pytest.raises(ValueError):
        x_ranges(5, 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import dataclasses

    import torch
    import torch.distributed as dist

    import oracle
    import synthetic as syn
    from paper_1503_08809_gb300.shard import allreduce_sum_, x_ranges
    dist.init_process_group("gloo")
    P = syn.make_problem(48, 4, 11, seed=3)                 # the same problem on every rank
    xw_full = oracle.x_weights(P.x)
    lo, hi = x_ranges(P.n_x, world)[rank]
    Ps = dataclasses.replace(P, qt=P.qt[lo:hi].copy(), x=P.x[lo:hi].copy(), n_x=hi - lo)
    g = oracle.separable(Ps, xw=xw_full[lo:hi]) if hi > lo else np.zeros((P.n_late, P.n_prim))
    t = torch.tensor(g)
    allreduce_sum_(t)
    out.put((rank, hi - lo, t.numpy().copy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_x_shards_sum_to_full(world):
    import oracle
    import synthetic as syn
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [n for _, n, _ in res] == [6, 5]
    full = oracle.separable(syn.make_problem(48, 4, 11, seed=3))
    for _, _, g in res:                                     # every rank holds the whole Gamma'
        assert np.abs(g - full).max() / np.abs(full).max() < 1e-13
