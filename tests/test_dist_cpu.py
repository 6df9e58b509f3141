"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
every rank projects its own problem (weak scaling), the step time is the
maximum over ranks, and the whole-job value counts every rank's slices.
No GPU and no collective on the data path."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    ws, r, local = bench.dist_setup(backend_gpu=False)
    assert (ws, r, local) == (world, rank, rank)
    # rank-dependent "step time": the job's time is the slowest rank's
    t = 10.0 + 5.0 * rank
    tmax = bench.max_over_ranks(t, ws)
    bench.barrier(ws)
    import synthetic as syn
    P = syn.make_problem(10, 2, 3, seed=1 + rank)      # the seed bench.py gives rank r
    value = ws * P.slices / (tmax * 1e-3)
    out.put((rank, tmax, float(P.phi[0]), value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, phi0, v0), (r1, t1, phi1, v1) = res
    assert t0 == t1 == 15.0                    # max over ranks
    assert phi0 != phi1                        # independent problems per rank
    assert v0 == v1                            # same whole-job value on every rank
