"""Slice sharding of one projection over several GPUs (one process per GPU).

Gamma' of Eq. 2D is a sum over (x, mu) slices, so the radial points can be
split into contiguous ranges, one per rank: every rank projects its range
with the radial weights of the FULL grid (the trapezium and Hermite weights
of a point depend on its neighbours, so they are computed once on the whole
grid and then sliced), and one sum all-reduce of the FP64 Gamma' (n_late x
n_prim) gives every rank the full matrix -- the paper's scheme of a
decomposition agreed at the start and a reduction of Gamma at the end
(Section 4), with the radial points as the decomposed index.

The partition and the reduction are plain host logic (no CUDA here); the
projection of a rank's range is ``api.project_separable`` on a view of the
device tables (no copy).
"""
from __future__ import annotations

from typing import List, Tuple


def x_ranges(n_x: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous radial ranges [lo, hi) of ``n_x`` points over ``world``
    ranks, sizes differing by at most one (the first n_x % world ranks take
    one more); a rank may get an empty range when world > n_x."""
    if n_x < 0 or world < 1:
        raise ValueError("n_x >= 0 and world >= 1 required")
    base, extra = divmod(n_x, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def allreduce_sum_(t, group=None):
    """In-place sum over the ranks of the default (or given) process group;
    a no-op without an initialised group of more than one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def shard_problem(dp, rank: int, world: int):
    """The DeviceProblem of rank ``rank``'s radial range: views of q~ and of
    the full grid's radial weights (same storage, no copy)."""
    from .api import DeviceProblem
    lo, hi = x_ranges(dp.n_x, world)[rank]
    sub = DeviceProblem.__new__(DeviceProblem)
    sub.__dict__.update(dp.__dict__)
    sub.qt = dp.qt[lo:hi]
    sub.x_w = dp.x_w[lo:hi]
    return sub


def project_separable_sharded(dp, rank: int, world: int, precision: int = 0, out=None, handle=None,
                              group=None, **kw):
    """Gamma' of the whole problem on every rank: this rank's radial range
    through ``project_separable``, then a sum all-reduce (NCCL between GPUs).
    A rank with an empty range contributes zeros."""
    import torch
    from .api import project_separable
    sub = shard_problem(dp, rank, world)
    if sub.n_x > 0:
        g = project_separable(sub, precision=precision, out=out, handle=handle, **kw)
    else:
        g = out if out is not None else torch.empty(dp.n_late, dp.n_prim, dtype=torch.float64,
                                                    device=dp.device)
        g.zero_()
    return allreduce_sum_(g, group)
