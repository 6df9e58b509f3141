"""The device side of slice sharding on one GPU: the radial-range views of
shard_problem, projected one after another (no collective, no waiting
between them), sum to the whole problem's Gamma' -- FP64 to 1e-12 of the
unsharded call and 1e-10 of the oracle, the tensor-core form within its
1e-8; and project_separable_sharded without a process group is the plain
call."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("world", [2, 3, 30])
def test_shards_sum_to_whole(mg, world):
    P = syn.make_problem(60, 6, 25, seed=12)
    dp = mg.DeviceProblem.from_host(P)
    whole = mg.project_separable(dp).cpu().numpy()
    ref = oracle.separable(P)
    for prec, tol in ((mg.PREC_FP64, 1e-10), (mg.PREC_OZAKI_BF16, 1e-8)):
        acc = torch.zeros(P.n_late, P.n_prim, dtype=torch.float64, device="cuda")
        for r in range(world):
            sub = mg.shard_problem(dp, r, world)
            if sub.n_x:
                acc += mg.project_separable(sub, precision=prec)
        mg.handle_status()
        assert normwise(acc, ref) < tol
        if prec == mg.PREC_FP64:
            assert normwise(acc, whole) < 1e-12
    g = mg.project_separable_sharded(dp, 0, 1)
    assert normwise(g, whole) == 0.0
