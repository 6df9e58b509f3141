"""GPU parity of the batched form (row a10): many uneven problems in one call,
captured once into a CUDA graph and replayed, against the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (2, 1e-8)])
def test_batched_uneven_models(mg, precision, tol):
    """A scaled-down mix of the 64-model workload (uneven l_max, basis size,
    x count); every result matches the oracle, and a second call replays the
    cached graph with new data in the same buffers."""
    probs = syn.batched_models(n=6, scale=0.04)
    h = mg.Handle()
    dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
    gs = mg.project_separable_batched(dps, precision=precision, handle=h)
    if precision == 2:
        mg.handle_status(handle=h)
    refs = [oracle.separable(P) for P in probs]
    for g, ref in zip(gs, refs):
        assert normwise(g, ref) < tol
    # same buffers, new values: the replayed graph reads the new data
    for dp in dps:
        dp.qt.mul_(-0.5)
    gs2 = mg.project_separable_batched(dps, precision=precision, outs=gs, handle=h)
    if precision == 2:
        mg.handle_status(handle=h)
    for g, ref in zip(gs2, refs):      # Gamma' is cubic in q~: factor (-1/2)^3
        assert normwise(g, -0.125 * ref) < tol
    h.close()
