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


@pytest.mark.parametrize("streams", [0, 1, 3, 8])
def test_batched_streams(mg, streams):
    """The batch spread over concurrent streams (MODAL_OPT_BATCH_STREAMS; 0 =
    chosen by timing on the first call): each result equals the single-problem
    entry point on the same inputs -- to the rounding of the FP64 sums of the
    exact chunk products, since a single-problem call overlaps its operand
    passes with the previous chunk's GEMM and may group the K chunks
    differently from the graph's one-stream form -- and the replayed graph
    reads new data."""
    probs = syn.batched_models(n=7, scale=0.03, base_seed=2000)
    h = mg.Handle()
    mg.set_option(mg.OPT_BATCH_STREAMS, streams, handle=h)
    dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
    gs = mg.project_separable_batched(dps, precision=2, handle=h)
    mg.handle_status(handle=h)
    singles = [mg.project_separable(dp, precision=2, handle=h).cpu().numpy() for dp in dps]
    mg.handle_status(handle=h)
    for g, ref in zip(gs, singles):
        assert normwise(g, ref) < 1e-11
    for dp in dps:
        dp.qt.mul_(2.0)
    gs2 = mg.project_separable_batched(dps, precision=2, outs=gs, handle=h)
    mg.handle_status(handle=h)
    for g, ref in zip(gs2, singles):   # cubic in q~: factor 8
        assert normwise(g, 8.0 * ref) < 1e-11
    h.close()


def test_batched_bounded_wait_status_from_every_stream(mg):
    """A wait bound of one clock makes the tensor-core kernels give up on every
    stream of a batched call; the status word of each stream reaches
    modal_handle_status, and the next call with the default bound is right."""
    probs = syn.batched_models(n=4, scale=0.03, base_seed=3000)
    h = mg.Handle()
    mg.set_option(mg.OPT_BATCH_STREAMS, 4, handle=h)
    dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
    mg.set_wait_limit(1, handle=h)
    mg.project_separable_batched(dps, precision=2, handle=h)
    with pytest.raises(mg.ModalError) as ei:
        mg.handle_status(handle=h)
    assert ei.value.code == 4        # MODAL_ETIMEOUT
    mg.set_wait_limit(0, handle=h)
    gs = mg.project_separable_batched(dps, precision=2, handle=h)
    mg.handle_status(handle=h)
    for g, P in zip(gs, probs):
        assert normwise(g, oracle.separable(P)) < 1e-8
    h.close()


def test_batched_larger_bases_against_oracle(mg):
    """Bases of 12 to 20 functions (up to 1540 modes a side) in one batched
    call, in the plain FP64 form and the tensor-core form: every result
    against the oracle at that form's bound."""
    probs = [syn.make_problem(40, 12, 4, seed=61, nb_prim=12),
             syn.make_problem(52, 16, 3, seed=62, nb_prim=14),
             syn.make_problem(36, 20, 3, seed=63, nb_prim=20)]
    refs = [oracle.separable(P) for P in probs]
    for precision, tol in ((0, 1e-10), (2, 1e-8)):
        h = mg.Handle()
        dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
        gs = mg.project_separable_batched(dps, precision=precision, handle=h)
        if precision == 2:
            mg.handle_status(handle=h)
        for g, ref in zip(gs, refs):
            assert normwise(g, ref) < tol
        h.close()
