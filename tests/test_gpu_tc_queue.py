"""GPU parity of the triple-product GEMM as a persistent kernel over a
device work queue (MODAL_OPT_TC_QUEUE = 1): work items (G tile, range of
exact K chunks) taken by atomic fetch-add in order of decreasing cost; on
small problems the tiles are split into K ranges summed with FP64 atomics.
Against the FP64 oracle (tensor-core bound 1e-8 normwise), the one-CTA-per-
tile form, the bounded waits and the batched call."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8
# Two tensor-core forms (one CTA per tile with or without K splits, the
# queue with split tiles, the Y pass beside the GEMM) add the same exact chunk
# products in different groupings, so they agree to the rounding of the
# double-FP32 running sums and FP64 partial sums (~1e-14 of the G entries,
# amplified by the cancellation in the gather), not bit for bit.
TOL_FORMS = 1e-11


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def queue_handle(mg, on=1):
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_QUEUE, on, handle=h)
    return h


@pytest.mark.parametrize("shape,x_chunk", [((48, 5, 5, 24), 0), ((37, 7, 3, 13), 5), ((20, 1, 5, 3), 0),
                                           ((60, 12, 11, 7), 0), ((300, 10, 10, 6), 0), ((37, 21, 21, 3), 0),
                                           ((400, 6, 6, 12), 0)])
def test_queue_separable(mg, shape, x_chunk):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=33, nb_prim=nbp)
    h = queue_handle(mg)
    g = mg.project_separable(mg.DeviceProblem.from_host(P, handle=h), precision=mg.PREC_OZAKI_BF16,
                             x_chunk=x_chunk, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()


def test_queue_matches_one_cta_per_tile(mg):
    """Split tiles (K ranges summed by atomics) and whole tiles give the same
    Gamma' as the one-CTA-per-tile GEMM to the rounding of the FP64 sums."""
    P = syn.make_problem(700, 8, 9, seed=35)      # few tiles, many K chunks: split
    h0, h1 = queue_handle(mg, 0), queue_handle(mg, 1)
    dp = mg.DeviceProblem.from_host(P, handle=h0)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h0).cpu().numpy()
    g1 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h1)
    mg.handle_status(handle=h0)
    mg.handle_status(handle=h1)
    assert normwise(g1, g0) < TOL_FORMS
    assert normwise(g1, oracle.separable(P)) < TOL_MIXED
    h0.close()
    h1.close()


def test_queue_bounded_wait_gives_up_cleanly(mg):
    P = syn.make_problem(40, 6, 4, seed=37)
    h = queue_handle(mg)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    mg.set_wait_limit(1, handle=h)
    mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    with pytest.raises(mg.ModalError) as ei:
        mg.handle_status(handle=h)
    assert ei.value.code == 4        # MODAL_ETIMEOUT
    mg.set_wait_limit(0, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()


def test_queue_batched(mg):
    probs = [syn.make_problem(40, 12, 4, seed=71, nb_prim=12), syn.make_problem(90, 5, 6, seed=72),
             syn.make_problem(30, 16, 3, seed=73, nb_prim=9), syn.make_problem(150, 3, 5, seed=74)]
    h = queue_handle(mg)
    mg.set_option(mg.OPT_TC_AUTOTUNE, 0, handle=h)    # keep the queue form for every problem
    dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
    gs = mg.project_separable_batched(dps, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    for P, g in zip(probs, gs):
        assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()


def test_queue_planck_sampled(mg):
    P = syn.planck_size()
    h = queue_handle(mg)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    g = g.cpu().numpy()
    late_pick = np.array([i for i, m in enumerate(P.late_modes) if set(m) <= {3, 10, 17}])
    prim_pick = np.array([i for i, m in enumerate(P.prim_modes) if set(m) <= {1, 8, 19}])
    ref = oracle.separable(P, late=P.late_modes[late_pick], prim=P.prim_modes[prim_pick])
    assert np.abs(g[np.ix_(late_pick, prim_pick)] - ref).max() / np.abs(ref).max() < TOL_MIXED
    mg.set_option(mg.OPT_TC_QUEUE, 0, handle=h)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    assert normwise(g, g0) < TOL_FORMS
    h.close()


def test_batched_tile_autotuner(mg):
    """The first batched call times the triple GEMM's tile shapes per bucket
    (MODAL_OPT_TC_AUTOTUNE, on by default) and keeps the fastest: results
    against the oracle; a replay, and single-problem calls that reuse the
    buckets' choices, give the same Gamma' to the FP64 sums' rounding."""
    probs = [syn.make_problem(40, 12, 4, seed=81, nb_prim=12), syn.make_problem(260, 5, 6, seed=82),
             syn.make_problem(45, 12, 3, seed=83, nb_prim=12)]       # the first and last share a bucket
    h = mg.Handle()
    dps = [mg.DeviceProblem.from_host(P, handle=h) for P in probs]
    gs = [g.clone() for g in mg.project_separable_batched(dps, precision=mg.PREC_OZAKI_BF16, handle=h)]
    mg.handle_status(handle=h)
    for P, g in zip(probs, gs):
        assert normwise(g, oracle.separable(P)) < TOL_MIXED
    gs2 = mg.project_separable_batched(dps, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    for g, g2 in zip(gs, gs2):
        assert normwise(g2, g.cpu().numpy()) < TOL_FORMS
    for dp, g in zip(dps, gs):
        single = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
        mg.handle_status(handle=h)
        assert normwise(single, g.cpu().numpy()) < TOL_FORMS
    h.close()


@pytest.mark.parametrize("shape,x_chunk", [((48, 5, 5, 24), 3), ((40, 4, 4, 70), 5), ((37, 21, 21, 3), 1),
                                           ((300, 10, 10, 6), 0)])
def test_overlap_separable(mg, shape, x_chunk):
    """The Y pass of each radial chunk on a second stream beside the previous
    chunk's queue GEMM (MODAL_OPT_TC_OVERLAP): several l-chunks and chunks,
    alternating scratch sets, against the oracle and the plain form."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=91, nb_prim=nbp)
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_OVERLAP, 24, handle=h)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=x_chunk, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    mg.set_option(mg.OPT_TC_OVERLAP, 0, handle=h)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=x_chunk, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    assert normwise(g, g0) < TOL_FORMS
    h.close()


def test_overlap_planck(mg):
    P = syn.planck_size()
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    mg.set_option(mg.OPT_TC_OVERLAP, 32, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, g0) < TOL_FORMS
    late_pick = np.array([i for i, m in enumerate(P.late_modes) if set(m) <= {2, 9, 16}])
    prim_pick = np.array([i for i, m in enumerate(P.prim_modes) if set(m) <= {4, 13, 18}])
    ref = oracle.separable(P, late=P.late_modes[late_pick], prim=P.prim_modes[prim_pick])
    got = g.cpu().numpy()[np.ix_(late_pick, prim_pick)]
    assert np.abs(got - ref).max() / np.abs(ref).max() < TOL_MIXED
    h.close()


@pytest.mark.parametrize("shape,x_chunk", [((300, 8, 8, 100), 8), ((200, 6, 6, 150), 16), ((120, 5, 5, 7), 0)])
def test_tail_overlap_separable(mg, shape, x_chunk):
    """The operand and Y passes on a second stream beside the previous
    chunk's GEMM (MODAL_OPT_TC_OVERLAP_TAIL, on by default), the next l
    contraction issued before an l-chunk's last GEMM into the other M buffer:
    several l-chunks (64 radial points each) and ragged last chunks, against
    the oracle and against the one-stream form."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=95, nb_prim=nbp)
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=x_chunk, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    mg.set_option(mg.OPT_TC_OVERLAP_TAIL, 0, handle=h)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=x_chunk, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    assert normwise(g, g0) < TOL_FORMS
    h.close()


def test_tail_overlap_graph_capture(mg):
    """A single-problem call with its passes on the handle's second and
    high-priority streams forks from and joins the caller's stream with
    events, so it can be captured into a CUDA graph (after one call has sized
    the scratch); replays match the oracle, also after new tables are copied
    into the same device buffers."""
    P = syn.make_problem(200, 6, 70, seed=97)
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    out = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device="cuda")
    mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, out=out, x_chunk=8, handle=h)
    mg.handle_status(handle=h)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, out=out, x_chunk=8, handle=h)
    out.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert normwise(out, oracle.separable(P)) < TOL_MIXED
    P2 = syn.make_problem(200, 6, 70, seed=98)
    dp.qt.copy_(torch.tensor(P2.qt))
    dp.q.copy_(torch.tensor(P2.q))
    graph.replay()
    torch.cuda.synchronize()
    assert normwise(out, oracle.separable(P2)) < TOL_MIXED
    h.close()


@pytest.mark.parametrize("split_k", [0, 2])
def test_tail_overlap_split_k(mg, split_k):
    """The overlapped form with its GEMM in two halves (the G blocks of each
    expansion) and, on request, K splits whose partial sums are added per
    half: against the oracle and the one-stream form."""
    P = syn.make_problem(400, 7, 40, seed=99)
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_SPLIT_K, split_k, handle=h)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=8, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    mg.set_option(mg.OPT_TC_OVERLAP_TAIL, 0, handle=h)
    g0 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, x_chunk=8, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    assert normwise(g, g0) < TOL_FORMS
    h.close()
