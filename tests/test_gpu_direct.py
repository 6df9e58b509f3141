"""GPU parity of the direct path (row a8, Eq. 3D) against the FP64 oracle."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from tests._golden import delta_cases

pytestmark = pytest.mark.gpu

TOL = 1e-10


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def test_direct_dense_cpu_size(mg):
    P = syn.cpu_size()
    dp = mg.DeviceProblem.from_host(P)
    g = mg.project_direct(dp)
    assert normwise(g, oracle.direct(P)) < TOL
    # the two forms agree on a dense grid (Section 2.2)
    assert normwise(g, oracle.separable(P)) < TOL
    assert normwise(mg.project_separable(dp), g.cpu().numpy()) < TOL


@pytest.mark.parametrize("mode", [0, 1])
def test_direct_sparse_grid(mg, mode):
    P = syn.make_problem(160, 4, 9, seed=3, nb_prim=3)
    lg, dw = syn.sparse_l_grid(160)
    g = mg.project_direct(mg.DeviceProblem.from_host(P), lg, dw, weight_mode=mode)
    ref = oracle.direct(P, l_grid=lg, l_dw=dw, weight_mode=mode)
    assert normwise(g, ref) < TOL


@pytest.mark.parametrize("case", list(delta_cases()), ids=lambda c: c[0])
def test_direct_golden(mg, case):
    name, P, expected = case
    dp = mg.DeviceProblem.from_host(P, x_w=np.ones(1))
    g = float(mg.project_direct(dp)[0, 0])
    assert g == pytest.approx(expected, rel=1e-13, abs=1e-15 / (70 * math.pi))


def test_direct_edge_cases(mg):
    P = syn.make_problem(10, 2, 3, seed=1)
    dp = mg.DeviceProblem.from_host(P)
    # empty grid -> zeros
    g = mg.project_direct(dp, l_grid=np.zeros(0, dtype=np.int32))
    assert torch.count_nonzero(g) == 0
    # a grid whose triples all break the triangle condition -> zeros
    g = mg.project_direct(dp, l_grid=np.array([2, 9]), l_dw=np.ones(2))
    ref = oracle.direct(P, l_grid=np.array([2, 9]), l_dw=np.ones(2))
    assert np.allclose(g.cpu().numpy(), ref, rtol=1e-12, atol=0)
    # single point grid (only (l,l,l))
    g = mg.project_direct(dp, l_grid=np.array([4]), l_dw=np.array([2.5]))
    ref = oracle.direct(P, l_grid=np.array([4]), l_dw=np.array([2.5]))
    assert normwise(g, ref) < TOL


def test_direct_planck_sparse_sampled(mg):
    """Planck-scale direct check on the sparse grid (every l to 50, step 2 to
    200, step 5 to 500, step 10 above): full Gamma' on the GPU, sampled
    rows/columns from the oracle."""
    P = syn.planck_size()
    lg, dw = syn.sparse_l_grid(P.l_max)
    g = mg.project_direct(mg.DeviceProblem.from_host(P), lg, dw).cpu().numpy()
    rows = np.array([0, 5, 100, 777, 1539])
    cols = np.array([3, 400, 1200])
    ref = oracle.direct(P, l_grid=lg, l_dw=dw, late=P.late_modes[rows], prim=P.prim_modes[cols])
    got = g[np.ix_(rows, cols)]
    assert np.abs(got - ref).max() / np.abs(ref).max() < TOL
    assert np.isfinite(g).all()


def test_direct_graph_capture(mg):
    """modal_project_direct makes no host synchronisation: after one call
    (which sizes the handle's scratch) it is captured into a CUDA graph;
    replays match the oracle, also after new tables are copied into the same
    device buffers."""
    P = syn.make_problem(160, 4, 9, seed=3, nb_prim=3)
    lg, dw = syn.sparse_l_grid(160)
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    lgd = torch.tensor(lg, dtype=torch.int32, device="cuda")
    dwd = torch.tensor(dw, dtype=torch.float64, device="cuda")
    out = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device="cuda")
    mg.project_direct(dp, lgd, dwd, out=out, handle=h)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        mg.project_direct(dp, lgd, dwd, out=out, handle=h)
    out.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert normwise(out, oracle.direct(P, l_grid=lg, l_dw=dw)) < TOL
    P2 = syn.make_problem(160, 4, 9, seed=4, nb_prim=3)
    dp.qt.copy_(torch.tensor(P2.qt))
    dp.q.copy_(torch.tensor(P2.q))
    graph.replay()
    torch.cuda.synchronize()
    assert normwise(out, oracle.direct(P2, l_grid=lg, l_dw=dw)) < TOL
    h.close()


# The tensor-core form of the Gamma' update (MODAL_OPT_DIRECT_TENSOR): five
# 7-bit BF16 slices per operand, products of levels <= 4 and exact level-0/1
# sums per 1024-triple chunk leave a relative error of a few 2^-35 per term
# against sum |Y||X|; the tolerance is the mixed-precision gate of the
# separable path (1e-8 of max|Gamma'|).
TOL_TC = 1e-8


def _tensor_handle(mg, level=1):
    h = mg.Handle()
    mg.set_option(mg.OPT_DIRECT_TENSOR, level, handle=h)
    return h


# level 1: the Gamma' update on the tensor cores; level 2: the radial
# integrals too (pairs (l2, l3) grouped into one GEMM each)
@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("mode", [0, 1])
def test_direct_tensor_update_sparse(mg, mode, level):
    P = syn.make_problem(160, 4, 9, seed=3, nb_prim=3)
    lg, dw = syn.sparse_l_grid(160)
    h = _tensor_handle(mg, level)
    g = mg.project_direct(mg.DeviceProblem.from_host(P, handle=h), lg, dw, weight_mode=mode, handle=h)
    assert mg.handle_status(handle=h) == 0
    ref = oracle.direct(P, l_grid=lg, l_dw=dw, weight_mode=mode)
    err = normwise(g, ref)
    assert err < TOL_TC, err
    h.close()


@pytest.mark.parametrize("level", [1, 2])
def test_direct_tensor_update_dense_and_edges(mg, level):
    """Dense grid (several 1024-triple chunks and a ragged last batch), then
    an empty grid, a single-point grid and a grid whose triples all break
    the triangle condition on the same handle."""
    P = syn.cpu_size()
    h = _tensor_handle(mg, level)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_direct(dp, handle=h)
    assert normwise(g, oracle.direct(P)) < TOL_TC
    g = mg.project_direct(dp, l_grid=np.zeros(0, dtype=np.int32), handle=h)
    assert torch.count_nonzero(g) == 0
    g = mg.project_direct(dp, l_grid=np.array([4]), l_dw=np.array([2.5]), handle=h)
    assert normwise(g, oracle.direct(P, l_grid=np.array([4]), l_dw=np.array([2.5]))) < TOL_TC
    g = mg.project_direct(dp, l_grid=np.array([2, 9]), l_dw=np.ones(2), handle=h)
    ref = oracle.direct(P, l_grid=np.array([2, 9]), l_dw=np.ones(2))
    assert np.abs(g.cpu().numpy() - ref).max() <= TOL_TC * np.abs(ref).max()
    assert mg.handle_status(handle=h) == 0
    h.close()


@pytest.mark.parametrize("nb", [1, 32])
def test_direct_tensor_integrals_basis_sizes(mg, nb):
    """The radial integrals on the tensor cores at the smallest basis and at
    the largest this form takes (32 functions: 5 column tiles of the {u,v}
    rows, 4 triples per tile), against the oracle on few modes."""
    P = syn.make_problem(60, 3 if nb == 32 else 2, 7, seed=11, nb_prim=nb)
    lg, dw = syn.sparse_l_grid(60)
    h = _tensor_handle(mg, 2)
    g = mg.project_direct(mg.DeviceProblem.from_host(P, handle=h), lg, dw, handle=h).cpu().numpy()
    assert mg.handle_status(handle=h) == 0
    cols = np.unique(np.linspace(0, P.n_prim - 1, 40).astype(int))
    ref = oracle.direct(P, l_grid=lg, l_dw=dw, prim=P.prim_modes[cols])
    assert np.abs(g[:, cols] - ref).max() < TOL_TC * np.abs(ref).max()
    h.close()


@pytest.mark.parametrize("level", [1, 2])
def test_direct_tensor_update_planck_sparse_sampled(mg, level):
    """Planck-scale sparse grid (many batches, the last one ragged): sampled
    entries against the oracle and the whole matrix against the FP64 GPU
    path."""
    P = syn.planck_size()
    lg, dw = syn.sparse_l_grid(P.l_max)
    h = _tensor_handle(mg, level)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_direct(dp, lg, dw, handle=h).cpu().numpy()
    assert mg.handle_status(handle=h) == 0
    g64 = mg.project_direct(dp, lg, dw).cpu().numpy()
    assert np.isfinite(g).all()
    assert normwise(g, g64) < TOL_TC
    rows = np.array([0, 5, 100, 777, 1539])
    cols = np.array([3, 400, 1200])
    ref = oracle.direct(P, l_grid=lg, l_dw=dw, late=P.late_modes[rows], prim=P.prim_modes[cols])
    got = g[np.ix_(rows, cols)]
    assert np.abs(got - ref).max() / np.abs(g64).max() < TOL_TC
    h.close()


def test_direct_tensor_integrals_many_radial_points(mg):
    """More radial points than one exact chunk of the slicing (1100 > 1024):
    the q~ rows and the U rows are split in two K chunks each."""
    P = syn.make_problem(50, 3, 1100, seed=21, nb_prim=4)
    lg, dw = syn.sparse_l_grid(50)
    h = _tensor_handle(mg, 2)
    g = mg.project_direct(mg.DeviceProblem.from_host(P, handle=h), lg, dw, handle=h)
    assert mg.handle_status(handle=h) == 0
    assert normwise(g, oracle.direct(P, l_grid=lg, l_dw=dw)) < TOL_TC
    h.close()
