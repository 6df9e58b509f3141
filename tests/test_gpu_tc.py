"""GPU parity of the tensor-core (tcgen05) form of the separable path: the
l contraction and the triple product with exponent-aligned BF16 slices,
against the FP64 oracle.  Tolerance for the mixed form: 1e-8 normwise (the
accuracy required of it), 1e-10 for the l contraction alone (M error)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_M = 1e-10
TOL_MIXED = 1e-8


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


@pytest.mark.parametrize("shape", [(48, 5, 5, 24), (37, 7, 3, 13), (300, 9, 6, 3)])
def test_tc_contract_l(mg, shape):
    """M[x][j][a][p] from the tcgen05 l contraction (Eq. legendre) vs the oracle."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=5, nb_prim=nbp)
    mu, _ = oracle.gl_nodes(P.n_mu)
    dp = mg.DeviceProblem.from_host(P)
    A = mg.legendre_table(torch.tensor(mu, device="cuda"), P.l_min, P.l_max, dp.w_l)
    M = mg.contract_l(dp, P.n_mu, A, precision=mg.PREC_OZAKI_BF16)
    mg.handle_status()
    ref = oracle.M_table(P, mu)
    assert normwise(M, ref) < TOL_M


def test_tc_separable_cpu_size(mg):
    P = syn.cpu_size()
    g = mg.project_separable(mg.DeviceProblem.from_host(P), precision=mg.PREC_OZAKI_BF16)
    mg.handle_status()
    assert normwise(g, oracle.separable(P)) < TOL_MIXED


@pytest.mark.parametrize("shape,x_chunk", [((37, 7, 3, 13), 0), ((37, 7, 3, 13), 5),
                                           ((60, 12, 11, 7), 0), ((130, 4, 4, 9), 2)])
def test_tc_separable_ragged(mg, shape, x_chunk):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=11, nb_prim=nbp)
    g = mg.project_separable(mg.DeviceProblem.from_host(P), precision=mg.PREC_OZAKI_BF16,
                             x_chunk=x_chunk)
    mg.handle_status()
    assert normwise(g, oracle.separable(P)) < TOL_MIXED


def test_tc_bounded_wait_gives_up_cleanly(mg):
    """A wait bound of one SM clock makes the tensor-core kernels give up on
    purpose: the call reports MODAL_ETIMEOUT through the status word, the
    context stays usable and the next call with the default bound is right."""
    P = syn.make_problem(20, 3, 4, seed=2)
    dp = mg.DeviceProblem.from_host(P)
    h = mg.Handle()
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


def test_tc_planck_sampled(mg):
    """Planck-scale problem on the tensor cores, 100 sampled entries vs the
    oracle (stated bound 1e-8), plus the full matrix vs the FP64 GPU path."""
    P = syn.planck_size()
    dp = mg.DeviceProblem.from_host(P)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16)
    mg.handle_status()
    g = g.cpu().numpy()
    late_pick = np.array([i for i, m in enumerate(P.late_modes) if set(m) <= {0, 7, 19}])
    prim_pick = np.array([i for i, m in enumerate(P.prim_modes) if set(m) <= {2, 11, 16}])
    ref = oracle.separable(P, late=P.late_modes[late_pick], prim=P.prim_modes[prim_pick])
    assert np.abs(g[np.ix_(late_pick, prim_pick)] - ref).max() / np.abs(ref).max() < TOL_MIXED
    g64 = mg.project_separable(dp).cpu().numpy()
    assert normwise(g, g64) < TOL_MIXED


@pytest.mark.parametrize("shape,split_k", [((48, 5, 5, 24), 0), ((60, 12, 11, 7), 0),
                                           ((130, 4, 4, 9), 3), ((300, 10, 10, 6), 0)])
def test_tc_fused_variant(mg, shape, split_k):
    """Y formed in shared memory inside the GEMM (MODAL_OPT_TC_TRIPLE_FUSED),
    with automatic or forced K splits (combined by FP64 atomic adds)."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=13, nb_prim=nbp)
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_TRIPLE_FUSED, 1, handle=h)
    mg.set_option(mg.OPT_TC_SPLIT_K, split_k, handle=h)
    g = mg.project_separable(mg.DeviceProblem.from_host(P, handle=h), precision=mg.PREC_OZAKI_BF16,
                             handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()


@pytest.mark.parametrize("shape", [(48, 5, 5, 24), (60, 12, 11, 7), (130, 4, 4, 9), (300, 10, 10, 6),
                                   (37, 21, 21, 3)])
def test_tc_fused2_variant(mg, shape):
    """Y formed by sixteen warps in the GEMM's shared-memory stages from a
    TMA-staged M~ tile (MODAL_OPT_TC_TRIPLE_FUSED = 2), against the oracle."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=19, nb_prim=nbp)
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_TRIPLE_FUSED, 2, handle=h)
    g = mg.project_separable(mg.DeviceProblem.from_host(P, handle=h), precision=mg.PREC_OZAKI_BF16,
                             handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()
