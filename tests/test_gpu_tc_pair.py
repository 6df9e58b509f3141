"""GPU parity of the triple-product GEMM on CTA pairs (2-SM tcgen05 MMA,
MODAL_OPT_TC_PAIR = 1) against the FP64 oracle, on shapes with one and many
row tiles per block (an odd count leaves the second CTA of the last pair
without rows), several column-tile widths and ragged radial chunks; the
Planck-size problem against the single-CTA form and sampled oracle entries;
and the bounded waits giving up on purpose.  Tolerance of the tensor-core
form: 1e-8 normwise."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def pair_handle(mg, on=1):
    h = mg.Handle()
    mg.set_option(mg.OPT_TC_PAIR, on, handle=h)
    return h


@pytest.mark.parametrize("shape,x_chunk", [((48, 5, 5, 24), 0), ((37, 7, 3, 13), 0), ((37, 7, 3, 13), 5),
                                           ((60, 12, 11, 7), 0), ((130, 4, 4, 9), 2), ((20, 1, 5, 3), 0),
                                           ((300, 10, 10, 6), 0), ((37, 21, 21, 3), 0)])
def test_pair_separable(mg, shape, x_chunk):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=23, nb_prim=nbp)
    h = pair_handle(mg)
    g = mg.project_separable(mg.DeviceProblem.from_host(P, handle=h), precision=mg.PREC_OZAKI_BF16,
                             x_chunk=x_chunk, handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_MIXED
    h.close()


def test_pair_matches_single_cta_and_error_scale(mg):
    """Same problem through both GEMM forms (they differ only in the order of
    the FP32 sums of levels >= 2 and the level-5 terms the pair form adds),
    and the |M| error-scale pass through the pair form."""
    P = syn.make_problem(200, 12, 5, seed=29)
    h1, h2 = pair_handle(mg, 0), pair_handle(mg, 1)
    dp = mg.DeviceProblem.from_host(P, handle=h1)
    e1, e2 = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device="cuda"), None
    e2 = torch.empty_like(e1)
    g1 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h1, error_estimate=e1)
    g2 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h2, error_estimate=e2)
    mg.handle_status(handle=h1)
    mg.handle_status(handle=h2)
    ref = oracle.separable(P)
    assert normwise(g2, ref) < TOL_MIXED
    assert normwise(g2, g1.cpu().numpy()) < 1e-9
    ref_abs = oracle.separable(P, magnitudes=True)
    assert normwise(e2, ref_abs) < TOL_MIXED
    h1.close()
    h2.close()


def test_pair_bounded_wait_gives_up_cleanly(mg):
    """A wait bound of one SM clock makes both CTAs of each pair give up: the
    call reports MODAL_ETIMEOUT, the context stays usable and the next call
    with the default bound is right."""
    P = syn.make_problem(40, 6, 4, seed=31)
    h = pair_handle(mg)
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


def test_pair_planck_sampled(mg):
    """Planck size (l_max 2000, 20 functions, 500 x): sampled entries against
    the oracle at 1e-8 and the full matrix against the single-CTA form."""
    P = syn.planck_size()
    h = pair_handle(mg)
    dp = mg.DeviceProblem.from_host(P, handle=h)
    g = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    g = g.cpu().numpy()
    late_pick = np.array([i for i, m in enumerate(P.late_modes) if set(m) <= {1, 9, 18}])
    prim_pick = np.array([i for i, m in enumerate(P.prim_modes) if set(m) <= {0, 12, 19}])
    ref = oracle.separable(P, late=P.late_modes[late_pick], prim=P.prim_modes[prim_pick])
    assert np.abs(g[np.ix_(late_pick, prim_pick)] - ref).max() / np.abs(ref).max() < TOL_MIXED
    mg.set_option(mg.OPT_TC_PAIR, 0, handle=h)
    g1 = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h).cpu().numpy()
    mg.handle_status(handle=h)
    assert normwise(g, g1) < TOL_MIXED
    h.close()
