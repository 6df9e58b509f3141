"""The per-entry error scale (modal_opts.error_estimate): the separable
projection with every P_ii' entry and weight in magnitude, against the
oracle's magnitude sum; and the conditioned entrywise check
|Gamma'_gpu - Gamma'_oracle| <= tol * estimate for each path.  Also radial
weights of both signs on the tensor-core path (the sign rides on the B
slices there)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

# (precision, bound on the estimate's entrywise relative error, bound of the
# conditioned check): FP64 sums; FP32 products and short FP32 sums (2^-24
# per term); five exponent-aligned BF16 slices (2^-36 of the row scale)
CASES = [(0, 1e-11, 1e-11), (1, 2e-6, 2e-6), (2, 1e-8, 1e-8)]


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


@pytest.mark.parametrize("shape", [(48, 5, 5, 24), (37, 7, 3, 13), (130, 4, 4, 9)])
@pytest.mark.parametrize("precision,tol_est,tol_cond", CASES)
def test_error_estimate_and_conditioned_check(mg, shape, precision, tol_est, tol_cond):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=11, nb_prim=nbp)
    dp = mg.DeviceProblem.from_host(P)
    est = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dp.device)
    g = mg.project_separable(dp, precision=precision, error_estimate=est)
    mg.handle_status()
    g, e = g.cpu().numpy(), est.cpu().numpy()
    ref = oracle.separable(P)
    ref_abs = oracle.separable(P, magnitudes=True)
    assert np.all(ref_abs > 0)
    assert (np.abs(e - ref_abs) / ref_abs).max() < tol_est
    assert (np.abs(g - ref) / ref_abs).max() < tol_cond


def test_estimate_leaves_the_projection_unchanged(mg):
    """FP64: bit for bit.  Tensor-core form: a call with an error estimate runs
    its passes on one stream (the plain call overlaps the operand passes with
    the previous chunk's GEMM and may group the K chunks differently), so the
    two agree to the rounding of the FP64 sums of the exact chunk products."""
    P = syn.cpu_size()
    dp = mg.DeviceProblem.from_host(P)
    for precision in (0, 2):
        plain = mg.project_separable(dp, precision=precision).cpu().numpy()
        est = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dp.device)
        g = mg.project_separable(dp, precision=precision, error_estimate=est).cpu().numpy()
        mg.handle_status()
        if precision == 0:
            assert np.array_equal(g, plain)
        else:
            assert np.abs(g - plain).max() <= 1e-11 * np.abs(plain).max()


def test_negative_radial_weights(mg):
    """Radial weights of both signs (e.g. an integrator with negative
    weights): each path against the oracle given the same weights."""
    P = syn.cpu_size()
    xw = oracle.x_weights(P.x) * np.where(np.arange(P.n_x) % 3 == 1, -1.0, 1.0)
    dp = mg.DeviceProblem.from_host(P)
    dpn = mg.DeviceProblem(dp.q, dp.qt, dp.w_l, torch.tensor(xw, device=dp.device), dp.late_modes,
                           dp.prim_modes, P.l_min, P.l_max, dp.device)
    ref = oracle.separable(P, xw=xw)
    ref_abs = oracle.separable(P, xw=xw, magnitudes=True)
    for precision, _, tol in CASES:
        est = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dp.device)
        g = mg.project_separable(dpn, precision=precision, error_estimate=est).cpu().numpy()
        mg.handle_status()
        assert (np.abs(g - ref) / ref_abs).max() < tol
        assert (np.abs(est.cpu().numpy() - ref_abs) / ref_abs).max() < max(tol, 1e-11)


def test_estimate_rejected_in_batched_calls(mg):
    import ctypes
    from paper_1503_08809_gb300._lib import ModalError, Opts, Problem, check, lib
    P = syn.make_problem(20, 3, 4, seed=2)
    dp = mg.DeviceProblem.from_host(P)
    g = torch.empty(P.n_late, P.n_prim, dtype=torch.float64, device=dp.device)
    est = torch.empty_like(g)
    h = mg.Handle()
    arr = (Problem * 1)(dp.struct())
    outp = (ctypes.c_void_p * 1)(g.data_ptr())
    o = Opts(0, 0, 0, 0, est.data_ptr())
    with pytest.raises(ModalError) as ei:
        check(lib().modal_project_separable_batched(h.ptr, 1, arr, ctypes.byref(o), outp, None), h.ptr)
    assert ei.value.code == 1
    h.close()
