"""GPU parity of the adjoint (row a9): dL/dq~ and dL/dq against the oracle's
adjoint, central finite differences of the GPU forward, and the fit-loss
gradients through the autograd wrapper."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 1e-4


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


@pytest.mark.parametrize("shape,x_chunk", [((14, 3, 3, 3), 0), ((48, 5, 5, 24), 0),
                                           ((37, 6, 4, 13), 5)])
def test_backward_matches_oracle_fp64(mg, shape, x_chunk):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=7, nb_prim=nbp)
    gbar = syn.random_cotangent(P.n_late, P.n_prim, seed=5)
    dqt_ref, dq_ref = oracle.backward(P, gbar)
    dp = mg.DeviceProblem.from_host(P)
    dqt, dq = mg.project_backward(dp, torch.tensor(gbar, device="cuda"), x_chunk=x_chunk)
    assert normwise(dqt, dqt_ref) < TOL_FP64
    assert normwise(dq, dq_ref) < TOL_FP64


def test_backward_fp32(mg):
    P = syn.cpu_size()
    gbar = syn.random_cotangent(P.n_late, P.n_prim, seed=6)
    dqt_ref, dq_ref = oracle.backward(P, gbar)
    dqt, dq = mg.project_backward(mg.DeviceProblem.from_host(P), torch.tensor(gbar, device="cuda"),
                                  precision=mg.PREC_FP32)
    assert normwise(dqt, dqt_ref) < TOL_FP32
    assert normwise(dq, dq_ref) < TOL_FP32


def test_backward_without_dq_and_edge(mg):
    P = syn.make_problem(12, 2, 3, seed=3)
    gbar = syn.random_cotangent(P.n_late, P.n_prim, seed=1)
    dqt, dq = mg.project_backward(mg.DeviceProblem.from_host(P), torch.tensor(gbar, device="cuda"),
                                  want_dq=False)
    assert dq is None
    assert normwise(dqt, oracle.backward(P, gbar, want_dq=False)[0]) < TOL_FP64
    # zero cotangent -> zero gradient
    z = torch.zeros(P.n_late, P.n_prim, dtype=torch.float64, device="cuda")
    dqt0, dq0 = mg.project_backward(mg.DeviceProblem.from_host(P), z)
    assert torch.count_nonzero(dqt0) == 0 and torch.count_nonzero(dq0) == 0


def test_fit_loss_gradients(mg):
    """L = ||Gamma' alpha - b||^2: dL/dalpha = 2 Gamma'^T r in closed form and
    dL/dq~ = adjoint with dL/dGamma' = 2 r alpha^T (oracle adjoint)."""
    P = syn.make_problem(30, 4, 6, seed=2)
    dp = mg.DeviceProblem.from_host(P)
    alpha, delta = syn.fit_vectors(P.n_prim, seed=1)
    gam = oracle.separable(P)
    b = gam @ (alpha + delta)
    loss, dqt, dalpha = mg.fit_loss_and_grads(dp, torch.tensor(alpha, device="cuda"),
                                              torch.tensor(b, device="cuda"))
    r = gam @ alpha - b
    assert float(loss) == pytest.approx(float(r @ r), rel=1e-9)
    assert normwise(dalpha, 2 * gam.T @ r) < 1e-9
    dqt_ref, _ = oracle.backward(P, 2 * np.outer(r, alpha), want_dq=False)
    assert normwise(dqt, dqt_ref) < 1e-9


def test_grad_config_finite_differences(mg):
    """l_max = 1000, 16 functions (816 modes), 300 x points, FP32 forward with
    FP64 reduction: the adjoint's directional derivative along a random
    direction matches a central difference (h = 1e-6 relative) of the FP64
    forward."""
    P = syn.grad_size()
    dp = mg.DeviceProblem.from_host(P)
    rng = np.random.default_rng(9)
    gbar = torch.tensor(syn.random_cotangent(P.n_late, P.n_prim, seed=4), device="cuda")
    dqt, _ = mg.project_backward(dp, gbar, precision=mg.PREC_FP32, want_dq=False)
    v = torch.tensor(rng.standard_normal(P.qt.shape), device="cuda") * dp.qt.abs().max()
    h = 1e-6
    lp = (gbar * mg.project_separable(dp, qt=(dp.qt + h * v).contiguous())).sum()
    lm = (gbar * mg.project_separable(dp, qt=(dp.qt - h * v).contiguous())).sum()
    fd = float((lp - lm) / (2 * h))
    an = float((dqt * v).sum())
    assert an == pytest.approx(fd, rel=1e-4)


TOL_TC = 1e-8


@pytest.mark.parametrize("shape,x_chunk", [((14, 3, 3, 3), 0), ((48, 5, 5, 24), 0), ((37, 6, 4, 13), 5),
                                           ((60, 12, 11, 7), 2), ((20, 1, 5, 3), 0)])
def test_backward_tensor_form(mg, shape, x_chunk):
    """The adjoint's three contractions on tcgen05 (MODAL_PREC_OZAKI_BF16):
    dL/dM over the 2 x 2 minors of the permanent, then dL/dq~ and dL/dq,
    against the oracle's adjoint at the tensor form's bound, 1e-8 normwise."""
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=17, nb_prim=nbp)
    gbar = syn.random_cotangent(P.n_late, P.n_prim, seed=8)
    dqt_ref, dq_ref = oracle.backward(P, gbar)
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    dqt, dq = mg.project_backward(dp, torch.tensor(gbar, device="cuda"), precision=mg.PREC_OZAKI_BF16,
                                  x_chunk=x_chunk, handle=h)
    mg.handle_status(handle=h)
    assert normwise(dqt, dqt_ref) < TOL_TC
    assert normwise(dq, dq_ref) < TOL_TC
    h.close()


def test_backward_tensor_form_grad_config(mg):
    """The gradient workload (l_max 1000, 16 functions, 300 x) in the tensor
    form: against the FP64 GPU adjoint at 1e-8, and the directional
    derivative against a central difference of the FP64 forward."""
    P = syn.grad_size()
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    gbar = torch.tensor(syn.random_cotangent(P.n_late, P.n_prim, seed=4), device="cuda")
    dqt, dq = mg.project_backward(dp, gbar, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    dqt64, dq64 = mg.project_backward(dp, gbar, handle=h)
    assert normwise(dqt, dqt64.cpu().numpy()) < TOL_TC
    assert normwise(dq, dq64.cpu().numpy()) < TOL_TC
    rng = np.random.default_rng(9)
    v = torch.tensor(rng.standard_normal(P.qt.shape), device="cuda") * dp.qt.abs().max()
    hh = 1e-6
    lp = (gbar * mg.project_separable(dp, qt=(dp.qt + hh * v).contiguous(), handle=h)).sum()
    lm = (gbar * mg.project_separable(dp, qt=(dp.qt - hh * v).contiguous(), handle=h)).sum()
    fd = float((lp - lm) / (2 * hh))
    assert float((dqt * v).sum()) == pytest.approx(fd, rel=1e-4)
    h.close()


def test_backward_tensor_form_bounded_wait(mg):
    P = syn.make_problem(30, 4, 5, seed=19)
    gbar = torch.tensor(syn.random_cotangent(P.n_late, P.n_prim, seed=2), device="cuda")
    h = mg.Handle()
    dp = mg.DeviceProblem.from_host(P, handle=h)
    mg.set_wait_limit(1, handle=h)
    mg.project_backward(dp, gbar, precision=mg.PREC_OZAKI_BF16, handle=h)
    with pytest.raises(mg.ModalError) as ei:
        mg.handle_status(handle=h)
    assert ei.value.code == 4
    mg.set_wait_limit(0, handle=h)
    dqt, dq = mg.project_backward(dp, gbar, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    dqt_ref, dq_ref = oracle.backward(P, gbar.cpu().numpy())
    assert normwise(dqt, dqt_ref) < TOL_TC and normwise(dq, dq_ref) < TOL_TC
    h.close()
