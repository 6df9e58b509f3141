"""torch.autograd.Function over the separable projection and its adjoint.

Forward: Gamma'(q~, q) by modal_project_separable.  Backward: dL/dq~ and
dL/dq by modal_project_backward (M slices recomputed, not stored).  For the
fit loss L = ||Gamma' alpha - b||^2 the alpha gradient 2 Gamma'^T (Gamma'
alpha - b) is plain torch on the device.
"""
from __future__ import annotations

import torch

from . import _lib
from .api import DeviceProblem, project_backward, project_separable


class ModalProjection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, qt: torch.Tensor, q: torch.Tensor, dp: DeviceProblem, precision: int,
                n_mu: int):
        qt_c, q_c = qt.detach().contiguous(), q.detach().contiguous()
        gamma = project_separable(dp, precision=precision, n_mu=n_mu, qt=qt_c, q=q_c)
        ctx.save_for_backward(qt_c, q_c)
        ctx.dp, ctx.precision, ctx.n_mu = dp, precision, n_mu
        return gamma

    @staticmethod
    def backward(ctx, grad_gamma):
        qt_c, q_c = ctx.saved_tensors
        want_dq = ctx.needs_input_grad[1]
        dqt, dq = project_backward(ctx.dp, grad_gamma, precision=ctx.precision, n_mu=ctx.n_mu,
                                   want_dq=want_dq, qt=qt_c, q=q_c)
        return dqt, dq, None, None, None


def fit_loss_and_grads(dp: DeviceProblem, alpha: torch.Tensor, b: torch.Tensor,
                       precision: int = _lib.PREC_FP64, n_mu: int = 0):
    """L = ||Gamma' alpha - b||^2 with dL/dq~ (adjoint kernels) and dL/dalpha."""
    qt = dp.qt.detach().clone().requires_grad_(True)
    alpha = alpha.detach().clone().to(torch.float64).requires_grad_(True)
    gamma = ModalProjection.apply(qt, dp.q, dp, precision, n_mu)
    r = gamma @ alpha - b
    loss = (r * r).sum()
    loss.backward()
    return loss.detach(), qt.grad, alpha.grad
