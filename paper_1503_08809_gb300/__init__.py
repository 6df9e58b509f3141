"""GB300 (sm_103a) implementation of the Modal Gamma' projection of
arXiv 1503.08809 behind the C ABI in ``include/modal.h``.

This module only marshals arguments: torch CUDA tensors for device memory
and streams, ctypes for the calls.  Every step of the projection runs in
``libmodal.so``'s kernels; there is no CPU fallback -- importing the library
fails loudly if it has not been built.
"""
from __future__ import annotations

from ._lib import (OPT_BATCH_STREAMS, OPT_DIRECT_TENSOR, OPT_TC_AUTOTUNE, OPT_TC_OVERLAP, OPT_TC_OVERLAP_TAIL, OPT_TC_PAIR, OPT_TC_QUEUE, OPT_TC_SPLIT_K, OPT_TC_TRIPLE_FUSED, ModalError, PREC_FP32, PREC_FP64,
                   PREC_BF16X3, PREC_OZAKI_BF16, PREC_TF32, W_EXACT_3J, W_SMOOTH_GOSPER, XW_HERMITE, XW_TRAPEZOID, lib,
                   lib_path)
from .api import (DeviceProblem, Handle, contract_l, default_handle, gl_nodes, gram, gram_solve,
                  handle_status, legendre_table, project_backward, project_direct, project_full,
                  project_separable, project_separable_batched, set_option, set_wait_limit, x_weights)
from .autograd import ModalProjection, fit_loss_and_grads
from .shard import project_separable_sharded, shard_problem, x_ranges

__all__ = [
    "ModalError", "PREC_BF16X3", "PREC_FP32", "PREC_FP64", "PREC_OZAKI_BF16", "PREC_TF32", "W_EXACT_3J", "W_SMOOTH_GOSPER",
    "XW_HERMITE", "XW_TRAPEZOID", "lib", "lib_path", "DeviceProblem", "Handle", "contract_l",
    "default_handle", "gl_nodes", "handle_status", "set_option", "set_wait_limit", "legendre_table", "project_backward", "project_direct",
    "project_separable", "project_separable_batched", "x_weights", "ModalProjection", "gram",
    "gram_solve", "project_full",
    "fit_loss_and_grads", "project_separable_sharded", "shard_problem", "x_ranges",
]
