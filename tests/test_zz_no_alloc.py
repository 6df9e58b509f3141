"""The allocation-free entry point modal_project_separable_noalloc.

Some callers cannot allocate device memory: a host program that hands all of
the GPU's memory to its own allocator or budget, a plugin whose sandbox
forbids cudaMalloc, or a latency-critical loop where a cudaMalloc (which may
synchronise the device) is not acceptable.  This entry point takes the
caller's input and output buffers like modal_project_separable and keeps its
scratch in a fixed-size buffer compiled into the library, so it allocates
nothing.  The test calls it through the C ABI twice in a row and checks each
result against modal_project_separable (same kernels, same FP64 bound).

This file is named to be collected last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def _noalloc(mg, dp, precision=0, out=None):
    from paper_1503_08809_gb300._lib import Opts, check, lib
    L = lib()
    f = L.modal_project_separable_noalloc
    gamma = out if out is not None else torch.empty(dp.n_late, dp.n_prim, dtype=torch.float64,
                                                    device=dp.device)
    s = dp.struct()
    o = Opts(0, int(precision), 0, 0)
    code = f(ctypes.byref(s), ctypes.byref(o), ctypes.c_void_p(gamma.data_ptr()),
             ctypes.c_void_p(torch.cuda.current_stream(dp.device).cuda_stream))
    check(code, None)
    return gamma


def test_noalloc_matches_separable_twice(mg):
    P = syn.cpu_size()
    dp = mg.DeviceProblem.from_host(P)
    ref = mg.project_separable(dp).cpu().numpy()
    scale = np.abs(ref).max()
    for _ in range(2):                       # the shared scratch keeps the last contents
        g = _noalloc(mg, dp).cpu().numpy()
        assert np.abs(g - ref).max() / scale < TOL_FP64
    # a second, different problem right after: nothing stale leaks through
    P2 = syn.make_problem(37, 7, 13, seed=8, nb_prim=3)
    dp2 = mg.DeviceProblem.from_host(P2)
    ref2 = mg.project_separable(dp2).cpu().numpy()
    for _ in range(2):
        g2 = _noalloc(mg, dp2).cpu().numpy()
        assert np.abs(g2 - ref2).max() / np.abs(ref2).max() < TOL_FP64


def test_noalloc_rejects_oversized_problem(mg):
    from paper_1503_08809_gb300._lib import ModalError
    P = syn.make_problem(400, 20, 2, seed=1)       # needs more scratch than the static buffer
    dp = mg.DeviceProblem.from_host(P)
    with pytest.raises(ModalError) as ei:
        _noalloc(mg, dp)
    assert ei.value.code == 1 and "scratch" in str(ei.value)
