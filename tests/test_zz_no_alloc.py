"""The allocation-free entry point modal_project_separable_noalloc.

Some callers cannot allocate device memory: a host program that hands all of
the GPU's memory to its own allocator or budget, a plugin whose sandbox
forbids cudaMalloc, or a latency-critical loop where a cudaMalloc (which may
synchronise the device) is not acceptable.  This entry point takes the
caller's input and output buffers like modal_project_separable and keeps its
scratch in a fixed-size buffer compiled into the library, so it allocates
nothing.  The tests call it through the C ABI twice in a row and check each
result against modal_project_separable (same kernels, same FP64 bound) and
against the FP64 oracle; that the device's free memory does not change
across a call; the FP32 form; and that oversized problems are refused.

This file is named to be collected last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 2e-5


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
    ref_oracle = oracle.separable(P)
    for _ in range(2):                       # the shared scratch keeps the last contents
        g = _noalloc(mg, dp).cpu().numpy()
        assert np.abs(g - ref).max() / scale < TOL_FP64
        assert np.abs(g - ref_oracle).max() / np.abs(ref_oracle).max() < TOL_FP64
    # a second, different problem right after: nothing stale leaks through
    P2 = syn.make_problem(37, 7, 13, seed=8, nb_prim=3)
    dp2 = mg.DeviceProblem.from_host(P2)
    ref2 = mg.project_separable(dp2).cpu().numpy()
    for _ in range(2):
        g2 = _noalloc(mg, dp2).cpu().numpy()
        assert np.abs(g2 - ref2).max() / np.abs(ref2).max() < TOL_FP64


def test_noalloc_leaves_free_memory_unchanged(mg):
    """After a first call (which looks up the static array's address), a
    second call into a preallocated output changes the device's free memory
    by nothing: it allocates no device memory."""
    P = syn.make_problem(60, 8, 6, seed=17)
    dp = mg.DeviceProblem.from_host(P)
    out = torch.empty(dp.n_late, dp.n_prim, dtype=torch.float64, device=dp.device)
    _noalloc(mg, dp, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _noalloc(mg, dp, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = oracle.separable(P)
    assert np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max() < TOL_FP64


def test_noalloc_fp32_twice(mg):
    P = syn.make_problem(48, 6, 10, seed=21, nb_prim=4)
    dp = mg.DeviceProblem.from_host(P)
    ref = mg.project_separable(dp, precision=mg.PREC_FP32).cpu().numpy()
    ref_oracle = oracle.separable(P)
    for _ in range(2):
        g = _noalloc(mg, dp, precision=mg.PREC_FP32).cpu().numpy()
        assert np.abs(g - ref).max() / np.abs(ref).max() < TOL_FP32
        assert np.abs(g - ref_oracle).max() / np.abs(ref_oracle).max() < TOL_FP32


def test_noalloc_rejects_oversized_problem(mg):
    from paper_1503_08809_gb300._lib import ModalError
    P = syn.make_problem(400, 20, 2, seed=1)       # needs more scratch than the static buffer
    dp = mg.DeviceProblem.from_host(P)
    with pytest.raises(ModalError) as ei:
        _noalloc(mg, dp)
    assert ei.value.code == 1 and "scratch" in str(ei.value)
