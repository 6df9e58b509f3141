"""CPU checks of the C ABI: the library builds/loads, exports every symbol
that include/modal.h declares, and reports errors as status codes (no GPU
compute is issued here)."""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def header_symbols():
    src = (ROOT / "include" / "modal.h").read_text()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*\*?\s*(modal_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libmodal():
    from paper_1503_08809_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(str(path))


def test_header_declares_expected_entry_points():
    syms = header_symbols()
    for need in ["modal_project_separable", "modal_project_direct", "modal_project_backward",
                 "modal_project_separable_batched", "modal_gl_nodes", "modal_x_weights"]:
        assert need in syms


def test_library_exports_every_declared_symbol(libmodal):
    missing = [s for s in header_symbols() if not hasattr(libmodal, s)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1503_08809_gb300 import _lib
    assert sorted(_lib.EXPORTS) == sorted(s for s in header_symbols())


def test_status_codes_without_gpu(libmodal):
    """With no usable device, handle creation fails with a status code and a
    message instead of aborting; null arguments are EINVAL."""
    import torch
    libmodal.modal_handle_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
    libmodal.modal_last_error.restype = ctypes.c_char_p
    libmodal.modal_last_error.argtypes = [ctypes.c_void_p]
    assert libmodal.modal_handle_create(None) == 1          # EINVAL
    assert b"null" in libmodal.modal_last_error(None)
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        code = libmodal.modal_handle_create(ctypes.byref(h))
        assert code in (3,)                                  # ECUDA
        assert libmodal.modal_last_error(None)


def test_workspace_size_is_host_only(libmodal):
    """modal_workspace_size validates and plans on the host."""
    from paper_1503_08809_gb300._lib import Opts, Problem
    libmodal.modal_workspace_size.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Opts),
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    fake = 4096  # never dereferenced by the planner
    p = Problem(2, 2000, 20, 20, 500, 1540, 1540, 0, fake, fake, fake, fake, fake, fake)
    o = Opts(0, 0, 0, 0)
    n = ctypes.c_size_t()
    assert libmodal.modal_workspace_size(ctypes.byref(p), ctypes.byref(o), 0, ctypes.byref(n)) == 0
    # A table (48 MB) + M chunk (<= 2 GiB) + G (52 MB)
    assert 40e6 < n.value < 4e9
    o_bad = Opts(100, 0, 0, 0)          # n_mu below the exact GL order
    assert libmodal.modal_workspace_size(ctypes.byref(p), ctypes.byref(o_bad), 0,
                                         ctypes.byref(n)) == 1
    o_ok = Opts(100, 0, 1, 0)           # allowed when asked for
    assert libmodal.modal_workspace_size(ctypes.byref(p), ctypes.byref(o_ok), 0,
                                         ctypes.byref(n)) == 0
    p_bad = Problem(5, 2, 20, 20, 500, 1540, 1540, 0, fake, fake, fake, fake, fake, fake)
    assert libmodal.modal_workspace_size(ctypes.byref(p_bad), ctypes.byref(o), 0,
                                         ctypes.byref(n)) == 1


def test_workspace_size_validation_and_planning(libmodal):
    """Host-side validation and planning through modal_workspace_size (no
    device needed): each rejected argument gets its status code and a
    message; the tensor-core form needs more scratch than FP64 (slices, Y),
    the adjoint at least as much as the forward call, and an explicit radial
    chunk bounds the scratch."""
    from paper_1503_08809_gb300._lib import Opts, Problem
    libmodal.modal_workspace_size.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Opts),
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    libmodal.modal_last_error.restype = ctypes.c_char_p
    libmodal.modal_last_error.argtypes = [ctypes.c_void_p]
    fake = 4096
    n = ctypes.c_size_t()

    def ws(p, o, backward=0):
        code = libmodal.modal_workspace_size(ctypes.byref(p), ctypes.byref(o), backward, ctypes.byref(n))
        return code, n.value

    def prob(l_min=2, l_max=200, nbl=8, nbp=8, nx=40, nl=10, np_=10):
        return Problem(l_min, l_max, nbl, nbp, nx, nl, np_, 0, fake, fake, fake, fake, fake, fake)

    ok = Opts(0, 0, 0, 0)
    code, b64 = ws(prob(), ok)
    assert code == 0 and b64 > 0
    code, btc = ws(prob(), Opts(0, 2, 0, 0))
    assert code == 0 and btc > b64                       # slices and Y of the tensor-core form
    code, bwd = ws(prob(), ok, backward=1)
    assert code == 0 and bwd >= b64
    code, b1 = ws(prob(nx=400), Opts(0, 0, 0, 1))        # one radial point per chunk
    code2, ball = ws(prob(nx=400), ok)
    assert code == 0 and code2 == 0 and b1 < ball
    # rejections: status code and a message naming the problem
    for p, o, code_expect, word in [
        (prob(nbl=65), ok, 1, b"basis sizes"),            # nb > 64
        (prob(nbl=0), ok, 1, b"basis sizes"),
        (prob(nx=-1), ok, 1, b"negative"),
        (prob(l_min=-1), ok, 1, b"l range"),
        (prob(), Opts(0, 7, 0, 0), 1, b"precision"),       # unknown precision
        (prob(), Opts(-3, 0, 0, 0), 1, b"n_mu"),
        (prob(), Opts(0, 0, 0, -2), 1, b"x_chunk"),
        (prob(l_max=5000), ok, 5, b"6400"),                # N_mu beyond the GL kernel's limit
    ]:
        code, _ = ws(p, o)
        assert code == code_expect, (p.nb_late, o.precision, code)
        assert word in libmodal.modal_last_error(None)
