"""ctypes declarations of the C ABI in include/modal.h."""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

_PKG = Path(__file__).resolve().parent

MODAL_OK, MODAL_EINVAL, MODAL_ENOMEM, MODAL_ECUDA, MODAL_ETIMEOUT, MODAL_EUNSUPPORTED = range(6)
PREC_FP64, PREC_FP32, PREC_OZAKI_BF16, PREC_TF32, PREC_BF16X3 = 0, 1, 2, 3, 4
XW_TRAPEZOID, XW_HERMITE = 0, 1
OPT_TC_TRIPLE_FUSED, OPT_TC_SPLIT_K, OPT_BATCH_STREAMS, OPT_TC_PAIR, OPT_TC_QUEUE, OPT_TC_AUTOTUNE, OPT_TC_OVERLAP = 1, 2, 3, 4, 5, 6, 7
OPT_DIRECT_TENSOR = 8
OPT_TC_OVERLAP_TAIL = 9
W_EXACT_3J, W_SMOOTH_GOSPER = 0, 1

_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}

# every symbol include/modal.h declares (checked by tests/test_abi.py)
EXPORTS = [
    "modal_handle_create", "modal_handle_destroy", "modal_last_error", "modal_workspace_size",
    "modal_handle_reserve", "modal_gl_nodes", "modal_legendre_table", "modal_x_weights",
    "modal_contract_l", "modal_project_separable", "modal_project_direct",
    "modal_project_backward", "modal_project_separable_batched", "modal_profile_enable",
    "modal_profile_read", "modal_handle_status", "modal_handle_set_wait_limit",
    "modal_project_separable_noalloc", "modal_handle_set_option", "modal_gram", "modal_gram_solve",
]


class ModalError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmodal {_STATUS.get(code, code)}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [
        ("l_min", ctypes.c_int32), ("l_max", ctypes.c_int32),
        ("nb_late", ctypes.c_int32), ("nb_prim", ctypes.c_int32),
        ("n_x", ctypes.c_int32), ("n_late", ctypes.c_int32), ("n_prim", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("q", ctypes.c_void_p), ("qt", ctypes.c_void_p), ("w_l", ctypes.c_void_p),
        ("x_w", ctypes.c_void_p), ("late_modes", ctypes.c_void_p),
        ("prim_modes", ctypes.c_void_p),
    ]


class Opts(ctypes.Structure):
    _fields_ = [("n_mu", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("allow_inexact_gl", ctypes.c_int32), ("x_chunk", ctypes.c_int32),
                ("error_estimate", ctypes.c_void_p)]


def lib_path() -> Path:
    debug = os.environ.get("MODAL_DEBUG", "") not in ("", "0")   # the checked-index build
    return _PKG / ("_build_debug" if debug else "_build") / "libmodal.so"


_LIB = None


def lib():
    """Load libmodal.so; raise if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = lib_path()
    if not p.exists():
        raise ImportError(f"{p} is missing: build it with paper_1503_08809_gb300/build.py "
                          "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(str(p))
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    P, O = ctypes.POINTER(Problem), ctypes.POINTER(Opts)
    sig = {
        "modal_handle_create": [ctypes.POINTER(vp)],
        "modal_handle_destroy": [vp],
        "modal_workspace_size": [P, O, ctypes.c_int, ctypes.POINTER(sz)],
        "modal_handle_reserve": [vp, sz],
        "modal_gl_nodes": [vp, i32, vp, vp, vp],
        "modal_legendre_table": [vp, i32, vp, i32, i32, vp, vp, vp],
        "modal_x_weights": [vp, i32, i32, vp, vp, vp],
        "modal_contract_l": [vp, P, i32, vp, i32, vp, vp],
        "modal_project_separable": [vp, P, O, vp, vp],
        "modal_project_direct": [vp, P, vp, vp, i32, i32, vp, vp],
        "modal_project_backward": [vp, P, O, vp, vp, vp, vp],
        "modal_project_separable_batched": [vp, i32, P, O, ctypes.POINTER(vp), vp],
        "modal_profile_enable": [vp, i32],
        "modal_handle_status": [vp],
        "modal_handle_set_option": [vp, i32, ctypes.c_int64],
        "modal_project_separable_noalloc": [P, O, vp, vp],
        "modal_gram": [vp, P, vp, O, vp, vp],
        "modal_gram_solve": [vp, i32, i32, vp, vp, vp, vp, vp],
        "modal_handle_set_wait_limit": [vp, ctypes.c_int64],
        "modal_profile_read": [vp, i32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.modal_last_error.argtypes = [vp]
    L.modal_last_error.restype = ctypes.c_char_p
    _LIB = L
    return L


def check(code: int, handle=None):
    if code != MODAL_OK:
        msg = lib().modal_last_error(handle)
        raise ModalError(code, msg.decode() if msg else "")
