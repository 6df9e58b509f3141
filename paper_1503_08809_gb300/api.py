"""Python names for the C ABI (argument marshalling only).

Device memory comes from torch CUDA tensors; each call runs on torch's
current stream of the tensors' device.  Names follow include/modal.h.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import Opts, Problem, check, lib

_f64, _i32 = torch.float64, torch.int32


class Handle:
    """Owns a ``modal_handle`` (scratch memory of the library) for one device."""

    def __init__(self, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            h = ctypes.c_void_p()
            check(lib().modal_handle_create(ctypes.byref(h)))
        self.ptr = h

    def close(self):
        if getattr(self, "ptr", None):
            lib().modal_handle_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nbytes: int):
        check(lib().modal_handle_reserve(self.ptr, ctypes.c_size_t(int(nbytes))), self.ptr)


_DEFAULT = {}


def default_handle(device=None) -> Handle:
    d = torch.device(device if device is not None else "cuda")
    if d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    h = _DEFAULT.get(d)
    if h is None:
        h = _DEFAULT[d] = Handle(d)
    return h


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, device, dtype):
    t = torch.as_tensor(t, dtype=dtype) if not isinstance(t, torch.Tensor) else t.to(dtype)
    return t.to(device).contiguous()


class DeviceProblem:
    """A projection problem resident in device memory (see modal_problem)."""

    def __init__(self, q, qt, w_l, x_w, late_modes, prim_modes, l_min: int, l_max: int,
                 device="cuda"):
        self.device = torch.device(device)
        self.q = _dev(q, self.device, _f64)
        self.qt = _dev(qt, self.device, _f64)
        self.w_l = _dev(w_l, self.device, _f64)
        self.x_w = _dev(x_w, self.device, _f64)
        self.late_modes = _dev(late_modes, self.device, _i32).reshape(-1, 3)
        self.prim_modes = _dev(prim_modes, self.device, _i32).reshape(-1, 3)
        self.l_min, self.l_max = int(l_min), int(l_max)
        L = self.l_max - self.l_min + 1
        if self.q.dim() != 2 or self.q.shape[1] != L:
            raise ValueError("q must be [nb_late][L]")
        if self.qt.dim() != 3 or self.qt.shape[2] != L:
            raise ValueError("qt must be [n_x][nb_prim][L]")

    @classmethod
    def from_host(cls, P, device="cuda", xw_kind: int = _lib.XW_TRAPEZOID, handle=None,
                  x_w=None):
        """Upload a ``synthetic.Problem``; the radial weights are computed on the
        device by ``modal_x_weights`` unless given."""
        dev = torch.device(device)
        if x_w is None:
            x_w = x_weights(torch.as_tensor(P.x, dtype=_f64, device=dev), xw_kind, handle=handle)
        return cls(P.q, P.qt, P.w_l, x_w, P.late_modes, P.prim_modes, P.l_min, P.l_max, dev)

    @property
    def nb_late(self):
        return int(self.q.shape[0])

    @property
    def nb_prim(self):
        return int(self.qt.shape[1])

    @property
    def n_x(self):
        return int(self.qt.shape[0])

    @property
    def L(self):
        return self.l_max - self.l_min + 1

    @property
    def n_late(self):
        return int(self.late_modes.shape[0])

    @property
    def n_prim(self):
        return int(self.prim_modes.shape[0])

    def n_mu_exact(self) -> int:
        return (3 * self.l_max + 2) // 2

    def struct(self, qt: Optional[torch.Tensor] = None, q: Optional[torch.Tensor] = None) -> Problem:
        qt = self.qt if qt is None else qt
        q = self.q if q is None else q
        return Problem(self.l_min, self.l_max, int(q.shape[0]), int(qt.shape[1]), int(qt.shape[0]),
                       self.n_late, self.n_prim, 0, q.data_ptr(), qt.data_ptr(),
                       self.w_l.data_ptr(), self.x_w.data_ptr(), self.late_modes.data_ptr(),
                       self.prim_modes.data_ptr())


def _opts(precision=_lib.PREC_FP64, n_mu=0, allow_inexact_gl=False, x_chunk=0,
          error_estimate: Optional[torch.Tensor] = None) -> Opts:
    return Opts(int(n_mu), int(precision), int(bool(allow_inexact_gl)), int(x_chunk),
                None if error_estimate is None else error_estimate.data_ptr())


def _h(handle, device):
    return handle if handle is not None else default_handle(device)


def gl_nodes(n_mu: int, device="cuda", handle=None):
    """modal_gl_nodes: Gauss-Legendre nodes (ascending) and weights."""
    device = torch.device(device)
    h = _h(handle, device)
    mu = torch.empty(n_mu, dtype=_f64, device=device)
    om = torch.empty(n_mu, dtype=_f64, device=device)
    check(lib().modal_gl_nodes(h.ptr, int(n_mu), _ptr(mu), _ptr(om), _stream(device)), h.ptr)
    return mu, om


def legendre_table(mu: torch.Tensor, l_min: int, l_max: int, w_l: Optional[torch.Tensor] = None,
                   handle=None):
    """modal_legendre_table: A[j][l - l_min] = w_l P_l(mu_j)."""
    h = _h(handle, mu.device)
    A = torch.empty(mu.numel(), l_max - l_min + 1, dtype=_f64, device=mu.device)
    check(lib().modal_legendre_table(h.ptr, int(mu.numel()), _ptr(mu), int(l_min), int(l_max),
                                     _ptr(w_l), _ptr(A), _stream(mu.device)), h.ptr)
    return A


def x_weights(x: torch.Tensor, kind: int = _lib.XW_TRAPEZOID, handle=None):
    """modal_x_weights: radial weights including x^2."""
    x = x.to(_f64).contiguous()
    h = _h(handle, x.device)
    w = torch.empty_like(x)
    check(lib().modal_x_weights(h.ptr, int(kind), int(x.numel()), _ptr(x), _ptr(w),
                                _stream(x.device)), h.ptr)
    return w


def contract_l(dp: DeviceProblem, n_mu: int, A: torch.Tensor, precision: int = _lib.PREC_FP64,
               handle=None):
    """modal_contract_l: M[x][j][a][p] (FP64)."""
    h = _h(handle, dp.device)
    M = torch.empty(dp.n_x, n_mu, dp.nb_late, dp.nb_prim, dtype=_f64, device=dp.device)
    s = dp.struct()
    check(lib().modal_contract_l(h.ptr, ctypes.byref(s), int(n_mu), _ptr(A), int(precision),
                                 _ptr(M), _stream(dp.device)), h.ptr)
    return M


def handle_status(handle=None, device=None) -> int:
    """modal_handle_status: MODAL_OK, or raise ModalError(ETIMEOUT) if a bounded
    device-side wait of an earlier call gave up."""
    h = _h(handle, device)
    code = lib().modal_handle_status(h.ptr)
    check(code, h.ptr)
    return code


def set_option(option: int, value: int, handle=None, device=None):
    """modal_handle_set_option (tunables of the tensor-core form)."""
    h = _h(handle, device)
    check(lib().modal_handle_set_option(h.ptr, int(option), int(value)), h.ptr)


def set_wait_limit(cycles: int, handle=None, device=None):
    """modal_handle_set_wait_limit (0 restores the default bound)."""
    h = _h(handle, device)
    check(lib().modal_handle_set_wait_limit(h.ptr, int(cycles)), h.ptr)


def project_separable(dp: DeviceProblem, precision: int = _lib.PREC_FP64, n_mu: int = 0,
                      allow_inexact_gl: bool = False, x_chunk: int = 0, out=None, handle=None,
                      qt: Optional[torch.Tensor] = None, q: Optional[torch.Tensor] = None,
                      error_estimate: Optional[torch.Tensor] = None):
    """modal_project_separable: Gamma' [n_late][n_prim] (FP64).  If
    ``error_estimate`` (a [n_late][n_prim] FP64 device tensor) is given, it
    receives the same projection of |M| with |weights| (the per-entry error
    scale)."""
    h = _h(handle, dp.device)
    gamma = out if out is not None else torch.empty(dp.n_late, dp.n_prim, dtype=_f64,
                                                    device=dp.device)
    s = dp.struct(qt, q)
    o = _opts(precision, n_mu, allow_inexact_gl, x_chunk, error_estimate)
    check(lib().modal_project_separable(h.ptr, ctypes.byref(s), ctypes.byref(o), _ptr(gamma),
                                        _stream(dp.device)), h.ptr)
    return gamma


def project_direct(dp: DeviceProblem, l_grid=None, l_dw=None, weight_mode: int = _lib.W_EXACT_3J,
                   out=None, handle=None):
    """modal_project_direct: the tetrahedral sum of Eq. 3D on a multipole grid
    (dense l_min..l_max when l_grid is None)."""
    h = _h(handle, dp.device)
    if l_grid is None:
        l_grid = np.arange(dp.l_min, dp.l_max + 1)
    lg = _dev(l_grid, dp.device, _i32)
    dw = None if l_dw is None else _dev(l_dw, dp.device, _f64)
    gamma = out if out is not None else torch.empty(dp.n_late, dp.n_prim, dtype=_f64,
                                                    device=dp.device)
    s = dp.struct()
    check(lib().modal_project_direct(h.ptr, ctypes.byref(s), _ptr(lg), _ptr(dw), int(lg.numel()),
                                     int(weight_mode), _ptr(gamma), _stream(dp.device)), h.ptr)
    return gamma


def project_backward(dp: DeviceProblem, dgamma: torch.Tensor, precision: int = _lib.PREC_FP64,
                     n_mu: int = 0, want_dq: bool = True, x_chunk: int = 0, handle=None,
                     qt: Optional[torch.Tensor] = None, q: Optional[torch.Tensor] = None):
    """modal_project_backward: (dL/dq~ [n_x][nb_prim][L], dL/dq [nb_late][L] or None)."""
    h = _h(handle, dp.device)
    g = dgamma.to(_f64).contiguous()
    qt_ = dp.qt if qt is None else qt
    q_ = dp.q if q is None else q
    dqt = torch.empty_like(qt_)
    dq = torch.empty_like(q_) if want_dq else None
    s = dp.struct(qt, q)
    o = _opts(precision, n_mu, False, x_chunk)
    check(lib().modal_project_backward(h.ptr, ctypes.byref(s), ctypes.byref(o), _ptr(g), _ptr(dqt),
                                       _ptr(dq), _stream(dp.device)), h.ptr)
    return dqt, dq


def project_separable_batched(dps: Sequence[DeviceProblem], precision: int = _lib.PREC_FP64,
                              outs=None, handle=None):
    """modal_project_separable_batched: one call for many uneven problems."""
    if not dps:
        return []
    dev = dps[0].device
    h = _h(handle, dev)
    gammas = outs if outs is not None else [
        torch.empty(d.n_late, d.n_prim, dtype=_f64, device=dev) for d in dps]
    arr = (Problem * len(dps))(*[d.struct() for d in dps])
    outp = (ctypes.c_void_p * len(dps))(*[g.data_ptr() for g in gammas])
    o = _opts(precision)
    check(lib().modal_project_separable_batched(h.ptr, len(dps), arr, ctypes.byref(o), outp,
                                                _stream(dev)), h.ptr)
    return gammas


def gram(dp: DeviceProblem, w_gram, precision: int = _lib.PREC_FP64, n_mu: int = 0,
         allow_inexact_gl: bool = False, out=None, handle=None,
         error_estimate: Optional[torch.Tensor] = None):
    """modal_gram: the late basis's Gram matrix <Q_n, Q_r> [n_late][n_late]
    (Appendix A inner product) with l weight ``w_gram`` ([L]; the paper's is
    (2l+1)^(2/3))."""
    h = _h(handle, dp.device)
    G = out if out is not None else torch.empty(dp.n_late, dp.n_late, dtype=_f64, device=dp.device)
    wg = _dev(w_gram, dp.device, _f64)
    s = dp.struct()
    o = _opts(precision, n_mu, allow_inexact_gl, 0, error_estimate)
    check(lib().modal_gram(h.ptr, ctypes.byref(s), _ptr(wg), ctypes.byref(o), _ptr(G),
                           _stream(dp.device)), h.ptr)
    return G


def gram_solve(G: torch.Tensor, rhs: torch.Tensor, out=None, handle=None, raise_if_not_pd: bool = True):
    """modal_gram_solve: X = G^{-1} rhs by Cholesky (FP64).  Returns X; with
    ``raise_if_not_pd`` (the default) waits for the stream and raises
    ModalError(MODAL_EINVAL) if G is not positive definite, else returns
    (X, info) where info is the device status word."""
    G = G.to(_f64).contiguous()
    rhs = rhs.to(_f64).contiguous()
    n, m = int(G.shape[0]), int(rhs.shape[1])
    if G.shape != (n, n) or rhs.shape[0] != n:
        raise ValueError("G must be [n][n] and rhs [n][m]")
    h = _h(handle, G.device)
    X = out if out is not None else torch.empty_like(rhs)
    info = torch.zeros(1, dtype=_i32, device=G.device)
    check(lib().modal_gram_solve(h.ptr, n, m, _ptr(G), _ptr(rhs), _ptr(X), _ptr(info),
                                 _stream(G.device)), h.ptr)
    if not raise_if_not_pd:
        return X, info
    k = int(info.item())
    if k:
        raise _lib.ModalError(_lib.MODAL_EINVAL,
                         f"the Gram matrix is not positive definite (leading minor of order {k})")
    return X


def project_full(dp: DeviceProblem, w_gram, precision: int = _lib.PREC_FP64, handle=None):
    """The full Gamma = <Q,Q>^{-1} Gamma' (Appendix A): Gamma' by
    modal_project_separable, the Gram matrix by modal_gram, then
    modal_gram_solve.  Raises ModalError if the Gram matrix is not positive
    definite or a device-side check of the tensor-core form failed."""
    h = _h(handle, dp.device)
    gp = project_separable(dp, precision=precision, handle=h)
    G = gram(dp, w_gram, precision=precision, handle=h)
    if precision == _lib.PREC_OZAKI_BF16:
        handle_status(handle=h)
    return gram_solve(G, gp, out=gp, handle=h)
