"""FP64 CPU oracle for the Modal Gamma' projection (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``modal_oracle.c`` (plain C, built by
``oracle/build.py`` with gcc) through ctypes and shares no code with the CUDA
library.  Each wrapper names the passage of arXiv 1503.08809 it follows; the
C file has the derivations.

Parity status: all functions (including ``gram`` and ``full_gamma``) pinned by
``tests/test_oracle_pins.py``.  ``direct(..., weight_mode=SMOOTH)`` on sparse
grids is pinned to its formula (a literal cube sum on a small grid), but it
only approximates the dense sum: how close it comes is measured and
reported, not pinned.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path
from types import SimpleNamespace

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB = None

EXACT, SMOOTH = 0, 1
TRAPEZOID, HERMITE = 0, 1

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)


def lib_path() -> Path:
    return _HERE / "_build" / "liboracle.so"


def _load():
    global _LIB
    if _LIB is not None:
        return _LIB
    p = lib_path()
    if not p.exists():
        from . import build as _b
        _b.build()
    lib = ctypes.CDLL(str(p))
    lib.oracle_threej000_sq.restype = ctypes.c_double
    lib.oracle_threej000_sq.argtypes = [ctypes.c_int] * 3
    lib.oracle_gosper_threej000_sq.restype = ctypes.c_double
    lib.oracle_gosper_threej000_sq.argtypes = [ctypes.c_int] * 3
    lib.oracle_gl_nodes.argtypes = [ctypes.c_int, _d, _d]
    lib.oracle_legendre_row.argtypes = [ctypes.c_int, ctypes.c_double, _d]
    lib.oracle_x_weights.argtypes = [ctypes.c_int, ctypes.c_int, _d, _d]
    lib.oracle_num_threads.restype = ctypes.c_int
    common = [ctypes.c_int] * 5 + [_d, _d, _d, _d]
    lib.oracle_separable.argtypes = common + [ctypes.c_int, _d, _d, ctypes.c_int, _i,
                                              ctypes.c_int, _i, _d]
    lib.oracle_separable_abs.argtypes = common + [ctypes.c_int, _d, _d, ctypes.c_int, _i,
                                              ctypes.c_int, _i, _d]
    lib.oracle_direct.argtypes = common + [ctypes.c_int, _i, _d, ctypes.c_int,
                                           ctypes.c_int, _i, ctypes.c_int, _i, _d]
    lib.oracle_backward.argtypes = common + [ctypes.c_int, _d, _d, ctypes.c_int, _i,
                                             ctypes.c_int, _i, _d, _d, _d]
    lib.oracle_M.argtypes = [ctypes.c_int] * 5 + [_d, _d, _d, ctypes.c_int, _d, _d]
    _LIB = lib
    return lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_d)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_i)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def threej000_sq(l1: int, l2: int, l3: int) -> float:
    """(l1 l2 l3; 0 0 0)^2 by the closed form (Section 2.1)."""
    return float(_load().oracle_threej000_sq(int(l1), int(l2), int(l3)))


def gosper_threej000_sq(l1: int, l2: int, l3: int) -> float:
    """Gosper approximation of (l1 l2 l3; 0 0 0)^2 (Section 2.1)."""
    return float(_load().oracle_gosper_threej000_sq(int(l1), int(l2), int(l3)))


def gl_nodes(n: int):
    """Gauss-Legendre nodes (ascending) and weights, long-double Newton (Section 2.2)."""
    mu = np.zeros(n)
    om = np.zeros(n)
    _load().oracle_gl_nodes(int(n), _pd(mu), _pd(om))
    return mu, om


def legendre_row(lmax: int, mu: float) -> np.ndarray:
    """P_0..P_lmax at mu by the three-term recurrence."""
    P = np.zeros(lmax + 1)
    _load().oracle_legendre_row(int(lmax), float(mu), _pd(P))
    return P


def x_weights(x, kind: int = TRAPEZOID) -> np.ndarray:
    """Radial weights including x^2 (Section 3.2.4: trapezium or Hermite)."""
    x = _f64(x)
    w = np.zeros_like(x)
    _load().oracle_x_weights(int(kind), int(x.size), _pd(x), _pd(w))
    return w


def _common(P, xw):
    return (int(P.l_min), int(P.l_max), int(P.nb_late), int(P.nb_prim), int(P.n_x),
            _f64(P.q), _f64(P.qt), _f64(P.w_l), _f64(xw))


def M_table(P, mu) -> np.ndarray:
    """P_{ii'}(x, mu_j) of Eq. legendre for every slice: [n_x][n_mu][nb_late][nb_prim]."""
    mu = _f64(mu)
    M = np.zeros((P.n_x, mu.size, P.nb_late, P.nb_prim))
    _load().oracle_M(int(P.l_min), int(P.l_max), int(P.nb_late), int(P.nb_prim), int(P.n_x),
                     _pd(_f64(P.q)), _pd(_f64(P.qt)), _pd(_f64(P.w_l)), int(mu.size), _pd(mu),
                     _pd(M))
    return M


def separable(P, n_mu: int | None = None, xw=None, mu=None, om=None,
              late=None, prim=None, magnitudes: bool = False) -> np.ndarray:
    """Gamma' by Eq. 2D (Section 2.2) with GL mu and trapezium x weights.
    ``late``/``prim`` restrict the mode lists (rows/columns).  With
    ``magnitudes`` every weight and each of the six products is taken in
    magnitude: the scale of the rounding error of each entry."""
    n_mu = P.n_mu if n_mu is None else int(n_mu)
    if mu is None:
        mu, om = gl_nodes(n_mu)
    if xw is None:
        xw = x_weights(P.x)
    late = _i32(P.late_modes if late is None else late)
    prim = _i32(P.prim_modes if prim is None else prim)
    l0, l1, nbl, nbp, nx, q, qt, wl, xw = _common(P, xw)
    mu, om = _f64(mu), _f64(om)
    g = np.zeros((late.shape[0], prim.shape[0]))
    fn = _load().oracle_separable_abs if magnitudes else _load().oracle_separable
    fn(l0, l1, nbl, nbp, nx, _pd(q), _pd(qt), _pd(wl), _pd(xw), int(mu.size), _pd(mu), _pd(om),
       int(late.shape[0]), _pi(late), int(prim.shape[0]), _pi(prim), _pd(g))
    return g


def direct(P, l_grid=None, l_dw=None, weight_mode: int = EXACT, xw=None,
           late=None, prim=None) -> np.ndarray:
    """Gamma' by the tetrahedral sum of Eq. 3D (Section 2.1) on a multipole grid."""
    if l_grid is None:
        l_grid = np.arange(P.l_min, P.l_max + 1)
        l_dw = np.ones(l_grid.size)
    if xw is None:
        xw = x_weights(P.x)
    late = _i32(P.late_modes if late is None else late)
    prim = _i32(P.prim_modes if prim is None else prim)
    lg = _i32(l_grid)
    dw = _f64(l_dw)
    l0, l1, nbl, nbp, nx, q, qt, wl, xw = _common(P, xw)
    g = np.zeros((late.shape[0], prim.shape[0]))
    _load().oracle_direct(l0, l1, nbl, nbp, nx, _pd(q), _pd(qt), _pd(wl), _pd(xw),
                          int(lg.size), _pi(lg), _pd(dw), int(weight_mode),
                          int(late.shape[0]), _pi(late), int(prim.shape[0]), _pi(prim),
                          _pd(g))
    return g


def gram(P, w_gram, late=None) -> np.ndarray:
    """Gram matrix <Q_n, Q_r> of the late basis (Appendix A: the inner product
    with weight (h / v1 v2 v3)^2, applied to two late-time basis functions).

    Q_r has the same form as the projected Q~ of Eq. 3D with q~(l, x) replaced
    by q(l) and no radial integral, so this is ``direct`` (the dense
    tetrahedral sum with the exact 3j^2) on a problem whose projected basis is
    q itself at one radial point of unit weight, with the l weight
    w_gram = (2l+1) / v_l^2 in place of w_l = (2l+1) / (v_l sqrt(C_l))."""
    late = _i32(P.late_modes if late is None else late)
    Pg = SimpleNamespace(l_min=P.l_min, l_max=P.l_max, nb_late=P.nb_late, nb_prim=P.nb_late, n_x=1,
                         q=_f64(P.q), qt=_f64(P.q)[None], w_l=_f64(w_gram),
                         late_modes=late, prim_modes=late)
    return direct(Pg, xw=np.ones(1))


def full_gamma(gram_matrix, gamma_prime) -> np.ndarray:
    """Gamma = <Q, Q>^{-1} Gamma' (Appendix A: Gamma_nm = sum_r <Q_n,Q_r>^{-1}
    <Q_r, Q~_m>), by numpy's Cholesky factor of the Gram matrix and two
    triangular solves (scipy).  Raises numpy.linalg.LinAlgError if the Gram
    matrix is not positive definite."""
    from scipy.linalg import solve_triangular
    Lc = np.linalg.cholesky(_f64(gram_matrix))
    y = solve_triangular(Lc, _f64(gamma_prime), lower=True)
    return solve_triangular(Lc.T, y, lower=False)


def backward(P, gbar, n_mu: int | None = None, xw=None, want_dq: bool = True):
    """Adjoint of ``separable``: (dL/dq~ [n_x][nb_prim][L], dL/dq [nb_late][L])."""
    n_mu = P.n_mu if n_mu is None else int(n_mu)
    mu, om = gl_nodes(n_mu)
    if xw is None:
        xw = x_weights(P.x)
    late = _i32(P.late_modes)
    prim = _i32(P.prim_modes)
    l0, l1, nbl, nbp, nx, q, qt, wl, xw = _common(P, xw)
    gb = _f64(gbar)
    dqt = np.zeros((nx, nbp, P.L))
    dq = np.zeros((nbl, P.L)) if want_dq else None
    _load().oracle_backward(l0, l1, nbl, nbp, nx, _pd(q), _pd(qt), _pd(wl), _pd(xw),
                            int(mu.size), _pd(mu), _pd(om), int(late.shape[0]), _pi(late),
                            int(prim.shape[0]), _pi(prim), _pd(gb), _pd(dqt),
                            _pd(dq) if dq is not None else None)
    return dqt, dq
