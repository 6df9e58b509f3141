"""Seeded synthetic inputs for the Modal Gamma' projection.

This module is shared by the oracle tests, the GPU tests and the benchmark.
It only *draws* inputs (basis tables, radial grids, weights, mode lists,
random phases and fit vectors); it performs none of the projection's own
arithmetic (no Gauss-Legendre nodes, no l contraction, no radial weights,
no 3j symbols).

The recipe stands in for the transfer-function tables of the paper's
appendix (Appendix A, the projected primordial basis q~_i(x, l)), which
need Boltzmann-code output that is not available here.  Shapes follow the
paper's typical sizes (Section 2.1: n_max ~ 2000, l_max ~ 2000, ~200 radial
points; Section 3.1.3: up to ~3000 mu points):

* late-time 1D basis   q_a(l)     = P_a(2 l / l_max - 1)
* projected primordial q~_p(l, x) = P_p(2 l / l_max - 1)
                                    * exp(-((x - 14000) / 300)^2)
                                    * cos(l (x - 14000) / 14000 + phi_p),
  phi_p ~ U[0, 2 pi) from numpy's PCG64 (default_rng(seed))
* l weight             w_l        = (2l+1) sqrt(l(l+1)) exp((l/1500)^2)
  (stands for (2l+1) / (v_l sqrt(C_l)) of Eq. legendre)
* radial grid          x          = linspace(13000, 14500, n_x), endpoints
  included (the last-scattering peak of Section 3.2.4 sits at ~14000).

The Legendre polynomials of the *basis* are evaluated with numpy's
``legval`` (a library routine), so nothing here is shared with either the
oracle's or the kernels' Legendre recurrence for P_l(mu).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial import legendre as _npleg

X_LO, X_HI = 13000.0, 14500.0
X_PEAK, X_WIDTH, X_FREQ = 14000.0, 300.0, 14000.0


def n_mu_exact(l_max: int) -> int:
    """Smallest GL order that integrates P_l1 P_l2 P_l3 exactly for l_i <= l_max:
    2 N - 1 >= 3 l_max  ->  N = ceil((3 l_max + 1) / 2)."""
    return (3 * l_max + 2) // 2


def basis_legendre(nb: int, ls: np.ndarray, l_max: int) -> np.ndarray:
    """[nb][len(ls)] array of P_a(2 l / l_max - 1), a = 0..nb-1 (numpy legval)."""
    t = 2.0 * ls.astype(np.float64) / float(l_max) - 1.0
    out = np.empty((nb, ls.size), dtype=np.float64)
    for a in range(nb):
        c = np.zeros(a + 1)
        c[a] = 1.0
        out[a] = _npleg.legval(t, c)
    return out


def mode_list(nb: int) -> np.ndarray:
    """All sorted index triples (i <= j <= k) of an nb-function 1D basis, in the
    order of the paper's example map (Appendix A: 000, 001, 011, 111, 002, 012,
    ...): k outermost, then j, then i.  Returns int32 [C(nb+2,3)][3]."""
    out = []
    for k in range(nb):
        for j in range(k + 1):
            for i in range(j + 1):
                out.append((i, j, k))
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)


def sparse_l_grid(l_max: int, l_min: int = 2):
    """Sparse multipole grid of the Planck-scale direct check: every l up to
    50, step 2 to 200, step 5 to 500, step 10 above.  Returns (l_grid int32,
    l_dw float64) where l_dw is the number of dense multipoles each grid point
    stands for (midpoint cells, clipped to [l_min, l_max])."""
    pts = list(range(l_min, min(50, l_max) + 1))
    pts += list(range(52, min(200, l_max) + 1, 2))
    pts += list(range(205, min(500, l_max) + 1, 5))
    pts += list(range(510, l_max + 1, 10))
    return _cells(pts, l_min, l_max)


def stepped_l_grid(l_max: int, step: int, dense_to: int = 50, l_min: int = 2):
    """Every l up to ``dense_to``, then every ``step``-th l up to l_max (and
    l_max itself), with midpoint cells as in ``sparse_l_grid``."""
    pts = list(range(l_min, min(dense_to, l_max) + 1))
    pts += list(range(dense_to + step, l_max + 1, step)) + [l_max]
    return _cells(pts, l_min, l_max)


def _cells(pts, l_min: int, l_max: int):
    g = np.asarray(sorted(set(p for p in pts if l_min <= p <= l_max)), dtype=np.int64)
    lo = np.empty(g.size)
    hi = np.empty(g.size)
    lo[0] = l_min - 0.5
    hi[-1] = l_max + 0.5
    mid = 0.5 * (g[1:] + g[:-1])
    lo[1:] = mid
    hi[:-1] = mid
    dw = hi - lo
    return g.astype(np.int32), dw.astype(np.float64)


@dataclass
class Problem:
    """One synthetic projection problem (host numpy arrays, C order)."""
    l_min: int
    l_max: int
    nb_late: int
    nb_prim: int
    n_x: int
    q: np.ndarray          # [nb_late][L]
    qt: np.ndarray         # [n_x][nb_prim][L]
    w_l: np.ndarray        # [L]
    x: np.ndarray          # [n_x]
    phi: np.ndarray        # [nb_prim]
    late_modes: np.ndarray  # [n_late][3] int32
    prim_modes: np.ndarray  # [n_prim][3] int32
    seed: int = 1
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return self.l_max - self.l_min + 1

    @property
    def n_mu(self) -> int:
        return n_mu_exact(self.l_max)

    @property
    def n_late(self) -> int:
        return int(self.late_modes.shape[0])

    @property
    def n_prim(self) -> int:
        return int(self.prim_modes.shape[0])

    @property
    def slices(self) -> int:
        return self.n_x * self.n_mu


def make_problem(l_max: int, nb: int, n_x: int, seed: int = 1, l_min: int = 2,
                 nb_prim: int | None = None, name: str = "") -> Problem:
    """Draw one problem with the recipe in the module docstring."""
    nb_prim = nb if nb_prim is None else nb_prim
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi, nb_prim)
    ls = np.arange(l_min, l_max + 1, dtype=np.int64)
    q = basis_legendre(nb, ls, l_max)
    qp = basis_legendre(nb_prim, ls, l_max)
    x = np.linspace(X_LO, X_HI, n_x)
    env = np.exp(-((x - X_PEAK) / X_WIDTH) ** 2)                      # [n_x]
    phase = ls[None, None, :] * ((x - X_PEAK) / X_FREQ)[:, None, None] + phi[None, :, None]
    qt = qp[None, :, :] * env[:, None, None] * np.cos(phase)          # [n_x][nb][L]
    lf = ls.astype(np.float64)
    w_l = (2.0 * lf + 1.0) * np.sqrt(lf * (lf + 1.0)) * np.exp((lf / 1500.0) ** 2)
    return Problem(l_min=l_min, l_max=l_max, nb_late=nb, nb_prim=nb_prim, n_x=n_x,
                   q=np.ascontiguousarray(q), qt=np.ascontiguousarray(qt),
                   w_l=np.ascontiguousarray(w_l), x=x, phi=phi,
                   late_modes=mode_list(nb), prim_modes=mode_list(nb_prim),
                   seed=seed, name=name)


def gram_weights(l_min: int, l_max: int) -> np.ndarray:
    """l weight of the Gram matrix <Q_n, Q_r> (Appendix A): (2l+1) / v_l^2
    with v_l = (2l+1)^(1/6), i.e. (2l+1)^(2/3)."""
    lf = np.arange(l_min, l_max + 1, dtype=np.float64)
    return (2.0 * lf + 1.0) ** (2.0 / 3.0)


# Named workloads -------------------------------------------------------------

def cpu_size(seed: int = 1) -> Problem:
    """l_max = 48, 5 basis functions (35 modes each side), 24 x points, N_mu = 73."""
    return make_problem(48, 5, 24, seed=seed, name="lmax48_nb5_nx24")


def planck_size(seed: int = 1, n_x: int = 500) -> Problem:
    """l_max = 2000, 20 basis functions (1540 modes each side), 500 x points,
    N_mu = 3001."""
    return make_problem(2000, 20, n_x, seed=seed, name=f"lmax2000_nb20_nx{n_x}")


def grad_size(seed: int = 1, nb: int = 16) -> Problem:
    """l_max = 1000, 16 basis functions (816 modes; 15 functions give 680),
    300 x points, N_mu = 1501."""
    return make_problem(1000, nb, 300, seed=seed, name=f"lmax1000_nb{nb}_nx300")


def batched_models(n: int = 64, base_seed: int = 1000, scale: float = 1.0):
    """n primordial models of uneven size: l_max ~ U[500, 2500], basis size
    ~ U{10..20}, x count ~ U{200..600}; model i uses seed base_seed + i.
    ``scale`` < 1 shrinks l_max and n_x (for tests), keeping the mix."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(base_seed + i)
        lmax = int(rng.integers(500, 2501))
        nb = int(rng.integers(10, 21))
        nx = int(rng.integers(200, 601))
        if scale != 1.0:
            lmax = max(8, int(round(lmax * scale)))
            nx = max(4, int(round(nx * scale)))
            nb = max(2, min(nb, int(round(nb * max(scale, 0.25)))))
        out.append(make_problem(lmax, nb, nx, seed=base_seed + i, name=f"model{i}"))
    return out


def fit_vectors(n_prim: int, seed: int = 1, perturb: float = 0.1):
    """alpha ~ N(0,1) and a perturbation delta ~ perturb * N(0,1); the fit
    target is b = Gamma (alpha + delta), formed by whoever owns Gamma."""
    rng = np.random.default_rng(seed + 7919)
    alpha = rng.standard_normal(n_prim)
    delta = perturb * rng.standard_normal(n_prim)
    return alpha, delta


def random_cotangent(n_late: int, n_prim: int, seed: int = 3) -> np.ndarray:
    """A seeded dL/dGamma for adjoint tests."""
    return np.random.default_rng(seed).standard_normal((n_late, n_prim))
