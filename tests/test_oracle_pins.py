"""Pins for the FP64 CPU oracle against facts fixed by the paper and by
mathematics (not against itself).  CPU only.

Each pin is chosen so that a plausible slip in the oracle (dropped term,
wrong sign or index, transposed operand, wrong prefactor, inaccurate nodes)
fails at least one of them.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
import synthetic as syn
from tests._golden import delta_cases


# --------------------------------------------------------------------------
# 1. Wigner 3j (l1 l2 l3; 0 0 0)^2 (Section 2.1, Eq. weight-function)
# --------------------------------------------------------------------------

def threej_factorial_exact(l1, l2, l3) -> Fraction:
    """Racah's factorial form with exact integers (textbook definition)."""
    L = l1 + l2 + l3
    if L % 2 or l3 > l1 + l2 or l1 > l2 + l3 or l2 > l1 + l3:
        return Fraction(0)
    g = L // 2
    f = math.factorial
    num = f(2 * g - 2 * l1) * f(2 * g - 2 * l2) * f(2 * g - 2 * l3) * f(g) ** 2
    den = f(2 * g + 1) * (f(g - l1) * f(g - l2) * f(g - l3)) ** 2
    return Fraction(num, den)


@pytest.mark.parametrize("l,val", [((1, 1, 2), Fraction(2, 15)), ((2, 2, 2), Fraction(2, 35)),
                                   ((3, 4, 5), Fraction(20, 1001)), ((2, 2, 4), Fraction(2, 35)),
                                   ((2, 3, 3), Fraction(4, 105)), ((0, 0, 0), Fraction(1))])
def test_threej_tabulated(l, val):
    assert oracle.threej000_sq(*l) == pytest.approx(float(val), rel=1e-15)


@pytest.mark.parametrize("l", [0, 1, 2, 7, 30, 200])
def test_threej_l_l_0(l):
    assert oracle.threej000_sq(l, l, 0) == pytest.approx(1.0 / (2 * l + 1), rel=1e-14)


def test_threej_brute_force_factorial():
    worst = 0.0
    for l1 in range(0, 36):
        for l2 in range(l1, 36):
            for l3 in range(l2, min(l1 + l2, 40) + 1):
                ex = threej_factorial_exact(l1, l2, l3)
                got = oracle.threej000_sq(l1, l2, l3)
                if ex == 0:
                    assert got == 0.0
                else:
                    worst = max(worst, abs(got / float(ex) - 1.0))
                # symmetric under permutations of the l's
                assert oracle.threej000_sq(l3, l1, l2) == pytest.approx(got, rel=5e-16)
    assert worst < 5e-15


def test_threej_zero_conditions():
    assert oracle.threej000_sq(2, 3, 4) == 0.0          # odd sum
    assert oracle.threej000_sq(2, 2, 6) == 0.0          # triangle broken, even sum
    assert oracle.threej000_sq(10, 3, 5) == 0.0
    assert oracle.threej000_sq(5, 5, 10) > 0.0          # degenerate triangle allowed


@pytest.mark.parametrize("l1,l2", [(2, 3), (10, 17), (40, 45)])
def test_threej_orthogonality(l1, l2):
    """sum_l3 (2 l3 + 1) (l1 l2 l3; 0 0 0)^2 = 1 (orthogonality of 3j symbols)."""
    s = sum((2 * l3 + 1) * oracle.threej000_sq(l1, l2, l3) for l3 in range(0, l1 + l2 + 1))
    assert s == pytest.approx(1.0, abs=1e-13)


def test_gosper_close_to_exact():
    """Section 2.1: the Gosper form approximates the factorial form; it gets
    better with l (coarse bounds, not a parity claim)."""
    for (l1, l2, l3), tol in [((2, 3, 5), 0.05), ((20, 30, 40), 5e-3), ((500, 600, 700), 1e-5),
                              ((1000, 1200, 1500), 5e-6)]:
        ex = oracle.threej000_sq(l1, l2, l3)
        assert oracle.gosper_threej000_sq(l1, l2, l3) == pytest.approx(ex, rel=tol)
    assert oracle.gosper_threej000_sq(2, 2, 6) == 0.0


# --------------------------------------------------------------------------
# 2. Gauss-Legendre rule (Section 2.2)
# --------------------------------------------------------------------------

def test_gl_small_closed_forms():
    mu, om = oracle.gl_nodes(2)
    assert np.allclose(mu, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=2.5e-16)
    assert np.allclose(om, [1.0, 1.0], rtol=0, atol=2.5e-16)
    mu, om = oracle.gl_nodes(3)
    r = math.sqrt(3.0 / 5.0)
    assert np.allclose(mu, [-r, 0.0, r], rtol=0, atol=2.5e-16)
    assert np.allclose(om, [5 / 9, 8 / 9, 5 / 9], rtol=0, atol=2.5e-16)


@pytest.mark.parametrize("n", [5, 24, 73, 150])
def test_gl_moments_and_symmetry(n):
    mu, om = oracle.gl_nodes(n)
    assert np.all(np.diff(mu) > 0)
    assert np.array_equal(mu, -mu[::-1]) and np.array_equal(om, om[::-1])
    assert om.sum() == pytest.approx(2.0, abs=4e-15)
    for k in range(0, n):        # exact for degree 2k <= 2n - 1
        assert (om * mu ** (2 * k)).sum() == pytest.approx(2.0 / (2 * k + 1), rel=1e-13, abs=1e-300)
    # degree 2n is NOT integrated exactly: P_n vanishes at every node, so the
    # rule gives 0 for P_n^2 whose integral is 2/(2n+1)
    Pn = np.array([oracle.legendre_row(n, m)[n] for m in mu])
    assert abs((om * Pn ** 2).sum()) < 1e-12 * 2.0 / (2 * n + 1)


@pytest.mark.parametrize("n", [20, 100])
def test_gl_matches_numpy(n):
    mu, om = oracle.gl_nodes(n)
    m2, o2 = npleg.leggauss(n)
    assert np.allclose(mu, m2, rtol=0, atol=2e-15)
    # numpy's weights are themselves only good to ~1e-12 at n = 100 (the paper's
    # Section 2.2 complaint about library nodes); the moment tests above pin
    # the oracle's weights much tighter.
    assert np.allclose(om, o2, rtol=1e-11, atol=0)


@pytest.mark.parametrize("n", [1501, 3001])
def test_gl_large_exactness(n):
    """sum_j om_j P_l(mu_j) = 2 delta_l0 for l <= 2n-1 (scipy's P_l)."""
    sp = pytest.importorskip("scipy.special")
    mu, om = oracle.gl_nodes(n)
    assert om.sum() == pytest.approx(2.0, abs=1e-13)
    for l in [1, 2, 3, 100, 1001, 2 * n - 2, 2 * n - 1]:
        assert abs((om * sp.eval_legendre(l, mu)).sum()) < 2e-13


def test_legendre_row_matches_numpy():
    for mu in [-0.9, -0.3, 0.0, 0.41, 0.999]:
        P = oracle.legendre_row(40, mu)
        ref = np.array([npleg.legval(mu, np.eye(41)[l]) for l in range(41)])
        assert np.allclose(P, ref, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# 3. Gaunt integral (Section 2.2): sum_j om_j P_l1 P_l2 P_l3 = 2 3j^2
# --------------------------------------------------------------------------

def test_gaunt_identity():
    lmax = 12
    mu, om = oracle.gl_nodes(syn.n_mu_exact(lmax))
    P = np.stack([oracle.legendre_row(lmax, m) for m in mu])       # [j][l]
    worst = 0.0
    for l1, l2, l3 in itertools.product(range(lmax + 1), repeat=3):
        lhs = float((om * P[:, l1] * P[:, l2] * P[:, l3]).sum())
        rhs = 2.0 * float(threej_factorial_exact(l1, l2, l3))
        worst = max(worst, abs(lhs - rhs))
    assert worst < 2e-15


# --------------------------------------------------------------------------
# 4. Radial weights (Section 3.2.4)
# --------------------------------------------------------------------------

def test_trapezoid_weights():
    x = np.linspace(13000.0, 14500.0, 24)
    w = oracle.x_weights(x)
    h = x[1] - x[0]
    base = np.full(24, h)
    base[0] = base[-1] = h / 2
    assert np.allclose(w, base * x ** 2, rtol=1e-12)
    # without the x^2 factor the rule is exact for linear integrands
    y = 3.0 - 2e-4 * x
    assert (base * y).sum() == pytest.approx(
        3.0 * (x[-1] - x[0]) - 1e-4 * (x[-1] ** 2 - x[0] ** 2), rel=1e-13)


def test_hermite_weights():
    """Hermite rule of Section 3.2.4 (weights divided by x^2 to see the bare
    rule): exact for linear integrands, and converging faster than the
    trapezium rule on a smooth integrand."""
    x = np.sort(np.random.default_rng(5).uniform(1.0, 3.0, 40))
    x[0], x[-1] = 1.0, 3.0
    w = oracle.x_weights(x, oracle.HERMITE) / x ** 2
    y = 1.5 + 0.25 * x
    assert (w * y).sum() == pytest.approx(1.5 * 2 + 0.125 * (9 - 1), rel=1e-13)
    exact = math.cos(1.0) - math.cos(3.0)
    eh, et = [], []
    for n in (50, 100, 200):
        xs = np.linspace(1.0, 3.0, n)
        eh.append(abs((oracle.x_weights(xs, oracle.HERMITE) / xs ** 2 * np.sin(xs)).sum() - exact))
        et.append(abs((oracle.x_weights(xs) / xs ** 2 * np.sin(xs)).sum() - exact))
    assert eh[2] < eh[0] / 3.9          # at least second order
    assert all(h < t for h, t in zip(eh, et))


# --------------------------------------------------------------------------
# 5. Closed-form worked examples (tests/golden/delta_basis.txt)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", list(delta_cases()), ids=lambda c: c[0])
def test_delta_basis_golden(case):
    name, P, expected = case
    xw = np.ones(1)
    gs = oracle.separable(P, xw=xw)[0, 0]
    gd = oracle.direct(P, xw=xw)[0, 0]
    scale = 1.0 / (70 * math.pi)
    assert gs == pytest.approx(expected, rel=1e-14, abs=1e-15 * scale)
    assert gd == pytest.approx(expected, rel=1e-14, abs=1e-15 * scale)


# --------------------------------------------------------------------------
# 6. Brute force from the Appendix-A definitions on a tiny problem
# --------------------------------------------------------------------------

def brute_force_gamma(l_min, l_max, q, qt, v, C, xw, late, prim):
    """Gamma'_{n n'} = <Q_n, Q~'_{n'}> over the whole cube (Appendix A):
    <A,B> = sum (h/(v1 v2 v3))^2 A B, h^2 = prod(2l+1)/(4 pi) 3j^2,
    Q_n = 1/6 sum_perm q q q, Q~'_n = v1 v2 v3/sqrt(C1 C2 C3) Q~_n,
    Q~_n = 1/6 int r^2 dr sum_perm q~ q~ q~ (radial weights xw)."""
    ls = range(l_min, l_max + 1)
    G = np.zeros((len(late), len(prim)))
    for l1, l2, l3 in itertools.product(ls, repeat=3):
        tj = float(threej_factorial_exact(l1, l2, l3))
        if tj == 0.0:
            continue
        k = (l1 - l_min, l2 - l_min, l3 - l_min)
        h2 = (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi) * tj
        vv = v[k[0]] * v[k[1]] * v[k[2]]
        for n, (a, b, c) in enumerate(late):
            Q = sum(q[pa, k[0]] * q[pb, k[1]] * q[pc, k[2]]
                    for pa, pb, pc in itertools.permutations((a, b, c))) / 6.0
            for m_, (p, r, s) in enumerate(prim):
                Qt = sum(xw[x] * sum(qt[x, pa, k[0]] * qt[x, pb, k[1]] * qt[x, pc, k[2]]
                                     for pa, pb, pc in itertools.permutations((p, r, s)))
                         for x in range(qt.shape[0])) / 6.0
                Qtp = vv / math.sqrt(C[k[0]] * C[k[1]] * C[k[2]]) * Qt
                G[n, m_] += h2 / vv ** 2 * Q * Qtp
    return G


def test_brute_force_cube_tiny():
    rng = np.random.default_rng(11)
    l_min, l_max, nb, nx = 2, 7, 3, 3
    L = l_max - l_min + 1
    ls = np.arange(l_min, l_max + 1)
    q = rng.standard_normal((nb, L))
    qt = rng.standard_normal((nx, nb, L))
    v = (2 * ls + 1.0) ** (1 / 6)                      # Appendix A
    C = rng.uniform(0.5, 2.0, L)
    w = (2 * ls + 1.0) / (v * np.sqrt(C))              # Eq. legendre's l weight
    xw = rng.uniform(0.2, 1.0, nx)
    modes = syn.mode_list(nb)
    P = syn.Problem(l_min=l_min, l_max=l_max, nb_late=nb, nb_prim=nb, n_x=nx, q=q, qt=qt,
                    w_l=w, x=np.arange(nx, dtype=float), phi=np.zeros(nb),
                    late_modes=modes, prim_modes=modes)
    ref = brute_force_gamma(l_min, l_max, q, qt, v, C, xw, modes.tolist(), modes.tolist())
    gs = oracle.separable(P, xw=xw)
    gd = oracle.direct(P, xw=xw)
    s = np.abs(ref).max()
    assert np.abs(gs - ref).max() / s < 1e-13
    assert np.abs(gd - ref).max() / s < 1e-13


# --------------------------------------------------------------------------
# 7. Symmetries and agreement of the two forms
# --------------------------------------------------------------------------

def test_permutation_symmetry():
    P = syn.make_problem(20, 4, 5, seed=3)
    g = oracle.separable(P)
    rng = np.random.default_rng(0)
    late = np.array([rng.permutation(m) for m in P.late_modes], dtype=np.int32)
    prim = np.array([rng.permutation(m) for m in P.prim_modes], dtype=np.int32)
    g2 = oracle.separable(P, late=late, prim=prim)
    g3 = oracle.direct(P, late=late, prim=prim)
    s = np.abs(g).max()
    assert np.abs(g2 - g).max() / s < 1e-14
    assert np.abs(g3 - g).max() / s < 1e-12


def test_separable_equals_direct_cpu_size():
    """Eq. 2D with an exact GL rule equals Eq. 3D on the dense grid
    (Section 2.2); l_max = 48, 5 functions, 24 x points."""
    P = syn.cpu_size()
    gs = oracle.separable(P)
    gd = oracle.direct(P)
    assert np.abs(gs - gd).max() / np.abs(gd).max() < 1e-12


def test_too_few_mu_nodes_breaks_agreement():
    """With N_mu below (3 l_max + 1)/2 the rule is no longer exact and the
    forms disagree -- the accuracy condition is real, not vacuous."""
    P = syn.make_problem(24, 3, 4, seed=2)
    gd = oracle.direct(P)
    ok = oracle.separable(P, n_mu=syn.n_mu_exact(24))
    bad = oracle.separable(P, n_mu=syn.n_mu_exact(24) - 6)
    s = np.abs(gd).max()
    assert np.abs(ok - gd).max() / s < 1e-12
    assert np.abs(bad - gd).max() / s > 1e-9


def test_unequal_basis_sizes():
    P = syn.make_problem(16, 4, 3, seed=4, nb_prim=2)
    gs = oracle.separable(P)
    gd = oracle.direct(P)
    assert gs.shape == (20, 4)
    assert np.abs(gs - gd).max() / np.abs(gd).max() < 1e-12


def test_sparse_grid_exact_on_dense_grid_is_dense_sum():
    P = syn.make_problem(18, 3, 4, seed=6)
    lg = np.arange(2, 19)
    a = oracle.direct(P, l_grid=lg, l_dw=np.ones(lg.size))
    b = oracle.direct(P)
    assert np.array_equal(a, b)


def test_sparse_grid_smooth_approximates_dense():
    """Parity unpinned: SMOOTH on the sparse grid only approximates the dense
    sum; check it is in the right ballpark (sanity, not parity)."""
    P = syn.make_problem(120, 3, 6, seed=7)
    lg, dw = syn.sparse_l_grid(120)
    dense = oracle.direct(P)
    sm = oracle.direct(P, l_grid=lg, l_dw=dw, weight_mode=oracle.SMOOTH)
    rel = np.abs(sm - dense).max() / np.abs(dense).max()
    assert rel < 0.5


# --------------------------------------------------------------------------
# 8. Adjoint against central finite differences (h = 1e-6 relative)
# --------------------------------------------------------------------------

def test_backward_finite_differences():
    P = syn.make_problem(14, 3, 3, seed=9)
    mu, om = oracle.gl_nodes(P.n_mu)
    gbar = syn.random_cotangent(P.n_late, P.n_prim, seed=1)
    dqt, dq = oracle.backward(P, gbar)
    rng = np.random.default_rng(2)

    def loss(Pm):
        return float((gbar * oracle.separable(Pm)).sum())

    for _ in range(6):
        x, p, l = (int(rng.integers(P.n_x)), int(rng.integers(P.nb_prim)), int(rng.integers(P.L)))
        h = 1e-6 * max(abs(P.qt[x, p, l]), 1e-3)
        Pp = syn.Problem(**{**P.__dict__, "qt": P.qt.copy()})
        Pm = syn.Problem(**{**P.__dict__, "qt": P.qt.copy()})
        Pp.qt[x, p, l] += h
        Pm.qt[x, p, l] -= h
        fd = (loss(Pp) - loss(Pm)) / (2 * h)
        assert dqt[x, p, l] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dqt).max())
    for _ in range(4):
        a, l = int(rng.integers(P.nb_late)), int(rng.integers(P.L))
        h = 1e-6 * max(abs(P.q[a, l]), 1e-3)
        Pp = syn.Problem(**{**P.__dict__, "q": P.q.copy()})
        Pm = syn.Problem(**{**P.__dict__, "q": P.q.copy()})
        Pp.q[a, l] += h
        Pm.q[a, l] -= h
        fd = (loss(Pp) - loss(Pm)) / (2 * h)
        assert dq[a, l] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dq).max())


def test_backward_linearity_in_cotangent():
    P = syn.make_problem(10, 2, 2, seed=1)
    g1 = syn.random_cotangent(P.n_late, P.n_prim, seed=1)
    g2 = syn.random_cotangent(P.n_late, P.n_prim, seed=2)
    a1, _ = oracle.backward(P, g1, want_dq=False)
    a2, _ = oracle.backward(P, g2, want_dq=False)
    a3, _ = oracle.backward(P, 2 * g1 - g2, want_dq=False)
    assert np.allclose(a3, 2 * a1 - a2, rtol=1e-12, atol=1e-12 * np.abs(a1).max())


def test_M_table_matches_library_legendre():
    """P_{ii'} of Eq. legendre from the oracle equals the same sum formed with
    numpy's legval for P_l (a library routine)."""
    P = syn.make_problem(16, 3, 4, seed=12, nb_prim=2)
    mu, _ = oracle.gl_nodes(P.n_mu)
    M = oracle.M_table(P, mu)
    ls = np.arange(P.l_min, P.l_max + 1)
    Pl = np.array([[npleg.legval(m, np.eye(P.l_max + 1)[l]) for l in ls] for m in mu])
    ref = np.einsum("jl,l,al,xpl->xjap", Pl, P.w_l, P.q, P.qt)
    assert np.abs(M - ref).max() / np.abs(ref).max() < 1e-13


def _magnitude_sum_numpy(P, mu, om, xw):
    """The error-scale projection by plain numpy loops, independent of the
    oracle's C code: 1/(48 pi) sum_x |W_x| sum_j |om_j| sum over the six
    assignments sigma of |M_a sigma(p) M_b sigma(r) M_c sigma(s)|."""
    ls = np.arange(P.l_min, P.l_max + 1)
    Pl = npleg.legvander(mu, P.l_max)[:, ls]                  # [j][l]
    M = np.einsum("l,jl,al,xpl->xjap", P.w_l, Pl, P.q, P.qt)    # [x][j][a][p]
    g = np.zeros((P.n_late, P.n_prim))
    for n, (a, b, c) in enumerate(P.late_modes):
        for m, prs in enumerate(P.prim_modes):
            t = 0.0
            for s in itertools.permutations(prs):
                t = t + np.abs(M[:, :, a, s[0]] * M[:, :, b, s[1]] * M[:, :, c, s[2]])
            g[n, m] = np.sum(np.abs(xw)[:, None] * np.abs(om)[None, :] * t)
    return g / (48.0 * math.pi)


def test_error_scale_matches_brute_force():
    """The magnitude form of the separable sum (the per-entry rounding-error
    scale) equals a plain numpy evaluation on a tiny problem, bounds |Gamma'|
    entrywise, ignores a sign flip of q~ and is cubic in its scale."""
    P = syn.make_problem(10, 3, 3, seed=17)
    mu, om = oracle.gl_nodes(P.n_mu)
    xw = oracle.x_weights(P.x)
    ga = oracle.separable(P, magnitudes=True)
    ref = _magnitude_sum_numpy(P, mu, om, xw)
    assert np.allclose(ga, ref, rtol=1e-12, atol=0)
    g = oracle.separable(P)
    assert np.all(np.abs(g) <= ga * (1 + 1e-12))
    assert np.abs(g).max() < ga.max()            # cancellation happens somewhere
    Pn = syn.Problem(**{**P.__dict__, "qt": -2.0 * P.qt})
    assert np.allclose(oracle.separable(Pn, magnitudes=True), 8.0 * ga, rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# 11. Gram matrix <Q_n, Q_r> and the full Gamma = <Q,Q>^{-1} Gamma' (Appendix A)
# --------------------------------------------------------------------------

def brute_force_gram(l_min, l_max, q, v, modes):
    """<Q_n, Q_r> over the whole cube straight from Appendix A:
    sum (h/(v1 v2 v3))^2 Q_n Q_r with Q_n = 1/6 sum_perm q q q."""
    ls = range(l_min, l_max + 1)
    G = np.zeros((len(modes), len(modes)))
    for l1, l2, l3 in itertools.product(ls, repeat=3):
        tj = float(threej_factorial_exact(l1, l2, l3))
        if tj == 0.0:
            continue
        k = (l1 - l_min, l2 - l_min, l3 - l_min)
        h2 = (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi) * tj
        vv = v[k[0]] * v[k[1]] * v[k[2]]
        Q = np.array([sum(q[pa, k[0]] * q[pb, k[1]] * q[pc, k[2]]
                          for pa, pb, pc in itertools.permutations(m)) / 6.0 for m in modes])
        G += h2 / vv ** 2 * np.outer(Q, Q)
    return G


def test_gram_brute_force_tiny():
    """oracle.gram with w_gram = (2l+1)/v_l^2 equals the inner-product
    definition summed over every ordered (l1, l2, l3)."""
    rng = np.random.default_rng(21)
    l_min, l_max, nb = 2, 7, 3
    ls = np.arange(l_min, l_max + 1)
    q = rng.standard_normal((nb, ls.size))
    v = (2 * ls + 1.0) ** (1 / 6)
    modes = syn.mode_list(nb)
    P = syn.Problem(l_min=l_min, l_max=l_max, nb_late=nb, nb_prim=nb, n_x=1, q=q,
                    qt=q[None].copy(), w_l=np.ones(ls.size), x=np.zeros(1), phi=np.zeros(nb),
                    late_modes=modes, prim_modes=modes)
    ref = brute_force_gram(l_min, l_max, q, v, modes.tolist())
    g = oracle.gram(P, (2 * ls + 1.0) / v ** 2)
    assert np.abs(g - ref).max() / np.abs(ref).max() < 1e-13


def test_gram_symmetric_positive_definite():
    P = syn.cpu_size()
    g = oracle.gram(P, syn.gram_weights(P.l_min, P.l_max))
    assert np.abs(g - g.T).max() / np.abs(g).max() < 1e-14
    assert np.linalg.eigvalsh(g).min() > 0.0
    # a mode list with a repeated mode is singular: its Cholesky must fail
    late = np.concatenate([P.late_modes, P.late_modes[3:4]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.full_gamma(oracle.gram(P, syn.gram_weights(P.l_min, P.l_max), late=late),
                          np.eye(late.shape[0]))


def test_full_gamma_is_identity_when_projected_basis_is_late_basis():
    """With q~(l, x) = q(l) at one radial point of unit weight and the Gram
    weights as l weights, Q~' = Q, so Gamma' = <Q,Q> and Gamma = I.  Gamma'
    comes from the separable form (Eq. 2D), the Gram matrix from the direct
    sum: the two routes and the solve must agree."""
    P0 = syn.cpu_size()
    wg = syn.gram_weights(P0.l_min, P0.l_max)
    P = syn.Problem(**{**P0.__dict__, "qt": P0.q[None].copy(), "n_x": 1, "x": np.zeros(1),
                       "w_l": wg})
    gp = oracle.separable(P, xw=np.ones(1))
    G = oracle.gram(P, wg)
    assert np.abs(gp - G).max() / np.abs(G).max() < 1e-12
    cond = np.linalg.cond(G)
    gam = oracle.full_gamma(G, gp)
    assert np.abs(gam - np.eye(P.n_late)).max() < 1e-15 * cond


def test_full_gamma_backward_error_and_scaling():
    """The solve's backward error is at rounding level, and Gamma scales as
    Gamma' / (scale of the Gram matrix)."""
    P = syn.cpu_size()
    G = oracle.gram(P, syn.gram_weights(P.l_min, P.l_max))
    gp = oracle.separable(P)
    X = oracle.full_gamma(G, gp)
    r = np.abs(G @ X - gp).max() / (np.abs(G).max() * np.abs(X).max())
    assert r < 1e-13
    X2 = oracle.full_gamma(4.0 * G, gp)
    assert np.allclose(X2, X / 4.0, rtol=1e-12, atol=1e-12 * np.abs(X).max())


# --------------------------------------------------------------------------
# 12. Radial integrators on the synthetic tables (Section 3.2.4, accuracy study)
# --------------------------------------------------------------------------

def _unit_rmse_pct(g, ref):
    """Relative RMS error in percent of the unit-normalised Gamma' (Frobenius
    norm 1): 100 |G/|G| - R/|R||_F."""
    u = lambda a: a / np.sqrt((a ** 2).sum())
    return 100.0 * float(np.sqrt(((u(g) - u(ref)) ** 2).sum()))


def test_integrator_convergence_on_synthetic_tables():
    """Gamma' (l_max 48, 5 functions) with x resampled on 54..432 points
    against the Hermite rule on 1768 points (the sample size of the paper's
    reference): the trapezium rule converges at second order (x4 per
    doubling), the Hermite rule -- the trapezium sum plus the end-derivative
    correction from forward differences -- at third order or better, and is
    the more accurate from 108 points on."""
    def gam(nx, kind):
        P = syn.make_problem(48, 5, nx)
        return oracle.separable(P, xw=oracle.x_weights(P.x, kind))
    ref = gam(1768, oracle.HERMITE)
    ns = (54, 108, 216, 432)
    et = [_unit_rmse_pct(gam(n, oracle.TRAPEZOID), ref) for n in ns]
    eh = [_unit_rmse_pct(gam(n, oracle.HERMITE), ref) for n in ns]
    for a, b in zip(et, et[1:]):
        assert 3.5 < a / b < 4.5
    for a, b in zip(eh, eh[1:]):
        assert a / b > 7.0
    assert all(h < t for h, t in zip(eh[1:], et[1:]))


def test_smooth_weights_improve_with_grid_density():
    """The SMOOTH sparse-grid form (1/2 Gosper 3j^2, triangle only, midpoint
    cells) is an approximation (parity unpinned): here only its trend is
    checked -- at l_max 160 a grid with step 2 above l = 20 is more than ten
    times closer to the dense Gamma' than one with step 16."""
    P = syn.make_problem(160, 3, 4)
    dense = oracle.separable(P)
    u = lambda a: a / np.sqrt((a ** 2).sum())
    err = []
    for step in (16, 2):
        g, dw = syn.stepped_l_grid(160, step, dense_to=20)
        err.append(np.sqrt(np.mean((u(oracle.direct(P, g, dw, oracle.SMOOTH)) - u(dense)) ** 2)))
    assert err[1] < err[0] / 10


def test_gram_delta_basis_closed_forms():
    """Gram matrices of delta-function bases in closed form (Eq. 2D with
    q~ := q, the Gaunt integral of Section 2.2 and tabulated 3j values, Gram
    weight (2l+1)^(2/3)):
      one function at l = 2, mode (000):
        1/(48 pi) * 6 * (5^(2/3))^3 * 2 (2 2 2;000)^2 = 6*25*2*(2/35)/(48 pi) = 5/(14 pi);
      functions at l = 2, 4, mode (001) with itself: perm = 2 M_00^2 M_11, so
        1/(48 pi) * 2 * 5^(4/3) * 9^(2/3) * 2 (2 2 4;000)^2, (2 2 4;000)^2 = 2/35."""
    def problem(ls):
        l_min, l_max = 2, 6
        L = l_max - l_min + 1
        q = np.zeros((len(ls), L))
        for a, l in enumerate(ls):
            q[a, l - l_min] = 1.0
        modes = syn.mode_list(len(ls))
        return syn.Problem(l_min=l_min, l_max=l_max, nb_late=len(ls), nb_prim=len(ls), n_x=1, q=q,
                           qt=q[None].copy(), w_l=np.ones(L), x=np.zeros(1), phi=np.zeros(len(ls)),
                           late_modes=modes, prim_modes=modes)
    P = problem([2])
    g = oracle.gram(P, syn.gram_weights(2, 6))
    assert g[0, 0] == pytest.approx(5.0 / (14.0 * math.pi), rel=1e-13)
    P = problem([2, 4])
    g = oracle.gram(P, syn.gram_weights(2, 6), late=np.array([[0, 0, 1]], dtype=np.int32))
    expect = 2.0 * 5.0 ** (4.0 / 3.0) * 9.0 ** (2.0 / 3.0) * 2.0 * (2.0 / 35.0) / (48.0 * math.pi)
    assert g[0, 0] == pytest.approx(expect, rel=1e-13)


def test_mode_order_follows_the_appendix_example():
    """The n -> ijk map of the input generator starts as in Appendix A's
    example (000, 001, 011, 111, 002, 012, ...), lists each sorted triple
    once, and has C(nb+2, 3) modes."""
    m = syn.mode_list(4)
    assert [tuple(r) for r in m[:6]] == [(0, 0, 0), (0, 0, 1), (0, 1, 1), (1, 1, 1), (0, 0, 2), (0, 1, 2)]
    for nb in (1, 5, 20):
        m = syn.mode_list(nb)
        assert m.shape == (math.comb(nb + 2, 3), 3)
        assert all(a <= b <= c < nb for a, b, c in m)
        assert len({tuple(r) for r in m}) == m.shape[0]


def brute_force_direct_grid(P, grid, dw, xw, weight):
    """Eq. 3D on a multipole grid, literally: the ordered cube of grid points,
    (1/(144 pi)) dw1 dw2 dw3 w1 w2 w3 H(l1,l2,l3) [sum_perm q q q]
    [sum_x W_x sum_perm q~ q~ q~]."""
    G = np.zeros((P.n_late, P.n_prim))
    for (i1, l1), (i2, l2), (i3, l3) in itertools.product(list(enumerate(grid)), repeat=3):
        H = weight(l1, l2, l3)
        if H == 0.0:
            continue
        k = (l1 - P.l_min, l2 - P.l_min, l3 - P.l_min)
        wgt = dw[i1] * dw[i2] * dw[i3] * P.w_l[k[0]] * P.w_l[k[1]] * P.w_l[k[2]] * H / (144.0 * math.pi)
        Q = np.array([sum(P.q[a, k[0]] * P.q[b, k[1]] * P.q[c, k[2]]
                          for a, b, c in itertools.permutations(m)) for m in P.late_modes])
        Qt = np.array([sum(xw[x] * sum(P.qt[x, a, k[0]] * P.qt[x, b, k[1]] * P.qt[x, c, k[2]]
                                       for a, b, c in itertools.permutations(m))
                           for x in range(P.n_x)) for m in P.prim_modes])
        G += wgt * np.outer(Q, Qt)
    return G


@pytest.mark.parametrize("mode", ["exact", "smooth"])
def test_direct_sparse_grid_formula_brute_force(mode):
    """The sparse-grid direct sum (reading of the unstated weights: EXACT =
    exact 3j^2 with triangle and parity, SMOOTH = 1/2 Gosper 3j^2 with the
    triangle only, both times prod dw) equals the literal cube sum above on a
    stepped grid.  This pins the oracle's SMOOTH formula; how well SMOOTH
    approximates the dense sum stays unpinned (an approximation)."""
    P = syn.make_problem(30, 2, 2, seed=13)
    grid, dw = syn.stepped_l_grid(30, 3, dense_to=10)
    xw = oracle.x_weights(P.x)
    if mode == "exact":
        weight, wm = oracle.threej000_sq, oracle.EXACT
    else:
        weight, wm = (lambda a, b, c: 0.5 * oracle.gosper_threej000_sq(a, b, c)), oracle.SMOOTH
    ref = brute_force_direct_grid(P, grid, dw, xw, weight)
    got = oracle.direct(P, l_grid=grid, l_dw=dw, weight_mode=wm, xw=xw)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
