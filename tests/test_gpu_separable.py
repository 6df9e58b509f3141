"""GPU parity of the separable path (rows a1-a7) against the FP64 oracle,
called through the C ABI.  FP64 tolerance: 1e-10 normwise
(max |dGamma| / max |Gamma_ref|), the accuracy required of the FP64 path."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from tests._golden import delta_cases

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 2e-5


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


# ---- a1: Gauss-Legendre nodes ----------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 24, 31, 32, 33, 73, 1501, 3001, 6400])
def test_gl_nodes_parity(mg, n):
    mu, om = mg.gl_nodes(n)
    mo, oo = oracle.gl_nodes(n) if n > 1 else (np.zeros(1), np.full(1, 2.0))
    mu, om = mu.cpu().numpy(), om.cpu().numpy()
    assert np.abs(mu - mo).max() <= 4.5e-16           # two ulp of 1
    assert np.abs(om / oo - 1).max() <= 4e-15
    assert abs(om.sum() - 2.0) < 1e-13
    assert np.array_equal(mu, -mu[::-1])


# ---- a2: weighted Legendre table -------------------------------------------
def test_legendre_table_parity(mg):
    P = syn.planck_size(n_x=2)
    mu, _ = oracle.gl_nodes(P.n_mu)
    A = mg.legendre_table(torch.tensor(mu, device="cuda"), P.l_min, P.l_max,
                          torch.tensor(P.w_l, device="cuda")).cpu().numpy()
    ref = np.stack([oracle.legendre_row(P.l_max, m)[P.l_min:] * P.w_l for m in mu[::97]])
    got = A[::97]
    # Both sides run the FP64 forward recurrence; at l = 2000 that recurrence is
    # itself only good to ~3e-12 absolute (|P_l| <= 1, measured against
    # arbitrary-precision values), so two independent roundings differ by up
    # to ~2x that.
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-11


# ---- a3: radial weights ----------------------------------------------------
@pytest.mark.parametrize("kind", [0, 1])
def test_x_weights_parity(mg, kind):
    x = np.sort(np.random.default_rng(3).uniform(13000, 14500, 57))
    w = mg.x_weights(torch.tensor(x, device="cuda"), kind).cpu().numpy()
    ref = oracle.x_weights(x, kind)
    assert np.abs(w - ref).max() / np.abs(ref).max() < 1e-14


# ---- a5: l contraction -------------------------------------------------------
@pytest.mark.parametrize("shape", [(48, 5, 5, 24), (37, 7, 3, 13), (130, 2, 9, 5)])
def test_contract_l_parity(mg, shape):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=5, nb_prim=nbp)
    mu, _ = oracle.gl_nodes(P.n_mu)
    dp = mg.DeviceProblem.from_host(P)
    A = mg.legendre_table(torch.tensor(mu, device="cuda"), P.l_min, P.l_max, dp.w_l)
    M = mg.contract_l(dp, P.n_mu, A).cpu().numpy()
    ref = oracle.M_table(P, mu)
    assert M.shape == ref.shape
    assert np.abs(M - ref).max() / np.abs(ref).max() < 1e-13


# ---- the whole separable path ---------------------------------------------
def test_separable_cpu_size_fp64(mg):
    P = syn.cpu_size()
    g = mg.project_separable(mg.DeviceProblem.from_host(P))
    ref = oracle.separable(P)
    assert normwise(g, ref) < TOL_FP64
    # and the direct (non-separable) oracle, the exact definition
    assert normwise(g, oracle.direct(P)) < TOL_FP64


@pytest.mark.parametrize("x_chunk", [0, 5])
def test_separable_ragged_tiles(mg, x_chunk):
    """Sizes that leave ragged tails in every tile dimension, unequal bases,
    several radial chunks (K split + FP64 reduction of the partials)."""
    P = syn.make_problem(37, 7, 13, seed=8, nb_prim=3)
    g = mg.project_separable(mg.DeviceProblem.from_host(P), x_chunk=x_chunk)
    assert normwise(g, oracle.separable(P)) < TOL_FP64


def test_separable_many_tiles(mg):
    """12 late x 11 primordial functions: 364 x 286 Gamma, G spans many tiles."""
    P = syn.make_problem(60, 12, 7, seed=9, nb_prim=11)
    g = mg.project_separable(mg.DeviceProblem.from_host(P))
    assert normwise(g, oracle.separable(P)) < TOL_FP64


@pytest.mark.parametrize("case", list(delta_cases()), ids=lambda c: c[0])
def test_separable_golden(mg, case):
    name, P, expected = case
    dp = mg.DeviceProblem.from_host(P, x_w=np.ones(1))
    g = float(mg.project_separable(dp)[0, 0])
    assert g == pytest.approx(expected, rel=1e-13, abs=1e-15 / (70 * math.pi))


def test_separable_arbitrary_mode_lists(mg):
    """Unsorted and repeated-index triples, a subset of modes, in any order."""
    P = syn.make_problem(30, 4, 6, seed=10)
    rng = np.random.default_rng(4)
    late = np.array([rng.permutation(m) for m in P.late_modes[rng.permutation(20)[:9]]])
    prim = np.array([rng.permutation(m) for m in P.prim_modes[::-1][:13]])
    P.late_modes, P.prim_modes = late.astype(np.int32), prim.astype(np.int32)
    g = mg.project_separable(mg.DeviceProblem.from_host(P))
    assert g.shape == (9, 13)
    assert normwise(g, oracle.separable(P)) < TOL_FP64


def test_separable_fp32(mg):
    P = syn.cpu_size()
    g = mg.project_separable(mg.DeviceProblem.from_host(P), precision=mg.PREC_FP32)
    assert normwise(g, oracle.separable(P)) < TOL_FP32


def test_separable_inexact_gl_rejected_then_allowed(mg):
    P = syn.cpu_size()
    dp = mg.DeviceProblem.from_host(P)
    with pytest.raises(mg.ModalError) as ei:
        mg.project_separable(dp, n_mu=40)
    assert ei.value.code == 1 and "n_mu" in str(ei.value)
    g = mg.project_separable(dp, n_mu=40, allow_inexact_gl=True)
    assert normwise(g, oracle.separable(P, n_mu=40)) < TOL_FP64
    assert normwise(g, oracle.direct(P)) > 1e-9     # and it really is inexact


def test_separable_edge_cases(mg):
    P = syn.make_problem(12, 2, 3, seed=1)
    dp = mg.DeviceProblem.from_host(P)
    # no radial points: Gamma' = 0
    dp0 = mg.DeviceProblem(P.q, P.qt[:0], P.w_l, np.zeros(0), P.late_modes, P.prim_modes,
                           P.l_min, P.l_max)
    assert torch.count_nonzero(mg.project_separable(dp0)) == 0
    # no modes: nothing to do, no error
    dpe = mg.DeviceProblem(P.q, P.qt, P.w_l, dp.x_w, P.late_modes[:0], P.prim_modes, P.l_min,
                           P.l_max)
    assert mg.project_separable(dpe).shape == (0, P.n_prim)
    # a mode index outside the basis gives NaN in that row only
    bad = P.late_modes.copy()
    bad[1, 2] = 7
    dpb = mg.DeviceProblem(P.q, P.qt, P.w_l, dp.x_w, bad, P.prim_modes, P.l_min, P.l_max)
    g = mg.project_separable(dpb).cpu().numpy()
    assert np.isnan(g[1]).all() and np.isfinite(np.delete(g, 1, axis=0)).all()
    # single basis function, single x point, l_max = l_min
    P1 = syn.make_problem(2, 1, 1, seed=2)
    g1 = mg.project_separable(mg.DeviceProblem.from_host(P1, x_w=np.ones(1)))
    assert normwise(g1, oracle.separable(P1, xw=np.ones(1))) < TOL_FP64


def test_batched_matches_single(mg):
    probs = [syn.make_problem(l, nb, nx, seed=s)
             for l, nb, nx, s in [(20, 3, 5, 1), (33, 5, 9, 2), (12, 2, 4, 3), (48, 4, 7, 4)]]
    dps = [mg.DeviceProblem.from_host(P) for P in probs]
    gs = mg.project_separable_batched(dps)
    for P, g in zip(probs, gs):
        assert normwise(g, oracle.separable(P)) < TOL_FP64


def test_planck_size_sampled_entries(mg):
    """Full Planck-scale problem (l_max 2000, 20 functions, 500 x, N_mu 3001)
    in FP64, as the benchmark times it; 100 entries checked against the
    oracle (rows/columns whose basis indices lie in {0, 7, 19} x {2, 11, 16})."""
    P = syn.planck_size()
    g = mg.project_separable(mg.DeviceProblem.from_host(P)).cpu().numpy()
    late_pick = np.array([i for i, m in enumerate(P.late_modes) if set(m) <= {0, 7, 19}])
    prim_pick = np.array([i for i, m in enumerate(P.prim_modes) if set(m) <= {2, 11, 16}])
    ref = oracle.separable(P, late=P.late_modes[late_pick], prim=P.prim_modes[prim_pick])
    got = g[np.ix_(late_pick, prim_pick)]
    assert np.abs(got - ref).max() / np.abs(ref).max() < TOL_FP64
    assert np.isfinite(g).all()
