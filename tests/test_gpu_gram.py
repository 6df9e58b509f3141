"""GPU parity of the Gram matrix <Q_n, Q_r> and the full Gamma =
<Q,Q>^{-1} Gamma' (Appendix A), called through the C ABI (modal_gram,
modal_gram_solve) and compared with the oracle on the same inputs.

Tolerances: the Gram matrix as the separable projection (FP64 1e-10,
tensor-core form 1e-8, FP32 2e-5 normwise).  The solve is checked by its
backward error max|G X - R| / (max|G| max|X|) <= 1e-13, which does not depend
on the conditioning, and by its forward error against scipy on the same
inputs, bounded by 10 cond(G) eps (cond(G) ~ 4e7 at l_max = 48, 5 functions).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def backward_error(G, X, R):
    return float(np.abs(G @ X - R).max() / (np.abs(G).max() * np.abs(X).max()))


def spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return B @ B.T / n + np.eye(n)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5), (2, 1e-8)])
def test_gram_matches_oracle(mg, precision, tol):
    P = syn.cpu_size()
    wg = syn.gram_weights(P.l_min, P.l_max)
    h = mg.Handle()
    G = mg.gram(mg.DeviceProblem.from_host(P, handle=h), wg, precision=precision, handle=h)
    if precision == 2:
        mg.handle_status(handle=h)
    ref = oracle.gram(P, wg)
    assert normwise(G, ref) < tol
    Gh = G.cpu().numpy()
    assert np.array_equal(Gh, Gh.T)          # symmetrised
    h.close()


def test_gram_error_estimate_symmetric(mg):
    P = syn.make_problem(20, 4, 3, seed=5)
    wg = syn.gram_weights(P.l_min, P.l_max)
    dp = mg.DeviceProblem.from_host(P)
    est = torch.empty(P.n_late, P.n_late, dtype=torch.float64, device=dp.device)
    G = mg.gram(dp, wg, error_estimate=est)
    E = est.cpu().numpy()
    assert np.array_equal(E, E.T)
    assert np.all(np.abs(G.cpu().numpy()) <= E * (1 + 1e-12))


@pytest.mark.parametrize("n,m", [(1, 1), (35, 35), (64, 37), (65, 130), (200, 1), (301, 64)])
def test_gram_solve_random_spd(mg, n, m):
    """Blocked Cholesky + solves over several 64-blocks with ragged tails."""
    G = spd(n, seed=n)
    R = np.random.default_rng(n + 1).standard_normal((n, m))
    dev = torch.device("cuda")
    X = mg.gram_solve(torch.from_numpy(G).to(dev), torch.from_numpy(R).to(dev)).cpu().numpy()
    assert backward_error(G, X, R) < 1e-13
    ref = oracle.full_gamma(G, R)
    assert normwise(X, ref) < 10 * np.linalg.cond(G) * EPS


def test_gram_solve_in_place_and_factor_only(mg):
    n, m = 130, 20
    G = spd(n, seed=7)
    R = np.random.default_rng(8).standard_normal((n, m))
    dev = torch.device("cuda")
    Gd = torch.from_numpy(G).to(dev)
    Rd = torch.from_numpy(R).to(dev)
    X = mg.gram_solve(Gd, Rd, out=Rd)           # x aliases rhs
    assert X.data_ptr() == Rd.data_ptr()
    assert backward_error(G, X.cpu().numpy(), R) < 1e-13
    assert torch.equal(Gd.cpu(), torch.from_numpy(G))   # gram is not modified
    # m = 0: factor only, status still written
    X0, info = mg.gram_solve(Gd, torch.empty(n, 0, dtype=torch.float64, device=dev),
                             raise_if_not_pd=False)
    assert X0.shape == (n, 0) and int(info.item()) == 0


def test_gram_solve_reads_lower_triangle_only(mg):
    n = 100
    G = spd(n, seed=9)
    R = np.random.default_rng(10).standard_normal((n, 3))
    Gu = G.copy()
    Gu[np.triu_indices(n, 1)] = np.nan            # garbage above the diagonal
    X = mg.gram_solve(torch.from_numpy(Gu).cuda(), torch.from_numpy(R).cuda()).cpu().numpy()
    assert backward_error(G, X, R) < 1e-13


@pytest.mark.parametrize("where", [0, 70, 129])
def test_gram_solve_not_positive_definite(mg, where):
    """A non-positive pivot at any block (first, second, last) gives info = 1 +
    its index, NaN in x, and ModalError from the binding."""
    n = 130
    G = spd(n, seed=11)
    G[where, where] = -1.0 - np.abs(G[where]).sum()
    R = np.ones((n, 4))
    Gd, Rd = torch.from_numpy(G).cuda(), torch.from_numpy(R).cuda()
    X, info = mg.gram_solve(Gd, Rd, raise_if_not_pd=False)
    k = int(info.item())
    assert 1 <= k <= where + 1
    assert torch.isnan(X).all()
    with pytest.raises(mg.ModalError) as ei:
        mg.gram_solve(Gd, Rd)
    assert ei.value.code == 1 and "positive definite" in str(ei.value)
    # the next call on a good matrix is right
    X = mg.gram_solve(torch.from_numpy(spd(n, 12)).cuda(), Rd).cpu().numpy()
    assert backward_error(spd(n, 12), X, R) < 1e-13


@pytest.mark.parametrize("dup", [0, 5, 34])
def test_repeated_mode_is_singular(mg, dup):
    """A mode listed twice makes the Gram matrix singular: the pivot of the
    repeat (the last row) is rounding noise (~1e-16 of its diagonal) and is
    reported as info = n; a regular Gram matrix's smallest relative pivot is
    ~1e-2 at this size."""
    P = syn.cpu_size()
    P.late_modes = np.concatenate([P.late_modes, P.late_modes[dup:dup + 1]]).astype(np.int32)
    dp = mg.DeviceProblem.from_host(P)
    G = mg.gram(dp, syn.gram_weights(P.l_min, P.l_max))
    eye = torch.eye(P.n_late, dtype=torch.float64, device=G.device)
    X, info = mg.gram_solve(G, eye, raise_if_not_pd=False)
    assert int(info.item()) == P.n_late
    assert torch.isnan(X).all()
    with pytest.raises(mg.ModalError):
        mg.gram_solve(G, eye)


def test_full_gamma_cpu_size(mg):
    """project_full (Gamma', Gram, solve on the GPU) against the oracle's
    full Gamma from its own Gamma' and Gram."""
    P = syn.cpu_size()
    wg = syn.gram_weights(P.l_min, P.l_max)
    dp = mg.DeviceProblem.from_host(P)
    Gam = mg.project_full(dp, wg).cpu().numpy()
    Gref = oracle.gram(P, wg)
    ref = oracle.full_gamma(Gref, oracle.separable(P))
    assert normwise(Gam, ref) < 10 * np.linalg.cond(Gref) * EPS
    # tensor-core form: its Gamma' and Gram matrix are within 1e-8 of the
    # oracle's (tests above); the solve on them has a rounding-level backward
    # error (the forward error is cond(G) ~ 4e7 times larger than 1e-8 here)
    h = mg.Handle()
    gp = mg.project_separable(dp, precision=mg.PREC_OZAKI_BF16, handle=h)
    G = mg.gram(dp, wg, precision=mg.PREC_OZAKI_BF16, handle=h)
    mg.handle_status(handle=h)
    X = mg.gram_solve(G, gp, handle=h)
    assert backward_error(G.cpu().numpy(), X.cpu().numpy(), gp.cpu().numpy()) < 1e-13
    h.close()


def test_full_gamma_identity_special_case(mg):
    """q~(l, x) = q(l) at one unit-weight radial point with the Gram weights:
    Gamma' = <Q,Q>, so the full Gamma is the identity."""
    P0 = syn.cpu_size()
    wg = syn.gram_weights(P0.l_min, P0.l_max)
    P = syn.Problem(**{**P0.__dict__, "qt": P0.q[None].copy(), "n_x": 1, "x": np.zeros(1), "w_l": wg})
    dp = mg.DeviceProblem.from_host(P, x_w=torch.ones(1, dtype=torch.float64, device="cuda"))
    Gam = mg.project_full(dp, wg).cpu().numpy()
    cond = np.linalg.cond(oracle.gram(P, wg))
    assert np.abs(Gam - np.eye(P.n_late)).max() < 10 * cond * EPS


def test_gram_planck_size(mg):
    """l_max = 2000, 20 functions (1540 modes): sampled Gram columns against
    the oracle's separable form (q~ := q, unit radial weight).  With this
    synthetic Legendre basis the Gram matrix is singular to working precision
    (the oracle's full matrix has a smallest eigenvalue of -1.5e-4 against a
    largest of 3.8e8), which the factorisation reports; the solve at n = 1540
    is checked on a well-conditioned SPD matrix of that size."""
    P = syn.planck_size(n_x=1)
    wg = syn.gram_weights(P.l_min, P.l_max)
    dp = mg.DeviceProblem.from_host(P)
    h = mg.Handle()
    G = mg.gram(dp, wg, handle=h).cpu().numpy()
    cols = np.array([0, 1, 37, 500, 1100, 1539])
    Pg = syn.Problem(**{**P.__dict__, "qt": P.q[None].copy(), "w_l": wg})
    ref = oracle.separable(Pg, xw=np.ones(1), prim=P.late_modes[cols])
    assert normwise(G[:, cols], ref) < 1e-10
    R = np.random.default_rng(3).standard_normal((P.n_late, 17))
    Rd = torch.from_numpy(R).cuda()
    _, info = mg.gram_solve(torch.from_numpy(G).cuda(), Rd, handle=h, raise_if_not_pd=False)
    assert int(info.item()) > 0
    S = spd(P.n_late, seed=13)
    X = mg.gram_solve(torch.from_numpy(S).cuda(), Rd, handle=h).cpu().numpy()
    assert backward_error(S, X, R) < 1e-13
    assert normwise(X, oracle.full_gamma(S, R)) < 10 * np.linalg.cond(S) * EPS
    h.close()


def test_gram_solve_empty(mg):
    dev = torch.device("cuda")
    X, info = mg.gram_solve(torch.empty(0, 0, dtype=torch.float64, device=dev),
                            torch.empty(0, 5, dtype=torch.float64, device=dev), raise_if_not_pd=False)
    assert X.shape == (0, 5) and int(info.item()) == 0
