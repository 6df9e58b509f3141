"""GPU parity of the two FP32-accumulation forms of the l contraction on
tcgen05 (MODAL_PREC_TF32: operands rounded to TF32, one product;
MODAL_PREC_BF16X3: BF16 hi/lo operands, three products), against the FP64
oracle.

M is checked entry by entry against the rounding-error bound of its sum,
|dM| <= tol * sum_l |w_l q_a(l) q~_p(l,x)| (|P_l(mu)| <= 1), the scale taken
from the oracle's P_ii' table of the same problem with every table in
magnitude at mu = 1 (where P_l = 1).  tol: two operand roundings plus FP32
accumulation of L terms -- TF32: 2 * 2^-11 + L 2^-23; BF16x3: the hi/lo
representation and the dropped lo lo' product, 2^-16, plus the FP64 -> FP32
rounding of the operands (2 * 2^-24) and L 2^-23.  Gamma' (the FP32 triple
product over these M) is checked normwise at the tolerances stated below."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_GAMMA = {"tf32": 5e-3, "bf16x3": 1e-4}


def tol_M(form, L):
    return (2 * 2.0 ** -11 if form == "tf32" else 2.0 ** -16 + 2 * 2.0 ** -24) + L * 2.0 ** -23


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def prec_of(mg, form):
    return mg.PREC_TF32 if form == "tf32" else mg.PREC_BF16X3


def normwise(a, ref):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("form", ["tf32", "bf16x3"])
@pytest.mark.parametrize("shape", [(48, 5, 5, 24), (37, 7, 3, 13), (300, 9, 6, 3), (130, 4, 4, 9)])
def test_fa_contract_l(mg, form, shape):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=7, nb_prim=nbp)
    mu, _ = oracle.gl_nodes(P.n_mu)
    dp = mg.DeviceProblem.from_host(P)
    A = mg.legendre_table(torch.tensor(mu, device="cuda"), P.l_min, P.l_max, dp.w_l)
    M = mg.contract_l(dp, P.n_mu, A, precision=prec_of(mg, form))
    mg.handle_status()
    ref = oracle.M_table(P, mu)
    Pabs = dataclasses.replace(P, q=np.abs(P.q), qt=np.abs(P.qt), w_l=np.abs(P.w_l))
    S = oracle.M_table(Pabs, np.ones(1))            # [n_x][1][nbl][nbp]: sum_l |w q q~|
    d = np.abs(M.cpu().numpy() - ref)
    L = P.l_max - P.l_min + 1
    assert (d <= tol_M(form, L) * S).all()
    assert normwise(M, ref) > 0.0                   # the reduced-precision form really ran


@pytest.mark.parametrize("form", ["tf32", "bf16x3"])
@pytest.mark.parametrize("shape,x_chunk", [((48, 5, 5, 24), 0), ((37, 7, 3, 13), 5), ((60, 12, 11, 7), 0)])
def test_fa_separable(mg, form, shape, x_chunk):
    lmax, nbl, nbp, nx = shape
    P = syn.make_problem(lmax, nbl, nx, seed=9, nb_prim=nbp)
    g = mg.project_separable(mg.DeviceProblem.from_host(P), precision=prec_of(mg, form), x_chunk=x_chunk)
    mg.handle_status()
    assert normwise(g, oracle.separable(P)) < TOL_GAMMA[form]


def test_fa_batched(mg):
    """Several problems of uneven size in one batched call in the TF32 form:
    each result equals the single-problem call and stays within its bound."""
    probs = [syn.make_problem(30 + 17 * i, 3 + i, 4 + 3 * i, seed=40 + i) for i in range(3)]
    dps = [mg.DeviceProblem.from_host(P) for P in probs]
    h = mg.Handle()
    outs = mg.project_separable_batched(dps, precision=mg.PREC_TF32, handle=h)
    mg.handle_status(handle=h)
    for P, dp, g in zip(probs, dps, outs):
        single = mg.project_separable(dp, precision=mg.PREC_TF32).cpu().numpy()
        assert normwise(g, single) < 1e-6
        assert normwise(g, oracle.separable(P)) < TOL_GAMMA["tf32"]
    h.close()


@pytest.mark.parametrize("form", ["tf32", "bf16x3"])
def test_fa_bounded_wait_status(mg, form):
    """A one-clock wait bound makes both the l contraction's and the tensor-core
    triple product's waits give up: the call reports MODAL_ETIMEOUT through
    its single status word, and the next call with the default bound is
    right."""
    P = syn.make_problem(30, 4, 5, seed=12)
    dp = mg.DeviceProblem.from_host(P)
    h = mg.Handle()
    mg.set_wait_limit(1, handle=h)
    mg.project_separable(dp, precision=prec_of(mg, form), handle=h)
    with pytest.raises(mg.ModalError) as ei:
        mg.handle_status(handle=h)
    assert ei.value.code == 4        # MODAL_ETIMEOUT
    mg.set_wait_limit(0, handle=h)
    g = mg.project_separable(dp, precision=prec_of(mg, form), handle=h)
    mg.handle_status(handle=h)
    assert normwise(g, oracle.separable(P)) < TOL_GAMMA[form]
    h.close()
