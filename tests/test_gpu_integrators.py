"""GPU radial integrators (Section 3.2.4) on the synthetic tables: the error
curve of Gamma' -- relative RMS error of the unit-normalised matrix against
the Hermite rule on 1768 points -- matches the oracle's for both rules."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg(gpu):
    import paper_1503_08809_gb300 as mg
    return mg


def unit_rmse_pct(g, ref):
    u = lambda a: a / np.sqrt((a ** 2).sum())
    return 100.0 * float(np.sqrt(((u(g) - u(ref)) ** 2).sum()))


@pytest.mark.parametrize("kind", [0, 1], ids=["trapezium", "hermite"])
def test_integrator_error_curve_matches_oracle(mg, kind):
    Pr = syn.make_problem(48, 5, 1768)
    ref = oracle.separable(Pr, xw=oracle.x_weights(Pr.x, oracle.HERMITE))
    gref = mg.project_separable(mg.DeviceProblem.from_host(Pr, xw_kind=mg.XW_HERMITE)).cpu().numpy()
    assert np.abs(gref - ref).max() / np.abs(ref).max() < 1e-12
    for n in (27, 108, 432):
        P = syn.make_problem(48, 5, n)
        g = mg.project_separable(mg.DeviceProblem.from_host(P, xw_kind=kind)).cpu().numpy()
        e_gpu = unit_rmse_pct(g, gref)
        e_ora = unit_rmse_pct(oracle.separable(P, xw=oracle.x_weights(P.x, kind)), ref)
        assert abs(e_gpu - e_ora) <= 1e-2 * e_ora + 1e-11
